// Linear mean model (Section 2: z_i = mu(s_i) + y(s_i) + eps_i with
// mu(s) = x(s)^T beta and beta estimated by generalized least squares).
//
// The conditional draw becomes v = yhat(z) + y - yhat(z*) = y + yhat(z - z*)
// with the universal Kriging predictor
//   yhat(w) = X_g beta(w) + K_go A^-1 (w - X beta(w)),
//   beta(w) = G w,  G = (X^T A^-1 X)^-1 X^T A^-1 = S^-1 F^T,  F = A^-1 X.
// With E = z - z* (the residuals of step 4) and B = A^-1 E (the solve), per
// realization r:
//   beta_r = G e_r,   B_r <- B_r - F beta_r,   v_r += X_g beta_r,
// and the correction K_go B_r in between is unchanged.  The regressors are
// x(s) = [1] (degree 0) or [1, u, v] (degree 1), u, v the centred grid
// coordinates divided by m.  F and G are formed once in FP64 on the host from
// the stored inverse pair A^-1 = hi + lo; beta and the update of B are FP64.
#include <cmath>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

// beta[r][k] = sum_q G[k][q] E[r][q]; one block per realization.  Also the plane
// x_g^T beta_r = k0 + k1 j + k2 i at node (i, j) as FP32 coefficients kf[r] (formed in
// FP64): the field update then needs no FP64 arithmetic per node.
__global__ void trend_beta_kernel(const double* __restrict__ G, const float* __restrict__ E, int n, int p, int m,
                                  double* __restrict__ beta, float* __restrict__ kf) {
  const int r = blockIdx.x;
  __shared__ double part[3][8];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const double e = (double)E[(long long)r * n + q];
    for (int k = 0; k < p; ++k) acc[k] += G[(long long)k * n + q] * e;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < p; ++k) {
    double v = acc[k];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < p; ++k) {
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b[k] += part[k][i];
      beta[r * 3 + k] = b[k];
    }
    // u = (j - c) / m, v = (i - c) / m with c = (m - 1) / 2
    const double c = 0.5 * (m - 1);
    kf[r * 3 + 0] = (float)(b[0] - (b[1] + b[2]) * c / m);
    kf[r * 3 + 1] = (float)(b[1] / m);
    kf[r * 3 + 2] = (float)(b[2] / m);
  }
}

// B[r][q] <- B[r][q] - sum_k F[q][k] beta[r][k], in FP64 before rounding.
__global__ void trend_update_kernel(float* __restrict__ B, int ldb, const double* __restrict__ F, int n, int p, int R,
                                    const double* __restrict__ beta) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * n) return;
  const int r = (int)(e / n), q = (int)(e % n);
  double d = (double)B[(long long)r * ldb + q];
  for (int k = 0; k < p; ++k) d -= F[(long long)q * p + k] * beta[r * 3 + k];
  B[(long long)r * ldb + q] = (float)d;
}

// v[r][i][j] += beta_r . x(node (i, j)) = k0 + k1 j + k2 i (FP32).  grid.y = realization,
// grid.x covers the rows of the grid in 256-thread pieces of one row.
__global__ void trend_add_kernel(float* __restrict__ v, int m, int R, const float* __restrict__ kf) {
  const int r = blockIdx.y;
  const int per_row = (m + 255) / 256;
  const int i = blockIdx.x / per_row;
  const int j = (blockIdx.x % per_row) * 256 + threadIdx.x;
  if (i >= m || j >= m) return;
  const float k0 = __ldg(kf + 3 * r), k1 = __ldg(kf + 3 * r + 1), k2 = __ldg(kf + 3 * r + 2);
  float* vr = v + (long long)r * m * m + (long long)i * m;
  vr[j] += fmaf(k2, (float)i, fmaf(k1, (float)j, k0));
}

}  // namespace

void free_trend(ce_ctx* ctx) {
  dfree(ctx, ctx->trend_F); ctx->trend_F = nullptr;
  dfree(ctx, ctx->trend_G); ctx->trend_G = nullptr;
  dfree(ctx, ctx->trend_beta); ctx->trend_beta = nullptr;
  dfree(ctx, ctx->trend_kf); ctx->trend_kf = nullptr;
  ctx->trend_p = 0;
}

void launch_trend_solve(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s) {
  if (ctx->trend_p == 0) return;
  const int n = ctx->nobs;
  trend_beta_kernel<<<R, 256, 0, s>>>(ctx->trend_G, E, n, ctx->trend_p, ctx->m, ctx->trend_beta, ctx->trend_kf);
  const long long tot = (long long)R * n;
  trend_update_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, ldb, ctx->trend_F, n, ctx->trend_p, R,
                                                                      ctx->trend_beta);
  ctx->launches += 2;
}

void launch_trend_add(ce_ctx* ctx, int R, float* y, cudaStream_t s) {
  if (ctx->trend_p == 0) return;
  const int m = ctx->m;
  trend_add_kernel<<<dim3((unsigned)(m * ((m + 255) / 256)), (unsigned)R), 256, 0, s>>>(y, m, R, ctx->trend_kf);
  ctx->launches += 1;
}

}  // namespace ce

using namespace ce;

extern "C" int ce_set_trend(ce_ctx* ctx, int degree) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (degree < -1 || degree > 1) return fail(ctx, CE_ERR_ARG, "trend degree must be -1 (none), 0 or 1");
  if (ctx->mode != CE_LOCAL || !ctx->sites64 || !ctx->Ainv_hi) {
    return fail(ctx, CE_ERR_STATE, "the trend model needs local Kriging weights (ce_krige_weights with CE_LOCAL)");
  }
  free_trend(ctx);
  if (degree < 0) return CE_OK;
  const int p = degree == 0 ? 1 : 3;
  const int n = ctx->nobs, ld = ctx->nobs_pad, m = ctx->m;
  if (n <= p) return fail(ctx, CE_ERR_ARG, "the trend model needs more sites than regressors");
  cudaStream_t s = ctx->setup_stream;
  std::vector<double> xy(2 * (size_t)n);
  std::vector<float> hi((size_t)n * ld), lo((size_t)n * ld);
  CE_CUDA_TRY(cudaMemcpyAsync(xy.data(), ctx->sites64, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaMemcpyAsync(hi.data(), ctx->Ainv_hi, sizeof(float) * (size_t)n * ld, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaMemcpyAsync(lo.data(), ctx->Ainv_lo, sizeof(float) * (size_t)n * ld, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  // regressors at the sites (internal order)
  const double c = 0.5 * (m - 1);
  std::vector<double> X((size_t)n * p);
  for (int q = 0; q < n; ++q) {
    X[(size_t)q * p] = 1.0;
    if (p == 3) {
      X[(size_t)q * p + 1] = ((xy[2 * q] - ctx->x0) / ctx->h - c) / m;
      X[(size_t)q * p + 2] = ((xy[2 * q + 1] - ctx->y0) / ctx->h - c) / m;
    }
  }
  // F = A^-1 X (A^-1 symmetric, rows of length ld)
  std::vector<double> F((size_t)n * p, 0.0);
  for (int i = 0; i < n; ++i) {
    const float* h = hi.data() + (size_t)i * ld;
    const float* l = lo.data() + (size_t)i * ld;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < n; ++j) {
      const double a = (double)h[j] + (double)l[j];
      for (int k = 0; k < p; ++k) acc[k] += a * X[(size_t)j * p + k];
    }
    for (int k = 0; k < p; ++k) F[(size_t)i * p + k] = acc[k];
  }
  // S = X^T F (p x p, symmetric positive definite), Cholesky, G = S^-1 F^T
  double S[3][3] = {};
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      double t = 0.0;
      for (int q = 0; q < n; ++q) t += X[(size_t)q * p + a] * F[(size_t)q * p + b];
      S[a][b] = t;
    }
  double L[3][3] = {};
  for (int j = 0; j < p; ++j) {
    double d = S[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) return fail(ctx, CE_ERR_NOT_SPD, "X^T A^-1 X is not positive definite (collinear regressors)");
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < p; ++i) {
      double t = S[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  std::vector<double> G((size_t)p * n);
  for (int q = 0; q < n; ++q) {
    double w[3];
    for (int i = 0; i < p; ++i) {   // L w = F[q]
      double t = F[(size_t)q * p + i];
      for (int k = 0; k < i; ++k) t -= L[i][k] * w[k];
      w[i] = t / L[i][i];
    }
    for (int i = p - 1; i >= 0; --i) {   // L^T g = w
      double t = w[i];
      for (int k = i + 1; k < p; ++k) t -= L[k][i] * w[k];
      w[i] = t / L[i][i];
    }
    for (int k = 0; k < p; ++k) G[(size_t)k * n + q] = w[k];
  }
  ctx->trend_F = (double*)dalloc(ctx, sizeof(double) * (size_t)n * p);
  ctx->trend_G = (double*)dalloc(ctx, sizeof(double) * (size_t)p * n);
  ctx->trend_beta = (double*)dalloc(ctx, sizeof(double) * 3 * 4096);
  ctx->trend_kf = (float*)dalloc(ctx, sizeof(float) * 3 * 4096);
  if (!ctx->trend_F || !ctx->trend_G || !ctx->trend_beta || !ctx->trend_kf) {
    free_trend(ctx);
    return fail(ctx, CE_ERR_OOM, "trend model");
  }
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->trend_F, F.data(), sizeof(double) * (size_t)n * p, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->trend_G, G.data(), sizeof(double) * (size_t)p * n, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->trend_p = p;
  return CE_OK;
}
