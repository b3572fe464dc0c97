// Closed-form prediction standard errors at every grid node (Section 3.4's
// SE_E, SE_L and SE_N; the variances of Eq. (condmvn), Section 3.1 and
// Section 3.2), without drawing a realization.
//
// Exact (local mode, A = K_oo + tau^2 I):
//   var_E(g) = sigma^2 - k_g^T A^-1 k_g,                k_g = K(obs, g).
// Approximate draws v = y + W_2 (z - S y - eps*), W_2 = K_go A^-1, where S is the
// off-grid map (W_1 rows in local mode, J_N in NN mode) and eps* has covariance D
// (diag phi^2, or the grid-box blocks L_b L_b^T):
//   var(g) = sigma^2 - 2 w_g^T u_g + w_g^T Q w_g,
//   w_g = A^-1 k_g,  u_g = S K(grid, g),  Q = S K_gg S^T + D.
// In NN mode S K_gg = K(J_N, grid) and Q = A_N, so var = sigma^2 - k_g^T A_N^-1 k_g
// with the context's surrogate nodes and prediction matrix.
//
// The nodes are processed in chunks of rows; per chunk k_g and u_g are formed
// (FP64 evaluation, FP32 storage), w_g = A^-1 k_g and Q w_g are the FP32 hi/lo
// products of the solve (Kahan-compensated), and the quadratic forms are summed
// per node in FP64.  Grid-to-grid covariances depend only on the lag, so u_g and
// Q read an m x (2m - 1) FP64 lag table.
#include <algorithm>
#include <cmath>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

struct SeGrid {
  int m;
  double h, sigma2, theta;
  int nu3;
  Aniso an;
};

// tab[a][b + m - 1] = C of the lag of a rows and b columns, 0 <= a < m, -m < b < m
// (C(-lag) = C(lag), so rows of negative lag are not stored).
__global__ void se_lag_table_kernel(SeGrid g, double* __restrict__ tab) {
  const int W = 2 * g.m - 1;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)g.m * W) return;
  const double a = (double)(e / W), b = (double)(e % W - (g.m - 1));
  tab[e] = matern_d(aniso_dist(g.h * b, g.h * a, g.an), g.sigma2, g.theta, g.nu3);
}

// Kc[r][i] = C(node g0 + r, obs i), obs in grid units (integer part, fraction).
__global__ void se_cross_kernel(SeGrid g, const float4* __restrict__ obs, int n, long long g0, int rows,
                                float* __restrict__ Kc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * n) return;
  const int r = (int)(e / n), i = (int)(e % n);
  const long long node = g0 + r;
  const double gi = (double)(node / g.m), gj = (double)(node % g.m);
  const float4 o = obs[i];
  const double dx = ((double)o.x - gj) + (double)o.y, dy = ((double)o.z - gi) + (double)o.w;
  Kc[e] = (float)matern_d(aniso_dist(g.h * dx, g.h * dy, g.an), g.sigma2, g.theta, g.nu3);
}

__device__ __forceinline__ double lag_cov(const double* __restrict__ tab, int m, int p, int q) {
  int di = p / m - q / m, dj = p % m - q % m;
  if (di < 0) { di = -di; dj = -dj; }
  return tab[di * (2 * m - 1) + dj + m - 1];
}

// Uc[r][i] = sum_k W[i][k] C(idx[i][k], node g0 + r)  (local mode).
__global__ void se_u_kernel(const double* __restrict__ tab, int m, const int* __restrict__ idx, const float* __restrict__ W,
                            int K, int n, long long g0, int rows, float* __restrict__ Uc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * n) return;
  const int r = (int)(e / n), i = (int)(e % n);
  const int node = (int)(g0 + r);
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += (double)W[(long long)i * K + k] * lag_cov(tab, m, idx[(long long)i * K + k], node);
  Uc[e] = (float)s;
}

// Q = S K_gg S^T + D (local mode), written as the FP32 pair hi + lo (rows of length ld).
// Q[i][j] = sum_k sum_l W[i][k] W[j][l] C(idx[i][k], idx[j][l]); D = diag(phi^2), or for
// two rows of one jointly drawn grid box the product of their noise-factor rows.
__global__ void se_q_kernel(const double* __restrict__ tab, int m, const int* __restrict__ idx, const float* __restrict__ W,
                            int K, int n, const float* __restrict__ phi, const int* __restrict__ box_cnt,
                            const int* __restrict__ box_mem, const float* __restrict__ box_L, int ld,
                            float* __restrict__ Qhi, float* __restrict__ Qlo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (j > i) return;
  double s = 0.0;
  for (int k = 0; k < K; ++k) {
    const double wi = (double)W[(long long)i * K + k];
    const int p = idx[(long long)i * K + k];
    double t = 0.0;
    for (int l = 0; l < K; ++l) t += (double)W[(long long)j * K + l] * lag_cov(tab, m, p, idx[(long long)j * K + l]);
    s += wi * t;
  }
  const int ci = box_cnt ? box_cnt[i] : 0, cj = box_cnt ? box_cnt[j] : 0;
  if (ci > 0 && cj > 0 && box_mem[(long long)i * kBoxMax] == box_mem[(long long)j * kBoxMax]) {
    const int c = min(ci, cj);
    for (int t = 0; t < c; ++t) s += (double)box_L[(long long)i * kBoxMax + t] * (double)box_L[(long long)j * kBoxMax + t];
  } else if (i == j) {
    s += (double)phi[i] * (double)phi[i];
  }
  const float hi = (float)s, lo = (float)(s - (double)hi);
  Qhi[(long long)i * ld + j] = hi;
  Qlo[(long long)i * ld + j] = lo;
  Qhi[(long long)j * ld + i] = hi;
  Qlo[(long long)j * ld + i] = lo;
}

// se[g0 + r] = sqrt(sigma^2 - sum_i Kc Wc)                        (Uc == nullptr)
//            = sqrt(sigma^2 - 2 sum_i Uc Wc + sum_i Wc Tc)         (otherwise); one warp per node.
__global__ void se_reduce_kernel(const float* __restrict__ Kc, const float* __restrict__ Uc, const float* __restrict__ Wc,
                                 const float* __restrict__ Tc, int n, int rows, double sigma2, long long g0,
                                 float* __restrict__ se) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const long long o = (long long)r * n;
  double s = 0.0;
  if (Uc) {
    for (int i = lane; i < n; i += 32) s += (double)Wc[o + i] * ((double)Tc[o + i] - 2.0 * (double)Uc[o + i]);
  } else {
    for (int i = lane; i < n; i += 32) s -= (double)Kc[o + i] * (double)Wc[o + i];
  }
  for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) se[g0 + r] = (float)sqrt(fmax(sigma2 + s, 0.0));
}

}  // namespace
}  // namespace ce

using namespace ce;

extern "C" int ce_se_map(ce_ctx* ctx, float* se_exact_dev, float* se_approx_dev, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (ctx->mode < 0) return fail(ctx, CE_ERR_STATE, "no off-grid set-up (ce_krige_weights first)");
  if (se_exact_dev && ctx->mode != CE_LOCAL) {
    return fail(ctx, CE_ERR_STATE, "the exact standard errors need the sites' own prediction matrix (local mode)");
  }
  if (ctx->trend_p > 0) return fail(ctx, CE_ERR_STATE, "the closed forms assume a zero mean (ce_set_trend -1 first)");
  if (!se_exact_dev && !se_approx_dev) return CE_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool local = ctx->mode == CE_LOCAL;
  const bool need_u = se_approx_dev && local;
  const int n = ctx->nobs, m = ctx->m, ld = ctx->nobs_pad;
  const long long M = (long long)m * m;
  // rows per chunk: the split-K partial products stay within about 256 MB
  const long long cap = std::max<long long>(32, (256ll << 20) / ((long long)kSolveKSplit * 8 * n)) / 32 * 32;
  const int Mc = (int)std::min<long long>(M, cap);
  const size_t chunk = (size_t)Mc * n;
  SeGrid g{m, ctx->h, ctx->sigma * ctx->sigma, ctx->range, ctx->nu == 1.5 ? 1 : 0,
           make_aniso(ctx->aniso_ratio, ctx->aniso_angle)};

  float* Kc = (float*)dalloc(ctx, sizeof(float) * chunk);
  float* Wc = (float*)dalloc(ctx, sizeof(float) * chunk);
  float* part = (float*)dalloc(ctx, sizeof(float2) * chunk * kSolveKSplit);   // (sum, compensation) pairs
  float *Uc = nullptr, *Tc = nullptr, *Qhi = nullptr, *Qlo = nullptr;
  double* tab = nullptr;
  if (need_u) {
    Uc = (float*)dalloc(ctx, sizeof(float) * chunk);
    Tc = (float*)dalloc(ctx, sizeof(float) * chunk);
    Qhi = (float*)dalloc(ctx, sizeof(float) * (size_t)n * ld);
    Qlo = (float*)dalloc(ctx, sizeof(float) * (size_t)n * ld);
    tab = (double*)dalloc(ctx, sizeof(double) * (size_t)m * (2 * m - 1));
  }
  auto release = [&]() {
    dfree(ctx, Kc); dfree(ctx, Wc); dfree(ctx, part); dfree(ctx, Uc); dfree(ctx, Tc);
    dfree(ctx, Qhi); dfree(ctx, Qlo); dfree(ctx, tab);
  };
  if (!Kc || !Wc || !part || (need_u && (!Uc || !Tc || !Qhi || !Qlo || !tab))) {
    release();
    return fail(ctx, CE_ERR_OOM, "standard-error work buffers");
  }
  if (need_u) {
    CE_CUDA_TRY(cudaMemsetAsync(Qhi, 0, sizeof(float) * (size_t)n * ld, s));
    CE_CUDA_TRY(cudaMemsetAsync(Qlo, 0, sizeof(float) * (size_t)n * ld, s));
    const long long ntab = (long long)m * (2 * m - 1);
    se_lag_table_kernel<<<(unsigned)((ntab + 255) / 256), 256, 0, s>>>(g, tab);
    const long long nn = (long long)n * n;
    const bool boxes = ctx->box_joint > 0;
    se_q_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(tab, m, ctx->idx, ctx->W, ctx->K, n, ctx->phi,
                                                             boxes ? ctx->box_cnt : nullptr, boxes ? ctx->box_mem : nullptr,
                                                             boxes ? ctx->box_L : nullptr, ld, Qhi, Qlo);
    ctx->launches += 2;
  }
  for (long long g0 = 0; g0 < M; g0 += Mc) {
    const int rows = (int)std::min<long long>(Mc, M - g0);
    const long long tot = (long long)rows * n;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    se_cross_kernel<<<blocks, 256, 0, s>>>(g, ctx->obs, n, g0, rows, Kc);
    launch_gemm_hilo(Kc, rows, n, ctx->Ainv_hi, ctx->Ainv_lo, ld, part, Wc, n, s, false);   // w_g = A^-1 k_g
    ctx->launches += 3;
    if (se_exact_dev || !local) {
      se_reduce_kernel<<<(rows + 7) / 8, 256, 0, s>>>(Kc, nullptr, Wc, nullptr, n, rows, g.sigma2, g0,
                                                      local ? se_exact_dev : se_approx_dev);
      ctx->launches += 1;
    }
    if (need_u) {
      se_u_kernel<<<blocks, 256, 0, s>>>(tab, m, ctx->idx, ctx->W, ctx->K, n, g0, rows, Uc);
      launch_gemm_hilo(Wc, rows, n, Qhi, Qlo, ld, part, Tc, n, s, false);                   // Q w_g
      se_reduce_kernel<<<(rows + 7) / 8, 256, 0, s>>>(nullptr, Uc, Wc, Tc, n, rows, g.sigma2, g0, se_approx_dev);
      ctx->launches += 4;
    }
  }
  CE_CUDA_TRY(cudaGetLastError());
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  release();
  return CE_OK;
}
