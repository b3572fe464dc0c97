// Pathwise gradient of L = (1/R) sum_r mean_{g in W} v_r(g)^2 + l(theta, z) with
// respect to theta = (sigma, range, tau^2) and the data z, at fixed noise, for
// the local-Kriging conditional simulation (Section 2, Section 2.1) and the
// Gaussian log-likelihood l = -z^T A^-1 z / 2 - log det A / 2 - n log(2 pi) / 2
// of the model behind Eq. (condmvn), A = K_oo + tau^2 I.
//
// With g_r = dL/dv_r = 2 v_r 1_W / (R |W|), B_r = A^-1 (z - z*_r) and
// w_r = A^-1 K_og g_r (the adjoint of the correction), the forward
// v_r = y_r + K_go B_r, z*_r = W_1 y_r + phi eps*_r gives
//   dL/dz      = sum_r w_r - A^-1 z
//   dL/dtheta  = sum_r <g_r, dK_go B_r>                (through the correction)
//              + sum_ij dA_ij (a_i a_j / 2 - Ainv_ij / 2 - sum_r w_r,i B_r,j)
//                                                      (prediction matrix and l; a = A^-1 z)
//              - sum_r <w_r, dW_1 y_r + dphi eps*_r>   (off-grid weights and nugget)
//              + sum_r <h_r, dy_r>,  h_r = g_r - W_1^T w_r   (the unconditional fields)
// and the last term is evaluated per realization pair in Fourier space:
// <h_{2p}, d Re w> + <h_{2p+1}, d Im w> = sum_a ds_a Re(eps_a Y_a) with
// Y = DFT2(h_{2p} - i h_{2p+1}) and s = sqrt(lambda / N).
#include <cmath>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
int launch_adjoint_ensemble(ce_ctx* ctx, const float* H, int R, uint64_t seed, uint64_t r_offset, double* acc,
                            cudaStream_t s);
MaternF matern_grid_units(const ce_ctx* ctx);

namespace {

struct CovF {
  float s2, theta, h;   // sigma^2, range, grid spacing
  int nu3;
};

// C and d C / d theta at a distance given in grid units.
__device__ __forceinline__ void cov_and_dtheta(float dgrid, const CovF& k, float& c, float& dc) {
  const float d = dgrid * k.h;
  if (k.nu3) {
    const float t = 1.7320508f * d / k.theta;
    const float e = expf(-t);
    c = k.s2 * (1.0f + t) * e;
    dc = k.s2 * t * t * e / k.theta;
  } else {
    const float e = expf(-d / k.theta);
    c = k.s2 * e;
    dc = c * d / (k.theta * k.theta);
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;   // valid in thread 0
}

struct Window {
  int i0, i1, j0, j1;
};

// c[r][q] = f sum_{g in W} C(g, s_q) v_r(g) and, into acc[0..1], the correction
// term f sum_{g, q} (2 C / sigma, dC / dtheta)(g, q) sum_r v_r(g) B_r(q).
// Block: 32 sites (internal order) x a slice of the window nodes; 256 threads.
constexpr int GW_Q = 32, GW_G = 64;

__global__ void __launch_bounds__(256) grad_window_kernel(const float* __restrict__ v, int m, Window win, int R,
                                                          const float4* __restrict__ obs, int nobs,
                                                          const float* __restrict__ B, int ldb, CovF cov, float f,
                                                          float inv_sigma, float* __restrict__ c, double* __restrict__ acc) {
  extern __shared__ float gsm[];
  float* Bs = gsm;                        // [R][GW_Q]
  float* Vs = Bs + R * GW_Q;              // [R][GW_G]
  float* Cs = Vs + R * GW_G;              // [GW_Q][GW_G]
  float* Ds = Cs + GW_Q * GW_G;           // [GW_Q][GW_G]
  __shared__ double red[32];
  const int q0 = blockIdx.x * GW_Q;
  const int wj = win.j1 - win.j0;
  const long long nW = (long long)(win.i1 - win.i0) * wj;
  const long long per = (nW + gridDim.y - 1) / gridDim.y;
  const long long g_beg = blockIdx.y * per, g_end = min(nW, g_beg + per);
  const long long M = (long long)m * m;
  for (int e = threadIdx.x; e < R * GW_Q; e += blockDim.x) {
    const int r = e / GW_Q, qq = e % GW_Q;
    Bs[e] = (q0 + qq < nobs) ? B[(long long)r * ldb + q0 + qq] : 0.f;
  }
  const int tq = threadIdx.x % GW_Q, tr = threadIdx.x / GW_Q;   // 8 realization groups
  constexpr int RMAX = 16;                                        // R <= 128
  float cacc[RMAX];
#pragma unroll
  for (int k = 0; k < RMAX; ++k) cacc[k] = 0.f;
  double ks = 0.0, kt = 0.0;
  for (long long gb = g_beg; gb < g_end; gb += GW_G) {
    __syncthreads();
    for (int e = threadIdx.x; e < R * GW_G; e += blockDim.x) {
      const int r = e / GW_G, gg = e % GW_G;
      const long long gw = gb + gg;
      float val = 0.f;
      if (gw < g_end) {
        const int gi = win.i0 + (int)(gw / wj), gj = win.j0 + (int)(gw % wj);
        val = v[(long long)r * M + (long long)gi * m + gj];
      }
      Vs[e] = val;
    }
    for (int e = threadIdx.x; e < GW_Q * GW_G; e += blockDim.x) {
      const int qq = e / GW_G, gg = e % GW_G;
      const long long gw = gb + gg;
      float cv = 0.f, dv = 0.f;
      if (gw < g_end && q0 + qq < nobs) {
        const int gi = win.i0 + (int)(gw / wj), gj = win.j0 + (int)(gw % wj);
        const float4 s = obs[q0 + qq];
        const float dx = ((float)gj - s.x) - s.y, dy = ((float)gi - s.z) - s.w;
        cov_and_dtheta(sqrtf(dx * dx + dy * dy), cov, cv, dv);
      }
      Cs[e] = cv;
      Ds[e] = dv;
    }
    __syncthreads();
    // adjoint of the correction, thread (tq, tr): realizations tr, tr + 8, ...
    for (int gg = 0; gg < GW_G; ++gg) {
      const float cv = Cs[tq * GW_G + gg];
#pragma unroll
      for (int k = 0; k < RMAX; ++k) {
        const int r = tr + 8 * k;
        if (r < R) cacc[k] = fmaf(cv, Vs[r * GW_G + gg], cacc[k]);
      }
    }
    // correction term: 8 (g, q) pairs per thread
    for (int e = threadIdx.x; e < GW_Q * GW_G; e += blockDim.x) {
      const int qq = e / GW_G, gg = e % GW_G;
      float gsum = 0.f;
      for (int r = 0; r < R; ++r) gsum = fmaf(Vs[r * GW_G + gg], Bs[r * GW_Q + qq], gsum);
      ks += (double)(2.0f * inv_sigma * Cs[e]) * gsum;
      kt += (double)Ds[e] * gsum;
    }
  }
  if (q0 + tq < nobs) {
#pragma unroll
    for (int k = 0; k < RMAX; ++k) {
      const int r = tr + 8 * k;
      if (r < R) atomicAdd(c + (long long)r * nobs + q0 + tq, f * cacc[k]);
    }
  }
  const double a0 = block_sum(ks, red);
  if (threadIdx.x == 0) atomicAdd(acc + 0, (double)f * a0);
  const double a1 = block_sum(kt, red);
  if (threadIdx.x == 0) atomicAdd(acc + 1, (double)f * a1);
}

// sum over sites i, j of dA_ij (a_i a_j / 2 - Ainv_ij / 2 - sum_r w_r,i B_r,j), for
// dA = 2 K_oo / sigma, dK_oo / dtheta and I: acc[0..2].
constexpr int GP_T = 32;

__global__ void __launch_bounds__(256) grad_pairs_kernel(const float* __restrict__ w, const float* __restrict__ B, int ldb,
                                                         int R, int nobs, const float4* __restrict__ obs,
                                                         const float* __restrict__ alpha, const float* __restrict__ Ahi,
                                                         const float* __restrict__ Alo, int lda, CovF cov,
                                                         float inv_sigma, double* __restrict__ acc) {
  extern __shared__ float psm[];
  float* Ws = psm;                 // [R][GP_T]
  float* Bs = Ws + R * GP_T;       // [R][GP_T]
  __shared__ double red[32];
  const int i0 = blockIdx.y * GP_T, j0 = blockIdx.x * GP_T;
  for (int e = threadIdx.x; e < R * GP_T; e += blockDim.x) {
    const int r = e / GP_T, t = e % GP_T;
    Ws[e] = (i0 + t < nobs) ? w[(long long)r * nobs + i0 + t] : 0.f;
    Bs[e] = (j0 + t < nobs) ? B[(long long)r * ldb + j0 + t] : 0.f;
  }
  __syncthreads();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int e = threadIdx.x; e < GP_T * GP_T; e += blockDim.x) {
    const int ti = e / GP_T, tj = e % GP_T;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= nobs || j >= nobs) continue;
    float d = 0.f;
    for (int r = 0; r < R; ++r) d = fmaf(Ws[r * GP_T + ti], Bs[r * GP_T + tj], d);
    const float4 a = obs[i], b = obs[j];
    const float dx = (a.x - b.x) + (a.y - b.y), dy = (a.z - b.z) + (a.w - b.w);
    float cv, dv;
    cov_and_dtheta(sqrtf(dx * dx + dy * dy), cov, cv, dv);
    const double ainv = (double)Ahi[(long long)i * lda + j] + (double)Alo[(long long)i * lda + j];
    const double x = 0.5 * (double)alpha[i] * (double)alpha[j] - 0.5 * ainv - (double)d;
    s0 += 2.0 * inv_sigma * cv * x;
    s1 += (double)dv * x;
    if (i == j) s2 += x;
  }
  double t = block_sum(s0, red);
  if (threadIdx.x == 0) atomicAdd(acc + 0, t);
  t = block_sum(s1, red);
  if (threadIdx.x == 0) atomicAdd(acc + 1, t);
  t = block_sum(s2, red);
  if (threadIdx.x == 0) atomicAdd(acc + 2, t);
}

// H_r(g) = f v_r(g) on the window, 0 elsewhere.
__global__ void grad_hinit_kernel(const float* __restrict__ v, int m, Window win, int R, float f, float* __restrict__ H) {
  const long long M = (long long)m * m;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * M) return;
  const long long g = e % M;
  const int gi = (int)(g / m), gj = (int)(g % m);
  const bool in = gi >= win.i0 && gi < win.i1 && gj >= win.j0 && gj < win.j1;
  H[e] = in ? f * v[e] : 0.f;
}

// Off-grid and nugget terms, thread per (r, q): acc[0..2] -= w_r,q (dW_1 y_r + dphi eps*_r)
// for (sigma, theta, tau^2); scatters -w_r,q W_1[q, k] into H_r at the window nodes.
__global__ void __launch_bounds__(256) grad_offgrid_kernel(const float* __restrict__ w, const float* __restrict__ y,
                                                           long long M, int R, int nobs, int K, const int* __restrict__ idx,
                                                           const float* __restrict__ W1, const float* __restrict__ dW,
                                                           const float* __restrict__ dphi, const int* __restrict__ perm,
                                                           uint32_t k0, uint32_t k1, uint32_t r_base, float* __restrict__ H,
                                                           double* __restrict__ acc) {
  __shared__ double red[32];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (e < (long long)R * nobs) {
    const int r = (int)(e / nobs), q = (int)(e % nobs);
    const float wv = w[e];
    float dy = 0.f;
    for (int k = 0; k < K; ++k) {
      const int g = idx[(long long)q * K + k];
      dy = fmaf(dW[(long long)q * K + k], y[(long long)r * M + g], dy);
      atomicAdd(H + (long long)r * M + g, -wv * W1[(long long)q * K + k]);
    }
    const int i = perm[q];
    const uint4 x = philox4x32_10(make_uint4((uint32_t)i >> 2, r_base + (uint32_t)r, 1u, 0u), k0, k1);
    const int wd = i & 3;
    const float2 zz = (wd < 2) ? box_muller(x.x, x.y) : box_muller(x.z, x.w);
    const float eps = (wd & 1) ? zz.y : zz.x;
    s0 = -(double)wv * dphi[3 * q + 0] * eps;
    s1 = -(double)wv * (dy + dphi[3 * q + 1] * eps);
    s2 = -(double)wv * dphi[3 * q + 2] * eps;
  }
  double t = block_sum(s0, red);
  if (threadIdx.x == 0) atomicAdd(acc + 0, t);
  t = block_sum(s1, red);
  if (threadIdx.x == 0) atomicAdd(acc + 1, t);
  t = block_sum(s2, red);
  if (threadIdx.x == 0) atomicAdd(acc + 2, t);
}

// sum over the window of v^2, into acc[0].
__global__ void window_sumsq_kernel(const float* __restrict__ v, int m, Window win, int R, double* __restrict__ acc) {
  __shared__ double red[32];
  const int wj = win.j1 - win.j0;
  const long long nW = (long long)(win.i1 - win.i0) * wj;
  const long long M = (long long)m * m;
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)R * nW;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / nW);
    const long long gw = e % nW;
    const float val = v[(long long)r * M + (long long)(win.i0 + gw / wj) * m + win.j0 + gw % wj];
    s += (double)val * val;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) atomicAdd(acc, t);
}

// dL/dz[caller index perm[q]] = sum_r w_r,q - alpha_q.
__global__ void grad_z_kernel(const float* __restrict__ w, const float* __restrict__ alpha, int R, int nobs,
                              const int* __restrict__ perm, float* __restrict__ gz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nobs) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += w[(long long)r * nobs + q];
  gz[perm[q]] = s - alpha[q];
}

CovF covf(const ce_ctx* ctx) {
  CovF k;
  k.s2 = (float)(ctx->sigma * ctx->sigma);
  k.theta = (float)ctx->range;
  k.h = (float)ctx->h;
  k.nu3 = ctx->nu == 1.5 ? 1 : 0;
  return k;
}

}  // namespace
}  // namespace ce

using namespace ce;

extern "C" int ce_condsim_grad(ce_ctx* ctx, const float* z_dev, int R, uint64_t seed, uint64_t r_offset,
                               const int* window, float* out_dev, double* grad_theta, float* grad_z_dev, double* loss,
                               void* stream) {
  if (ctx && !ctx->sqrt_lam) return fail(ctx, CE_ERR_STATE, "the context has no embedding");
  if (ctx && ctx->trend_p > 0) return fail(ctx, CE_ERR_STATE, "the gradient does not cover the trend model (ce_set_trend -1 first)");
  if (ctx && (ctx->aniso_ratio != 1.0 || ctx->aniso_angle != 0.0)) {
    return fail(ctx, CE_ERR_STATE, "the gradient covers the isotropic covariance only (ce_set_anisotropy 1, 0 first)");
  }
  if (ctx && ctx->box_joint > 0) {
    return fail(ctx, CE_ERR_STATE, "the gradient does not cover joint grid-box draws (ce_set_box_joint 0 first)");
  }
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (ctx->mode != CE_LOCAL) return fail(ctx, CE_ERR_STATE, "the gradient needs local Kriging (ce_krige_weights, CE_LOCAL)");
  if (!z_dev || !window || !out_dev || !grad_theta || !grad_z_dev || !loss) return fail(ctx, CE_ERR_ARG, "null pointer");
  if (R < 1 || R > 128) return fail(ctx, CE_ERR_ARG, "the gradient takes 1 <= R <= 128");
  const Window win{window[0], window[1], window[2], window[3]};
  if (win.i0 < 0 || win.j0 < 0 || win.i1 > ctx->m || win.j1 > ctx->m || win.i0 >= win.i1 || win.j0 >= win.j1)
    return fail(ctx, CE_ERR_ARG, "window must be a non-empty sub-rectangle of the grid");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st;
  // set-up on first use: d sqrt(lambda)/d theta and the per-site derivatives
  if (!ctx->ds_theta) {
    ctx->ds_theta = (float*)dalloc(ctx, sizeof(float) * (size_t)ctx->P * ctx->P);
    if (!ctx->ds_theta) return fail(ctx, CE_ERR_OOM, "gradient set-up");
    if ((st = eigs_dsqrt_dtheta(ctx, ctx->ds_theta, s))) { dfree(ctx, ctx->ds_theta); ctx->ds_theta = nullptr; return st; }
    if ((st = krige_local_derivatives(ctx, s))) return st;
  }
  // forward pass (leaves B = A^-1 (z - z*) in ctx->Bm)
  if ((st = ce_condsim(ctx, z_dev, R, seed, r_offset, out_dev, stream))) return st;
  const int n = ctx->nobs;
  const long long M = (long long)ctx->m * ctx->m;
  const size_t need = sizeof(float) * ((size_t)R * M * 2 + (size_t)R * n * 2 + (size_t)n + 8);
  if (ctx->grad_bytes < need) {
    dfree(ctx, ctx->grad_buf);
    ctx->grad_buf = (float*)dalloc(ctx, need);
    ctx->grad_bytes = ctx->grad_buf ? need : 0;
    if (!ctx->grad_buf) return fail(ctx, CE_ERR_OOM, "gradient buffers");
  }
  float* Y = ctx->grad_buf;                 // R x M: the unconditional fields again
  float* H = Y + (size_t)R * M;             // R x M: h_r
  float* c = H + (size_t)R * M;             // R x n
  float* w = c + (size_t)R * n;             // R x n
  float* alpha = w + (size_t)R * n;         // n
  double* acc = (double*)dalloc(ctx, sizeof(double) * 16);
  if (!acc) return fail(ctx, CE_ERR_OOM, "gradient accumulators");
  CE_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 16, s));
  if ((st = fft_unconditional(ctx, R, seed, r_offset, Y, s))) { dfree(ctx, acc); return st; }
  launch_solve(ctx, ctx->zint, 1, alpha, n, s);   // alpha = A^-1 z
  const CovF cov = covf(ctx);
  const float inv_sigma = (float)(1.0 / ctx->sigma);
  const long long nW = (long long)(win.i1 - win.i0) * (win.j1 - win.j0);
  const float f = (float)(2.0 / ((double)R * (double)nW));
  // 1. adjoint of the correction over the window
  CE_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(float) * (size_t)R * n, s));
  {
    const size_t shm = sizeof(float) * ((size_t)R * GW_Q + (size_t)R * GW_G + 2 * GW_Q * GW_G);
    CE_CUDA_TRY(cudaFuncSetAttribute(grad_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int splits = (int)std::max<long long>(1, std::min<long long>(64, nW / 2048));
    dim3 g((n + GW_Q - 1) / GW_Q, splits);
    grad_window_kernel<<<g, 256, shm, s>>>(out_dev, ctx->m, win, R, ctx->obs, n, ctx->Bm, ctx->nobs_pad, cov, f, inv_sigma,
                                           c, acc + 0);
  }
  // 2. w = A^-1 c
  launch_solve(ctx, c, R, w, n, s);
  // 3. prediction matrix and log-likelihood
  {
    const size_t shm = sizeof(float) * 2 * (size_t)R * GP_T;
    CE_CUDA_TRY(cudaFuncSetAttribute(grad_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    dim3 g((n + GP_T - 1) / GP_T, (n + GP_T - 1) / GP_T);
    grad_pairs_kernel<<<g, 256, shm, s>>>(w, ctx->Bm, ctx->nobs_pad, R, n, ctx->obs, alpha, ctx->Ainv_hi, ctx->Ainv_lo,
                                          ctx->nobs_pad, cov, inv_sigma, acc + 2);
  }
  // 4. off-grid weights and nugget; h_r = g_r - W_1^T w_r
  grad_hinit_kernel<<<(unsigned)(((long long)R * M + 255) / 256), 256, 0, s>>>(out_dev, ctx->m, win, R, f, H);
  grad_offgrid_kernel<<<(unsigned)(((long long)R * n + 255) / 256), 256, 0, s>>>(
      w, Y, M, R, n, ctx->K, ctx->idx, ctx->W, ctx->dW, ctx->dphi, ctx->perm, (uint32_t)(seed & 0xffffffffu),
      (uint32_t)(seed >> 32), (uint32_t)r_offset, H, acc + 5);
  // 5. the unconditional fields, through the spectral weights
  if ((st = launch_adjoint_ensemble(ctx, H, R, seed, r_offset, acc + 8, s))) { dfree(ctx, acc); return st; }
  // 6. dL/dz, loss
  grad_z_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, alpha, R, n, ctx->perm, grad_z_dev);
  window_sumsq_kernel<<<256, 256, 0, s>>>(out_dev, ctx->m, win, R, acc + 10);
  CE_CUDA_TRY(cudaGetLastError());
  double h_acc[16];
  std::vector<float> h_alpha(n), h_z(n);
  std::vector<int> h_perm(n);
  CE_CUDA_TRY(cudaMemcpyAsync(h_acc, acc, sizeof(h_acc), cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaMemcpyAsync(h_alpha.data(), alpha, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaMemcpyAsync(h_z.data(), ctx->zint, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, acc);
  // acc: [0,1] correction (sigma, theta); [2,3,4] pairs (sigma, theta, tau2);
  //      [5,6,7] off-grid (sigma, theta, tau2); [8,9] fields (theta, sigma); [10] sum of squares
  grad_theta[0] = h_acc[0] + h_acc[2] + h_acc[5] + h_acc[9];
  grad_theta[1] = h_acc[1] + h_acc[3] + h_acc[6] + h_acc[8];
  grad_theta[2] = h_acc[4] + h_acc[7];
  double za = 0.0;
  for (int q = 0; q < n; ++q) za += (double)h_z[q] * (double)h_alpha[q];
  *loss = h_acc[10] / ((double)R * (double)nW) - 0.5 * za - 0.5 * ctx->logdet - 0.5 * n * std::log(2.0 * M_PI);
  return CE_OK;
}
