// Kriging correction, step 5 of Section 2: v_r = y_r + K_go B[:, r] on every
// grid node, with B = A^-1 (z - z*) the weighted residuals (Eq. (condmvn)).
// The grid x site covariance K_go is never stored: each block evaluates the
// Matern covariance (Section 3.3) for its tile of nodes against a chunk of
// sites in shared memory and contracts it with the matching rows of B.
//
// This file holds the plain FP32 form (CUDA cores).  Distances are formed in
// grid units from exact integer node coordinates and the sites' split
// coordinates (integer part + fraction), so each difference is rounded once.
// Per chunk of 32 sites the products accumulate in FP32; chunk sums join the
// running sum with Kahan compensation.
#include <cmath>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {

int launch_correct_tc(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);

namespace {

constexpr int TN = 64;   // grid nodes per block
constexpr int KC = 32;   // sites per chunk

template <int RT>
__global__ void __launch_bounds__(256) correct_simt(float* __restrict__ y, int m, const float4* __restrict__ obs, int nobs,
                                                    const float* __restrict__ B, int ldb, int R, MaternF mf) {
  constexpr int RTILE = 16 * RT;
  __shared__ float Cs[KC][TN];
  __shared__ float Bs[KC][RTILE];
  const long long M = (long long)m * m;
  const long long g0 = (long long)blockIdx.x * TN;
  const int r0 = blockIdx.y * RTILE;
  const int tn = threadIdx.x % 16, tr = threadIdx.x / 16;
  float sum[4][RT], comp[4][RT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) { sum[i][j] = 0.f; comp[i][j] = 0.f; }
  for (int k0 = 0; k0 < nobs; k0 += KC) {
#pragma unroll
    for (int t = 0; t < KC * TN / 256; ++t) {
      const int e = threadIdx.x + 256 * t;
      const int kk = e / TN, nn = e % TN;
      const long long g = g0 + nn;
      float c = 0.f;
      if (k0 + kk < nobs && g < M) {
        const float4 o = obs[k0 + kk];
        const float gi = (float)(int)(g / m), gj = (float)(int)(g % m);
        const float dx = (gj - o.x) - o.y, dy = (gi - o.z) - o.w;
        c = matern_f_d2(fmaf(dx, dx, dy * dy), mf);
      }
      Cs[kk][nn] = c;
    }
    for (int e = threadIdx.x; e < KC * RTILE; e += 256) {
      const int kk = e / RTILE, rr = e % RTILE;
      Bs[kk][rr] = (k0 + kk < nobs && r0 + rr < R) ? B[(long long)(r0 + rr) * ldb + k0 + kk] : 0.f;
    }
    __syncthreads();
    float part[4][RT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < RT; ++j) part[i][j] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      float c[4], b[RT];
#pragma unroll
      for (int i = 0; i < 4; ++i) c[i] = Cs[kk][tn + 16 * i];
#pragma unroll
      for (int j = 0; j < RT; ++j) b[j] = Bs[kk][tr + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) part[i][j] = fmaf(c[i], b[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < RT; ++j) {
        const float yv = part[i][j] - comp[i][j];
        const float t = sum[i][j] + yv;
        comp[i][j] = (t - sum[i][j]) - yv;
        sum[i][j] = t;
      }
    __syncthreads();
  }
  // all loads in flight before any store
  float yv[4][RT];
#pragma unroll
  for (int j = 0; j < RT; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tr + 16 * j;
      const long long g = g0 + tn + 16 * i;
      yv[i][j] = (r < R && g < M) ? y[(long long)r * M + g] : 0.f;
    }
#pragma unroll
  for (int j = 0; j < RT; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tr + 16 * j;
      const long long g = g0 + tn + 16 * i;
      if (r < R && g < M) y[(long long)r * M + g] = yv[i][j] + sum[i][j];
    }
}

}  // namespace

MaternF matern_grid_units(const ce_ctx* ctx) {
  MaternF k;
  const double log2e = 1.4426950408889634;
  k.s2 = (float)(ctx->sigma * ctx->sigma);
  if (ctx->nu == 1.5) {
    const double a = std::sqrt(3.0) * ctx->h / ctx->range;
    k.a = (float)a;
    k.b = (float)(-a * log2e);
  } else {
    k.a = 0.f;
    k.b = (float)(-ctx->h / ctx->range * log2e);
  }
  return k;
}

int launch_correct(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  if (ctx->prec != CE_PREC_FP32) return launch_correct_tc(ctx, B, R, y, s);
  const MaternF mf = matern_grid_units(ctx);
  const long long M = (long long)ctx->m * ctx->m;
  const unsigned gx = (unsigned)((M + TN - 1) / TN);
  const int ldb = ctx->nobs_pad;
  if (R <= 16) {
    correct_simt<1><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf);
  } else if (R <= 32) {
    correct_simt<2><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf);
  } else if (R <= 64) {
    correct_simt<4><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf);
  } else {
    correct_simt<8><<<dim3(gx, (R + 127) / 128), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf);
  }
  ctx->launches += 1;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace ce
