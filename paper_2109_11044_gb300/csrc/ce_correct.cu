// Kriging correction, step 5 of Section 2: v_r = y_r + K_go B[:, r] on every
// grid node, with B = A^-1 (z - z*) the weighted residuals (Eq. (condmvn)).
// The grid x site covariance K_go is never stored: each block evaluates the
// Matern covariance (Section 3.3) for its tile of nodes against a chunk of
// sites in shared memory and contracts it with the matching rows of B.
//
// This file holds the plain FP32 form (CUDA cores).  Distances are formed in
// grid units from exact integer node coordinates and the sites' split
// coordinates (integer part + fraction), so each difference is rounded once.
// Each covariance value is evaluated with compensated FP32 arithmetic (below),
// so it carries about one rounding error, not the larger error of the
// hardware approximations: with clustered sites the weights B are large and of
// alternating sign, the sum K_go B cancels by a factor of 10^2-10^3, and every
// random error of a covariance term is amplified by that factor.  Per chunk of
// 32 sites the products accumulate in FP32; chunk sums join the running sum
// with Kahan compensation.
#include <cmath>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {

int launch_correct_tc(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s);

namespace {

constexpr int TN = 64;   // grid nodes per block
constexpr int KC = 32;   // sites per chunk

// Matern constants for the compensated evaluation, in grid units:
// C(d) = s2 (1 + a d) 2^(b d), b = b_hi + b_lo held as two floats.
struct MaternFC {
  float s2, a, b_hi, b_lo;
};

// q(g) ~ (2^g - 1) / g on [-0.5005, 0.5005]: a weighted least-squares fit of the
// relative error of 1 + g q(g) against 2^g on Chebyshev nodes, coefficients
// rounded to FP32 (relative error of 1 + g q(g) below 3e-9 in exact arithmetic).
__constant__ float kExp2Q[7] = {0.6931471824645996f,   0.24022650718688965f,    0.055504102259874344f,
                                0.00961803738027811f,  0.0013334081741049886f,  0.00015467044431716204f,
                                1.5165644072112627e-05f};

// C at grid-unit offsets (dx, dy).  d^2 is kept as an unevaluated sum t + te
// (error-free products and sum), d = sqrt(t + te) as d0 + d1 (one correction
// step from the hardware reciprocal square root), the exponent b d as x0 + x1
// (error-free product), and 2^(b d) = 2^n 2^g with n = rint(x0) and
// g = (x0 - n) + x1 by the polynomial above.  The result carries about one
// FP32 rounding of relative error.  The error-free steps use the _rn
// intrinsics, which the compiler never fuses into FMAs (a fused product would
// break the two-sum identities).
__device__ __forceinline__ float matern_f_comp(float dx, float dy, const MaternFC& k) {
  const float px = __fmul_rn(dx, dx), ex = fmaf(dx, dx, -px);
  const float py = __fmul_rn(dy, dy), ey = fmaf(dy, dy, -py);
  const float t0 = __fadd_rn(px, py);
  const float bp = __fsub_rn(t0, px);
  const float te = __fadd_rn(__fadd_rn(__fsub_rn(px, __fsub_rn(t0, bp)), __fsub_rn(py, bp)), __fadd_rn(ex, ey));
  const float t = fmaxf(t0, 1e-30f);
  const float r = fast_rsqrt(t);
  const float d0 = __fmul_rn(t, r);
  const float d1 = (fmaf(-d0, d0, t) + te) * (0.5f * r);
  const float x0 = __fmul_rn(k.b_hi, d0);
  const float x1 = fmaf(k.b_hi, d0, -x0) + fmaf(k.b_hi, d1, k.b_lo * d0);
  const float n = rintf(x0);
  const float g = __fsub_rn(x0, n) + x1;
  float q = kExp2Q[6];
#pragma unroll
  for (int i = 5; i >= 0; --i) q = fmaf(q, g, kExp2Q[i]);
  const float e = fmaf(g, q, 1.0f);
  const float lin = fmaf(k.a, d0, fmaf(k.a, d1, 1.0f));
  const int ni = (int)n;   // b < 0, so n <= 0
  return ni < -126 ? 0.f : (k.s2 * lin) * e * __int_as_float((ni + 127) << 23);
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// The weights of the next chunk are copied into shared memory with cp.async
// while the current chunk is evaluated and multiplied (two buffers).
// Anisotropic covariance (an.x = 1): the grid-unit offset is mapped by the 2 x 2
// matrix (an.y, an.z; an.w, a22) before the evaluation.
template <int RT>
__global__ void __launch_bounds__(256) correct_simt(float* __restrict__ y, int m, const float4* __restrict__ obs, int nobs,
                                                    const float* __restrict__ B, int ldb, int R, MaternFC mf, float4 an,
                                                    float a22) {
  constexpr int RTILE = 16 * RT;
  __shared__ float Cs[KC][TN];
  __shared__ float Bs[2][KC][RTILE];
  const long long M = (long long)m * m;
  const long long g0 = (long long)blockIdx.x * TN;
  const int r0 = blockIdx.y * RTILE;
  const int tn = threadIdx.x % 16, tr = threadIdx.x / 16;
  float sum[4][RT], comp[4][RT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) { sum[i][j] = 0.f; comp[i][j] = 0.f; }
  // every element this thread evaluates belongs to the same node (256 is a multiple of TN)
  const long long gt = g0 + threadIdx.x % TN;
  const float gti = gt < M ? (float)(int)(gt / m) : 0.f, gtj = gt < M ? (float)(int)(gt % m) : 0.f;
  auto load_b = [&](int bf, int k0) {
    for (int e = threadIdx.x; e < KC * RTILE; e += 256) {
      const int kk = e / RTILE, rr = e % RTILE;
      const bool ok = k0 + kk < nobs && r0 + rr < R;
      cp_async4(static_cast<uint32_t>(__cvta_generic_to_shared(&Bs[bf][kk][rr])),
                ok ? B + (long long)(r0 + rr) * ldb + k0 + kk : B, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (nobs > 0) load_b(0, 0);
  int bf = 0;
  for (int k0 = 0; k0 < nobs; k0 += KC, bf ^= 1) {
#pragma unroll
    for (int t = 0; t < KC * TN / 256; ++t) {
      const int e = threadIdx.x + 256 * t;
      const int kk = e / TN, nn = e % TN;
      float c = 0.f;
      if (k0 + kk < nobs && gt < M) {
        const float4 o = obs[k0 + kk];
        const float dx = (gtj - o.x) - o.y, dy = (gti - o.z) - o.w;
        c = an.x != 0.f ? matern_f_comp(fmaf(an.y, dx, an.z * dy), fmaf(an.w, dx, a22 * dy), mf) : matern_f_comp(dx, dy, mf);
      }
      Cs[kk][nn] = c;
    }
    if (k0 + KC < nobs) {
      load_b(bf ^ 1, k0 + KC);   // that buffer was released by the barrier that ended the last chunk
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
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
      for (int j = 0; j < RT; ++j) b[j] = Bs[bf][kk][tr + 16 * j];
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

// The FP64 form: the same tiling with every step in FP64 (site coordinates from the
// FP64 copy where local Kriging keeps one, the covariance by the closed form of
// Section 3.3 with the library exp, products and sums in FP64), the field read and
// written once in FP32.  RT64 x 16 realizations per block; a comparison form for the
// reduced-precision ones, not a fast path (FP64 runs far below FP32 on this part).
// kh = h sqrt(3) / theta (nu = 3/2) or h / theta (nu = 1/2): C = s2 (1 + t) e^-t or
// s2 e^-t with t = kh times the grid-unit distance.
template <int RT64>
__global__ void __launch_bounds__(256) correct_f64(float* __restrict__ y, int m, const double* __restrict__ sxy,
                                                   const float4* __restrict__ obs, double x0, double y0, double inv_h,
                                                   int nobs, const float* __restrict__ B, int ldb, int R, double sigma2,
                                                   double kh, int nu3, Aniso ad) {
  constexpr int RTILE = 16 * RT64;
  __shared__ double Cs[KC][TN];
  __shared__ double Bs[KC][RTILE];
  const long long M = (long long)m * m;
  const long long g0 = (long long)blockIdx.x * TN;
  const int r0 = blockIdx.y * RTILE;
  const int tn = threadIdx.x % 16, tr = threadIdx.x / 16;
  double acc[4][RT64];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < RT64; ++j) acc[i][j] = 0.0;
  const long long gt = g0 + threadIdx.x % TN;
  const double gti = gt < M ? (double)(gt / m) : 0.0, gtj = gt < M ? (double)(gt % m) : 0.0;
  for (int k0 = 0; k0 < nobs; k0 += KC) {
#pragma unroll
    for (int t = 0; t < KC * TN / 256; ++t) {
      const int e = threadIdx.x + 256 * t;
      const int kk = e / TN, nn = e % TN;
      double c = 0.0;
      const int q = k0 + kk;
      if (q < nobs && gt < M) {
        double gx, gy;   // the site in grid units
        if (sxy) {
          gx = (sxy[2 * q] - x0) * inv_h;
          gy = (sxy[2 * q + 1] - y0) * inv_h;
        } else {
          const float4 o = obs[q];
          gx = (double)o.x + (double)o.y;
          gy = (double)o.z + (double)o.w;
        }
        const double t = kh * aniso_dist(gtj - gx, gti - gy, ad);
        c = nu3 ? sigma2 * (1.0 + t) * exp(-t) : sigma2 * exp(-t);
      }
      Cs[kk][nn] = c;
    }
    for (int e = threadIdx.x; e < KC * RTILE; e += 256) {
      const int kk = e / RTILE, rr = e % RTILE;
      Bs[kk][rr] = (k0 + kk < nobs && r0 + rr < R) ? (double)B[(long long)(r0 + rr) * ldb + k0 + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      double c[4], b[RT64];
#pragma unroll
      for (int i = 0; i < 4; ++i) c[i] = Cs[kk][tn + 16 * i];
#pragma unroll
      for (int j = 0; j < RT64; ++j) b[j] = Bs[kk][tr + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < RT64; ++j) acc[i][j] = fma(c[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < RT64; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tr + 16 * j;
      const long long g = g0 + tn + 16 * i;
      if (r < R && g < M) y[(long long)r * M + g] = (float)((double)y[(long long)r * M + g] + acc[i][j]);
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
  if (ctx->mode == CE_NN && ctx->nn_circulant) return launch_correct_circulant(ctx, B, R, y, s);
  if (ctx->prec == CE_PREC_FP64) {
    const long long M = (long long)ctx->m * ctx->m;
    const Aniso ad = make_aniso(ctx->aniso_ratio, ctx->aniso_angle);
    const double kh = (ctx->nu == 1.5 ? std::sqrt(3.0) : 1.0) * ctx->h / ctx->range;
    const double* sxy = ctx->mode == CE_LOCAL ? ctx->sites64 : nullptr;
    const double s2 = ctx->sigma * ctx->sigma;
    const int nu3 = ctx->nu == 1.5 ? 1 : 0;
    const unsigned gx = (unsigned)((M + TN - 1) / TN);
    if (R <= 16)
      correct_f64<1><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, sxy, ctx->obs, ctx->x0, ctx->y0, 1.0 / ctx->h, ctx->nobs, B,
                                                 ctx->nobs_pad, R, s2, kh, nu3, ad);
    else if (R <= 32)
      correct_f64<2><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, sxy, ctx->obs, ctx->x0, ctx->y0, 1.0 / ctx->h, ctx->nobs, B,
                                                 ctx->nobs_pad, R, s2, kh, nu3, ad);
    else
      correct_f64<4><<<dim3(gx, (unsigned)((R + 63) / 64)), 256, 0, s>>>(y, ctx->m, sxy, ctx->obs, ctx->x0, ctx->y0,
                                                                         1.0 / ctx->h, ctx->nobs, B, ctx->nobs_pad, R, s2,
                                                                         kh, nu3, ad);
    CE_CUDA_TRY(cudaGetLastError());
    return CE_OK;
  }
  if (ctx->prec != CE_PREC_FP32) return launch_correct_tc(ctx, B, R, y, s);
  const MaternF m1 = matern_grid_units(ctx);
  const double log2e = 1.4426950408889634;
  const double b = (ctx->nu == 1.5 ? -std::sqrt(3.0) : -1.0) * ctx->h / ctx->range * log2e;
  MaternFC mf;
  mf.s2 = m1.s2;
  mf.a = m1.a;
  mf.b_hi = (float)b;
  mf.b_lo = (float)(b - (double)mf.b_hi);
  const long long M = (long long)ctx->m * ctx->m;
  const unsigned gx = (unsigned)((M + TN - 1) / TN);
  const int ldb = ctx->nobs_pad;
  const Aniso ad = make_aniso(ctx->aniso_ratio, ctx->aniso_angle);
  const float4 an = make_float4(ad.on ? 1.f : 0.f, (float)ad.a11, (float)ad.a12, (float)ad.a21);
  const float a22 = (float)ad.a22;
  if (R <= 16) {
    correct_simt<1><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf, an, a22);
  } else if (R <= 32) {
    correct_simt<2><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf, an, a22);
  } else if (R <= 64) {
    correct_simt<4><<<dim3(gx, 1), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf, an, a22);
  } else {
    correct_simt<8><<<dim3(gx, (R + 127) / 128), 256, 0, s>>>(y, ctx->m, ctx->obs, ctx->nobs, B, ldb, R, mf, an, a22);
  }
  ctx->launches += 1;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace ce
