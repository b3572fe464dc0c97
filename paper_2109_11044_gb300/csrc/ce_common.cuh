// Device helpers shared by the kernels of the CE conditional-simulation library:
// the counter-based generator, Box-Muller normals, the Matern covariance and
// error-checking macros.  sm_103a only.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#define CE_CUDA_TRY(expr)                                                     \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) return ce::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

namespace ce {

int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32
// multiplications with the key advanced by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t w0 = (uint64_t)0xD2511F53u * c.x, w1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)w0;
    const uint32_t hi0 = (uint32_t)(w0 >> 32);
    const uint32_t lo1 = (uint32_t)w1;
    const uint32_t hi1 = (uint32_t)(w1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The ten round keys of one 64-bit seed, for kernels that draw many numbers
// with the same key: passed as a __grid_constant__ kernel parameter, the keys
// are read from the parameter bank instead of being advanced in every call.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
  for (int i = 0; i < 10; ++i) {
    K.k0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
    K.k1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return K;
}

// Philox4x32-10 with the round keys precomputed (same results as philox4x32_10).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t w0 = (uint64_t)0xD2511F53u * c.x, w1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)w0;
    const uint32_t hi0 = (uint32_t)(w0 >> 32);
    const uint32_t lo1 = (uint32_t)w1;
    const uint32_t hi1 = (uint32_t)(w1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ K.k0[i], lo1, hi0 ^ c.w ^ K.k1[i], lo0);
  }
  return c;
}

// Two uint32 words -> two N(0,1) values by Box-Muller, with u = (x + 1/2) 2^-32.
// ln(u) for u < 1/2 comes from the fast log (3 ulp there); for u >= 1/2 it is
// ln(1 - q) with q = (~x + 1/2) 2^-32 formed without cancellation: the fast log
// of 1 - q when q >= 1/16 (absolute error below 4e-7), else the series
// -(q + q^2/2 + ... + q^7/7).  The angle 2 pi u2 is taken as pi (2 u2 - 1) + pi
// so that the fast sine and cosine see arguments in (-pi, pi).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  // Branch-free (the three cases select, so a warp never runs two of them):
  // the fast log of u or of 1 - q, and the series for u close to 1.
  const bool upper = a >= 0x80000000u;
  const float q = fmaf((float)(~a), 0x1p-32f, 0x1p-33f);
  const float larg = upper ? 1.0f - q : fmaf((float)a, 0x1p-32f, 0x1p-33f);
  const float lfast = __logf(larg);
  float p = fmaf(q, 1.0f / 7.0f, 1.0f / 6.0f);
  p = fmaf(q, p, 0.2f);
  p = fmaf(q, p, 0.25f);
  p = fmaf(q, p, 1.0f / 3.0f);
  p = fmaf(q, p, 0.5f);
  p = fmaf(q, p, 1.0f);
  const float lnu = (upper && q < 0.0625f) ? -q * p : lfast;
  const float r2 = -2.0f * lnu;
  float rs;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(r2));
  const float rad = r2 * rs;
  const float th = fmaf((float)b, 0x1p-31f, -1.0f) * 3.14159265358979323846f;
  float s, c;
  __sincosf(th, &s, &c);
  return make_float2(-rad * c, -rad * s);
}

// ---------------------------------------------------------------------------
// Matern covariance, Section 3.3 closed forms: nu = 1/2 -> sigma^2 exp(-d/theta),
// nu = 3/2 -> sigma^2 (1 + sqrt(3) d/theta) exp(-sqrt(3) d/theta).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double matern_d(double d, double sigma2, double theta, int nu3) {
  if (nu3) {
    const double t = 1.7320508075688772 * d / theta;
    return sigma2 * (1.0 + t) * exp(-t);
  }
  return sigma2 * exp(-d / theta);
}

// d C / d theta (the range) of the same closed forms:
// nu = 1/2: C d / theta^2;  nu = 3/2: sigma^2 t^2 exp(-t) / theta with t = sqrt(3) d / theta.
__device__ __forceinline__ double matern_dtheta_d(double d, double sigma2, double theta, int nu3) {
  if (nu3) {
    const double t = 1.7320508075688772 * d / theta;
    return sigma2 * t * t * exp(-t) / theta;
  }
  return sigma2 * exp(-d / theta) * d / (theta * theta);
}

// Geometric anisotropy: the covariance of an offset (dx, dy) is C(|A (dx, dy)|) with
// A = diag(1, 1/ratio) Rot(-angle) (range theta along the direction at `angle`,
// theta * ratio across it); on = 0 is the isotropic model.
struct Aniso {
  int on;
  double a11, a12, a21, a22;
};

__host__ __device__ inline Aniso make_aniso(double ratio, double angle) {
  Aniso a;
  const double c = cos(angle), s = sin(angle);
  a.on = !(ratio == 1.0 && angle == 0.0);
  a.a11 = c;
  a.a12 = s;
  a.a21 = -s / ratio;
  a.a22 = c / ratio;
  return a;
}

// |A (dx, dy)| (Euclidean length when isotropic).
__device__ __forceinline__ double aniso_dist(double dx, double dy, const Aniso& a) {
  if (!a.on) return sqrt(dx * dx + dy * dy);
  const double u = a.a11 * dx + a.a12 * dy, v = a.a21 * dx + a.a22 * dy;
  return sqrt(u * u + v * v);
}

// FP32 evaluation from the distance in grid units.  The caller passes
// a = sqrt(3) h / theta (nu = 3/2) or 0 (nu = 1/2) and b = -(a or h/theta) log2(e),
// precomputed in FP64 and rounded once.  exp goes to the ex2 unit.
struct MaternF {
  float s2;  // sigma^2
  float a;   // linear factor (nu = 3/2) or 0
  float b;   // exponent factor in log2 units (negative)
};

__device__ __forceinline__ float fast_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fast_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// C from the squared distance in grid units.
__device__ __forceinline__ float matern_f_d2(float d2, const MaternF& k) {
  d2 = fmaxf(d2, 1e-30f);
  const float d = d2 * fast_rsqrt(d2);
  const float e = fast_ex2(k.b * d);
  return k.s2 * fmaf(k.a, d, 1.0f) * e;
}

}  // namespace ce
