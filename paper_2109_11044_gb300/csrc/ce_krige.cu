// Off-grid step of the method (Section 2.1 and 2.2; Section 3.6) and the
// nugget-perturbed residuals of steps 3-4.
//
// Local Kriging: each site takes the (2 np)^2 window of grid nodes around its
// grid box (shifted inward near the edges, keeping its shape); by stationarity
// the window covariance K_11 is the same for every site and is inverted once;
// W_1^i = K_21^i K_11^-1, gamma_i = sigma^2 - K_21^i K_11^-1 K_12^i, and the
// synthetic-data nugget is phi_i^2 = tau^2 + gamma_i.  All in FP64.
//
// Nearest-neighbour Kriging: each site's k nearest grid nodes (squared distance
// in FP64 without fused multiply-add, ties to the smaller flat index), their
// union J_N, the surrogate-data map K_No A^-1, the surrogate variances
// sigma_N^2 = sigma^2 - diag(K_No A^-1 K_oN) and the prediction matrix
// K_NN + tau^2 I + diag(sigma_N^2).
//
// Internal row order: the observation points (sites, or surrogate nodes) are
// sorted along a Morton curve so that neighbouring points are adjacent in the
// sums of the solve and of the correction; their terms largely cancel pairwise,
// which keeps FP32 partial sums small.  perm[q] maps a row back to the caller's
// index.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int KMAX = 64;   // (2 np)^2 for np <= 4

struct GridC {
  int m;
  double x0, y0, h, sigma2, theta;
  int nu3;
  Aniso an;
};

// Length of a lag of (dxu, dyu) grid units (columns, rows) in the covariance's metric.
__device__ __forceinline__ double grid_lag_dist(double dxu, double dyu, const GridC& g) {
  return g.an.on ? aniso_dist(g.h * dxu, g.h * dyu, g.an) : g.h * sqrt(dxu * dxu + dyu * dyu);
}

// Interleave the low 16 bits of x and y.
uint32_t morton2(uint32_t x, uint32_t y) {
  auto spread = [](uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
  };
  return spread(x) | (spread(y) << 1);
}

std::vector<int> morton_order(const std::vector<double>& gx, const std::vector<double>& gy, int m) {
  const int n = (int)gx.size();
  std::vector<uint64_t> key(n);
  const double scale = 65535.0 / std::max(1, m - 1);
  for (int i = 0; i < n; ++i) {
    const uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, gx[i] * scale));
    const uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, gy[i] * scale));
    key[i] = ((uint64_t)morton2(qx, qy) << 32) | (uint32_t)i;
  }
  std::sort(key.begin(), key.end());
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = (int)(key[i] & 0xffffffffu);
  return perm;
}

// K_11 of the (2 np)^2 window and its inverse (FP64, one block; K <= 64).
__global__ void k11_inverse_kernel(GridC g, int np, double* __restrict__ Kinv) {
  __shared__ double Lm[KMAX][KMAX + 1];
  __shared__ double X[KMAX][KMAX + 1];
  const int w = 2 * np, K = w * w;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int p = e / K, q = e % K;
    const double da = (double)(p / w - q / w), db = (double)(p % w - q % w);
    Lm[p][q] = matern_d(grid_lag_dist(db, da, g), g.sigma2, g.theta, g.nu3);
    X[p][q] = p == q ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {   // Cholesky, lower
    if (threadIdx.x == 0) Lm[j][j] = sqrt(Lm[j][j]);
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) Lm[i][j] /= Lm[j][j];
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
      const int i = e / K, c = e % K;
      if (i > j && c > j && c <= i) Lm[i][c] -= Lm[i][j] * Lm[c][j];
    }
    __syncthreads();
  }
  // X = L^-T L^-1 I, one thread per column
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    for (int i = 0; i < K; ++i) {
      double v = X[i][c];
      for (int t = 0; t < i; ++t) v -= Lm[i][t] * X[t][c];
      X[i][c] = v / Lm[i][i];
    }
    for (int i = K - 1; i >= 0; --i) {
      double v = X[i][c];
      for (int t = i + 1; t < K; ++t) v -= Lm[t][i] * X[t][c];
      X[i][c] = v / Lm[i][i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) Kinv[e] = X[e / K][e % K];
}

// d K_11 / d theta of the (2 np)^2 window (K <= 64), row-major K x K.
__global__ void dk11_kernel(GridC g, int np, double* __restrict__ dK) {
  const int w = 2 * np, K = w * w;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int p = e / K, q = e % K;
    const double da = (double)(p / w - q / w), db = (double)(p % w - q % w);
    dK[e] = matern_dtheta_d(g.h * sqrt(da * da + db * db), g.sigma2, g.theta, g.nu3);
  }
}

// Derivatives of the local-Kriging quantities of every site (internal order):
// W_1 = K_21 K_11^-1 does not depend on sigma; d W_1 / d theta = (dK_21 - W_1 dK_11) K_11^-1;
// gamma = sigma^2 - K_21 W_1^T gives d gamma / d sigma = 2 gamma / sigma and
// d gamma / d theta = -(2 dK_21 . W_1 - W_1 dK_11 W_1^T); phi = sqrt(tau^2 + gamma).
// Output dphi[q] = (d phi / d sigma, d phi / d theta, d phi / d tau^2).
__global__ void local_deriv_kernel(GridC g, int np, const double* __restrict__ xy, int n, const double* __restrict__ Kinv,
                                   const double* __restrict__ dK11, double tau2, float* __restrict__ dW,
                                   float* __restrict__ dphi) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int w = 2 * np, K = w * w;
  const double sx = xy[2 * q], sy = xy[2 * q + 1];
  const double u = __ddiv_rn(__dsub_rn(sx, g.x0), g.h);
  const double v = __ddiv_rn(__dsub_rn(sy, g.y0), g.h);
  const int j0 = (int)floor(u), i0 = (int)floor(v);
  const int js = min(max(j0 - np + 1, 0), g.m - w);
  const int is = min(max(i0 - np + 1, 0), g.m - w);
  double k21[KMAX], dk21[KMAX], w1[KMAX];
  for (int k = 0; k < K; ++k) {
    const int ii = is + k / w, jj = js + k % w;
    const double dx = sx - (g.x0 + jj * g.h), dy = sy - (g.y0 + ii * g.h);
    const double d = sqrt(dx * dx + dy * dy);
    k21[k] = matern_d(d, g.sigma2, g.theta, g.nu3);
    dk21[k] = matern_dtheta_d(d, g.sigma2, g.theta, g.nu3);
  }
  double quad = 0.0, lin = 0.0;
  for (int k = 0; k < K; ++k) {
    double wk = 0.0;
    for (int t = 0; t < K; ++t) wk += Kinv[k * K + t] * k21[t];
    w1[k] = wk;
    quad += wk * k21[k];
    lin += dk21[k] * wk;
  }
  double wdw = 0.0;
  for (int k = 0; k < K; ++k) {
    double r = 0.0;
    for (int t = 0; t < K; ++t) r += dK11[k * K + t] * w1[t];
    wdw += w1[k] * r;
  }
  // t_l = dK21_l - (W_1 dK_11)_l ; dW_1 = t K_11^-1   (k21 is reused to hold t)
  for (int l = 0; l < K; ++l) {
    double tl = dk21[l];
    for (int t = 0; t < K; ++t) tl -= w1[t] * dK11[t * K + l];
    k21[l] = tl;
  }
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int l = 0; l < K; ++l) acc += k21[l] * Kinv[l * K + k];
    dW[(long long)q * K + k] = (float)acc;
  }
  const double gamma = fmax(g.sigma2 - quad, 0.0);
  const double phi = sqrt(tau2 + gamma);
  const double sigma = sqrt(g.sigma2);
  dphi[3 * q + 0] = (float)((2.0 * gamma / sigma) / (2.0 * phi));
  dphi[3 * q + 1] = (float)((-(2.0 * lin - wdw)) / (2.0 * phi));
  dphi[3 * q + 2] = (float)(1.0 / (2.0 * phi));
}

// Grid-unit coordinates split into an integer part and a fraction.
__device__ __forceinline__ float4 split_units(double sx, double sy, const GridC& g) {
  const double u = __ddiv_rn(__dsub_rn(sx, g.x0), g.h);
  const double v = __ddiv_rn(__dsub_rn(sy, g.y0), g.h);
  const double fu = floor(u), fv = floor(v);
  return make_float4((float)fu, (float)(u - fu), (float)fv, (float)(v - fv));
}

// One thread per site (internal order q): window, weights, gamma, phi.
__global__ void local_weights_kernel(GridC g, int np, const double* __restrict__ xy, int n, const double* __restrict__ Kinv,
                                     int* __restrict__ idx, float* __restrict__ W, float* __restrict__ phi,
                                     float4* __restrict__ obs, double tau2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int w = 2 * np, K = w * w;
  const double sx = xy[2 * q], sy = xy[2 * q + 1];
  const double u = __ddiv_rn(__dsub_rn(sx, g.x0), g.h);
  const double v = __ddiv_rn(__dsub_rn(sy, g.y0), g.h);
  const int j0 = (int)floor(u), i0 = (int)floor(v);
  const int js = min(max(j0 - np + 1, 0), g.m - w);
  const int is = min(max(i0 - np + 1, 0), g.m - w);
  double k21[KMAX];
  for (int k = 0; k < K; ++k) {
    const int ii = is + k / w, jj = js + k % w;
    const double dx = sx - (g.x0 + jj * g.h), dy = sy - (g.y0 + ii * g.h);
    k21[k] = matern_d(aniso_dist(dx, dy, g.an), g.sigma2, g.theta, g.nu3);
    idx[(long long)q * K + k] = ii * g.m + jj;
  }
  double quad = 0.0;
  for (int k = 0; k < K; ++k) {
    double wk = 0.0;
    for (int t = 0; t < K; ++t) wk += Kinv[k * K + t] * k21[t];
    W[(long long)q * K + k] = (float)wk;
    quad += wk * k21[k];
  }
  const double gamma = fmax(g.sigma2 - quad, 0.0);
  phi[q] = (float)sqrt(tau2 + gamma);
  obs[q] = split_units(sx, sy, g);
}

// Covariance matrix between two point sets in FP64, plus `diag` on the diagonal
// when the sets coincide (dst is rows x cols, row-major).
__global__ void cov_matrix_kernel(GridC g, const double* __restrict__ a, int rows, const double* __restrict__ b, int cols,
                                  double diag_add, const double* __restrict__ diag_vec, double* __restrict__ dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e / cols), j = (int)(e % cols);
  const double dx = a[2 * i] - b[2 * j], dy = a[2 * i + 1] - b[2 * j + 1];
  double c = matern_d(aniso_dist(dx, dy, g.an), g.sigma2, g.theta, g.nu3);
  if (diag_vec != nullptr && i == j) c += diag_add + diag_vec[i];
  else if (i == j && diag_vec == nullptr && diag_add != 0.0) c += diag_add;
  dst[e] = c;
}

// k nearest nodes of every site (caller order); marks them in `flags`.
__global__ void nn_select_kernel(GridC g, const double* __restrict__ xy, int n, int k, unsigned char* __restrict__ flags) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double sx = xy[2 * s], sy = xy[2 * s + 1];
  const int j0 = (int)floor(__ddiv_rn(__dsub_rn(sx, g.x0), g.h));
  const int i0 = (int)floor(__ddiv_rn(__dsub_rn(sy, g.y0), g.h));
  double bd[8];
  int bi[8];
  int cnt = 0;
  for (int di = -2; di <= 3; ++di) {
    const int ii = i0 + di;
    if (ii < 0 || ii >= g.m) continue;
    for (int dj = -2; dj <= 3; ++dj) {
      const int jj = j0 + dj;
      if (jj < 0 || jj >= g.m) continue;
      const double dx = __dsub_rn(sx, __dadd_rn(g.x0, __dmul_rn((double)jj, g.h)));
      const double dy = __dsub_rn(sy, __dadd_rn(g.y0, __dmul_rn((double)ii, g.h)));
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      const int flat = ii * g.m + jj;
      // insertion into the sorted list of the best k (d2, then flat index)
      int pos = cnt < k ? cnt : k;
      while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > flat))) {
        if (pos < k) { bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; }
        --pos;
      }
      if (pos < k) { bd[pos] = d2; bi[pos] = flat; }
      if (cnt < k) ++cnt;
    }
  }
  for (int t = 0; t < cnt; ++t) flags[bi[t]] = 1;
}

// sigma_N^2 = sigma^2 - sum_j WN[q][j] G[q][j] with WN = -C (C = -G A^-1 from the
// subtracting GEMM); writes WN in FP32 with rows in internal order.
__global__ void nn_finish_kernel(const double* __restrict__ negWN, const double* __restrict__ G, int nN, int n, double sigma2,
                                 float* __restrict__ WN32, double* __restrict__ sigN2) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= nN) return;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc += -negWN[(long long)row * n + j] * G[(long long)row * n + j];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  // row is the internal index q (G was built in internal order)
  for (int j = lane; j < n; j += 32) WN32[(long long)row * n + j] = (float)(-negWN[(long long)row * n + j]);
  if (lane == 0) sigN2[row] = sigma2 - acc;
}

__global__ void nn_phi_kernel(const double* __restrict__ sigN2, int nN, double tau2, float* __restrict__ phi) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nN) phi[q] = (float)sqrt(fmax(sigN2[q], 0.0) + tau2);
}

__global__ void nn_fill_kernel(const int* __restrict__ Jint, int nN, int m, double x0, double y0, double h,
                               int* __restrict__ idx, float* __restrict__ W, float4* __restrict__ obs, double* __restrict__ xy) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nN) return;
  const int node = Jint[q];
  const int i = node / m, j = node % m;
  idx[q] = node;
  W[q] = 1.0f;
  obs[q] = make_float4((float)j, 0.f, (float)i, 0.f);
  xy[2 * q] = x0 + j * h;
  xy[2 * q + 1] = y0 + i * h;
}

// Nugget draw eps*_r of caller site i: normal i mod 4 of counter (i / 4, r, 1, 0).
__device__ __forceinline__ float nugget_eps(int i, uint32_t r, uint32_t k0, uint32_t k1) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)i >> 2, r, 1u, 0u), k0, k1);
  const int w = i & 3;
  const float2 zz = (w < 2) ? box_muller(x.x, x.y) : box_muller(x.z, x.w);
  return (w & 1) ? zz.y : zz.x;
}

// E[r][q] = zint[q] - (sum_k W[q][k] y_r[idx[q][k]] + phi[q] eps*_r[perm[q]]).
// kBoxes: a site that shares its grid box takes the noise sum_t L_b[a][t] eps*_r[member t]
// instead, its row of the box's noise factor against its box-mates' draws.
template <bool kBoxes>
__global__ void residual_kernel(const float* __restrict__ y, long long M, const int* __restrict__ idx, const float* __restrict__ W,
                                int K, const float* __restrict__ phi, const float* __restrict__ zint, const int* __restrict__ perm,
                                int nobs, int R, uint32_t k0, uint32_t k1, uint32_t r_base, const int* __restrict__ box_cnt,
                                const int* __restrict__ box_mem, const float* __restrict__ box_L, float* __restrict__ E) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * nobs) return;
  const int r = (int)(e / nobs), q = (int)(e % nobs);
  const float* yr = y + (long long)r * M;
  float acc = 0.f;
  if ((K & 3) == 0) {
    // local windows: K = (2 np)^2, a multiple of 4, so the row of indices and weights
    // is read as 16-byte vectors and the gathers are issued back to back (same sum order)
    const int4* __restrict__ ip = reinterpret_cast<const int4*>(idx + (long long)q * K);
    const float4* __restrict__ wp = reinterpret_cast<const float4*>(W + (long long)q * K);
#pragma unroll 3
    for (int k4 = 0; k4 < K / 4; ++k4) {
      const int4 ii = __ldg(ip + k4);
      const float4 ww = __ldg(wp + k4);
      const float y0 = __ldg(yr + ii.x), y1 = __ldg(yr + ii.y), y2 = __ldg(yr + ii.z), y3 = __ldg(yr + ii.w);
      acc = fmaf(ww.x, y0, acc);
      acc = fmaf(ww.y, y1, acc);
      acc = fmaf(ww.z, y2, acc);
      acc = fmaf(ww.w, y3, acc);
    }
  } else {
    for (int k = 0; k < K; ++k) acc = fmaf(W[(long long)q * K + k], __ldg(yr + idx[(long long)q * K + k]), acc);
  }
  const uint32_t rr = r_base + (uint32_t)r;
  if (kBoxes) {
    const int c = box_cnt[q];
    if (c > 0) {
      float noise = 0.f;
      for (int t = 0; t < c; ++t)
        noise = fmaf(box_L[(long long)q * kBoxMax + t], nugget_eps(box_mem[(long long)q * kBoxMax + t], rr, k0, k1), noise);
      E[e] = zint[q] - (acc + noise);
      return;
    }
  }
  E[e] = zint[q] - fmaf(phi[q], nugget_eps(perm[q], rr, k0, k1), acc);
}

// Noise factor of every grid box that holds more than one site, one thread per box.
// Members bq[boff[b]] .. bq[boff[b+1]-1] (internal rows, ascending caller index) share
// the box's window S_b; Gamma_b = K(s_b, s_b) - K(s_b, S_b) K_11^-1 K(S_b, s_b) is their
// conditional covariance given the window, and L_b = chol(Gamma_b + tau^2 I), all FP64.
// Row a of L_b goes to the row of member a with the members' caller indices.
// A factor that is not positive definite sets *status and leaves its rows alone.
__global__ void box_factor_kernel(GridC g, int np, const double* __restrict__ xy, const double* __restrict__ Kinv,
                                  const int* __restrict__ boff, const int* __restrict__ bq, int nbox, const int* __restrict__ perm,
                                  double tau2, int* __restrict__ box_cnt, int* __restrict__ box_mem, float* __restrict__ box_L,
                                  int* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const int o = boff[b], k = boff[b + 1] - o;
  if (k < 2 || k > kBoxMax) { atomicExch(status, 2); return; }
  const int w = 2 * np, K = w * w;
  const int q0 = bq[o];
  const double u = __ddiv_rn(__dsub_rn(xy[2 * q0], g.x0), g.h);
  const double v = __ddiv_rn(__dsub_rn(xy[2 * q0 + 1], g.y0), g.h);
  const int js = min(max((int)floor(u) - np + 1, 0), g.m - w);
  const int is = min(max((int)floor(v) - np + 1, 0), g.m - w);
  double kv[kBoxMax][KMAX];
  for (int a = 0; a < k; ++a) {
    const int q = bq[o + a];
    const double sx = xy[2 * q], sy = xy[2 * q + 1];
    for (int t = 0; t < K; ++t) {
      const double dx = sx - (g.x0 + (js + t % w) * g.h), dy = sy - (g.y0 + (is + t / w) * g.h);
      kv[a][t] = matern_d(aniso_dist(dx, dy, g.an), g.sigma2, g.theta, g.nu3);
    }
  }
  double G[kBoxMax][kBoxMax];
  double tmp[KMAX];
  for (int c = 0; c < k; ++c) {
    for (int t = 0; t < K; ++t) {
      double s = 0.0;
      for (int t2 = 0; t2 < K; ++t2) s += Kinv[t * K + t2] * kv[c][t2];
      tmp[t] = s;
    }
    const int qc = bq[o + c];
    for (int a = c; a < k; ++a) {
      const int qa = bq[o + a];
      const double dx = xy[2 * qa] - xy[2 * qc], dy = xy[2 * qa + 1] - xy[2 * qc + 1];
      double s = matern_d(aniso_dist(dx, dy, g.an), g.sigma2, g.theta, g.nu3);
      for (int t = 0; t < K; ++t) s -= tmp[t] * kv[a][t];
      G[a][c] = a == c ? s + tau2 : s;
    }
  }
  for (int j = 0; j < k; ++j) {   // Cholesky, lower, in place
    double d = G[j][j];
    for (int t = 0; t < j; ++t) d -= G[j][t] * G[j][t];
    if (!(d > 0.0)) { atomicExch(status, 1); return; }
    G[j][j] = sqrt(d);
    for (int i = j + 1; i < k; ++i) {
      double s = G[i][j];
      for (int t = 0; t < j; ++t) s -= G[i][t] * G[j][t];
      G[i][j] = s / G[j][j];
    }
  }
  for (int a = 0; a < k; ++a) {
    const long long row = (long long)bq[o + a] * kBoxMax;
    box_cnt[bq[o + a]] = a + 1;
    for (int t = 0; t < kBoxMax; ++t) {
      box_mem[row + t] = t <= a ? perm[bq[o + t]] : 0;
      box_L[row + t] = t <= a ? (float)G[a][t] : 0.f;
    }
  }
}

__global__ void permute_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, const int* __restrict__ perm, int R,
                                    int nobs, int ld_src, int ld_dst, int to_caller) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * nobs) return;
  const int r = (int)(e / nobs), q = (int)(e % nobs);
  if (to_caller) dst[(long long)r * ld_dst + perm[q]] = src[(long long)r * ld_src + q];
  else dst[(long long)r * ld_dst + q] = src[(long long)r * ld_src + perm[q]];
}

GridC gridc(const ce_ctx* ctx) {
  GridC g;
  g.m = ctx->m;
  g.x0 = ctx->x0;
  g.y0 = ctx->y0;
  g.h = ctx->h;
  g.sigma2 = ctx->sigma * ctx->sigma;
  g.theta = ctx->range;
  g.nu3 = ctx->nu == 1.5 ? 1 : 0;
  g.an = make_aniso(ctx->aniso_ratio, ctx->aniso_angle);
  return g;
}

void free_boxes(ce_ctx* ctx) {
  dfree(ctx, ctx->box_cnt); ctx->box_cnt = nullptr;
  dfree(ctx, ctx->box_mem); ctx->box_mem = nullptr;
  dfree(ctx, ctx->box_L); ctx->box_L = nullptr;
  ctx->box_joint = 0;
}

void free_offgrid(ce_ctx* ctx) {
  free_boxes(ctx);
  dfree(ctx, ctx->perm); ctx->perm = nullptr;
  dfree(ctx, ctx->idx); ctx->idx = nullptr;
  dfree(ctx, ctx->W); ctx->W = nullptr;
  dfree(ctx, ctx->phi); ctx->phi = nullptr;
  dfree(ctx, ctx->J); ctx->J = nullptr;
  dfree(ctx, ctx->WN); ctx->WN = nullptr;
  dfree(ctx, ctx->obs); ctx->obs = nullptr;
  dfree(ctx, ctx->Ainv_hi); ctx->Ainv_hi = nullptr;
  dfree(ctx, ctx->Ainv_lo); ctx->Ainv_lo = nullptr;
  dfree(ctx, ctx->ainv_blk); ctx->ainv_blk = nullptr;
  dfree(ctx, ctx->solve_part); ctx->solve_part = nullptr; ctx->solve_part_bytes = 0;
  dfree(ctx, ctx->zint); ctx->zint = nullptr;
  dfree(ctx, ctx->sites64); ctx->sites64 = nullptr;
  free_trend(ctx);   // its regressors belong to the old sites
  dfree(ctx, ctx->dW); ctx->dW = nullptr;
  dfree(ctx, ctx->dphi); ctx->dphi = nullptr;
  dfree(ctx, ctx->ds_theta); ctx->ds_theta = nullptr;
  dfree(ctx, ctx->E); ctx->E = nullptr;
  dfree(ctx, ctx->Bpart); ctx->Bpart = nullptr;
  dfree(ctx, ctx->Bm); ctx->Bm = nullptr;
  dfree(ctx, ctx->Bsplit); ctx->Bsplit = nullptr; ctx->bsplit_bytes = 0;
  ctx->Rcap = 0;
}

int alloc_rows(ce_ctx* ctx, int nobs, int K) {
  ctx->nobs = nobs;
  ctx->K = K;
  ctx->nobs_pad = (nobs + 127) / 128 * 128;
  ctx->perm = (int*)dalloc(ctx, sizeof(int) * nobs);
  ctx->idx = (int*)dalloc(ctx, sizeof(int) * (size_t)nobs * K);
  ctx->W = (float*)dalloc(ctx, sizeof(float) * (size_t)nobs * K);
  ctx->phi = (float*)dalloc(ctx, sizeof(float) * nobs);
  ctx->obs = (float4*)dalloc(ctx, sizeof(float4) * ctx->nobs_pad);
  ctx->zint = (float*)dalloc(ctx, sizeof(float) * nobs);
  if (!ctx->perm || !ctx->idx || !ctx->W || !ctx->phi || !ctx->obs || !ctx->zint) return fail(ctx, CE_ERR_OOM, "off-grid set-up");
  return CE_OK;
}

}  // namespace

void release_offgrid(ce_ctx* ctx) {
  free_offgrid(ctx);
  ctx->mode = -1;
}

int check_sites(ce_ctx* ctx, const double* xy, int n) {
  const double top = (double)(ctx->m - 1);
  for (int i = 0; i < n; ++i) {
    const double u = (xy[2 * i] - ctx->x0) / ctx->h, v = (xy[2 * i + 1] - ctx->y0) / ctx->h;
    if (!(u >= 0.0 && v >= 0.0 && u <= top && v <= top))
      return fail(ctx, CE_ERR_ARG, "site " + std::to_string(i) + " lies outside the grid's bounding box");
  }
  return CE_OK;
}

int krige_local_setup(ce_ctx* ctx, const double* xy_host, int n, int np, cudaStream_t s) {
  if (2 * np > ctx->m) return fail(ctx, CE_ERR_ARG, "neighbourhood wider than the grid");
  int st = check_sites(ctx, xy_host, n);
  if (st) return st;
  free_offgrid(ctx);
  const int w = 2 * np, K = w * w;
  if ((st = alloc_rows(ctx, n, K))) return st;
  ctx->n = n;
  const GridC g = gridc(ctx);
  // Morton order of the sites in grid units
  std::vector<double> gx(n), gy(n);
  for (int i = 0; i < n; ++i) { gx[i] = (xy_host[2 * i] - ctx->x0) / ctx->h; gy[i] = (xy_host[2 * i + 1] - ctx->y0) / ctx->h; }
  const std::vector<int> perm = morton_order(gx, gy, ctx->m);
  std::vector<double> xy_int(2 * (size_t)n);
  for (int q = 0; q < n; ++q) { xy_int[2 * q] = xy_host[2 * perm[q]]; xy_int[2 * q + 1] = xy_host[2 * perm[q] + 1]; }
  double* d_xy = (double*)dalloc(ctx, sizeof(double) * 2 * n);
  double* d_kinv = (double*)dalloc(ctx, sizeof(double) * KMAX * KMAX);
  double* d_A = (double*)dalloc(ctx, sizeof(double) * (size_t)n * n);
  if (!d_xy || !d_kinv || !d_A) { dfree(ctx, d_xy); dfree(ctx, d_kinv); dfree(ctx, d_A); return fail(ctx, CE_ERR_OOM, "local set-up"); }
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemcpyAsync(d_xy, xy_int.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemsetAsync(ctx->obs, 0, sizeof(float4) * ctx->nobs_pad, s));
  k11_inverse_kernel<<<1, 256, 0, s>>>(g, np, d_kinv);
  local_weights_kernel<<<(n + 127) / 128, 128, 0, s>>>(g, np, d_xy, n, d_kinv, ctx->idx, ctx->W, ctx->phi, ctx->obs, ctx->tau2);
  cov_matrix_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(g, d_xy, n, d_xy, n, ctx->tau2, nullptr, d_A);
  CE_CUDA_TRY(cudaGetLastError());
  st = chol_inverse_f64(ctx, d_A, n, s, nullptr);
  dfree(ctx, d_kinv);
  dfree(ctx, d_A);
  if (st) { dfree(ctx, d_xy); return st; }
  ctx->sites64 = d_xy;   // kept for the gradient set-up
  ctx->mode = CE_LOCAL;
  ctx->np = np;
  return CE_OK;
}

int krige_nn_setup(ce_ctx* ctx, const double* xy_host, int n, int k, cudaStream_t s) {
  int st = check_sites(ctx, xy_host, n);
  if (st) return st;
  free_offgrid(ctx);
  const GridC g = gridc(ctx);
  const long long M = (long long)ctx->m * ctx->m;
  double* d_sites = (double*)dalloc(ctx, sizeof(double) * 2 * n);
  unsigned char* d_flags = (unsigned char*)dalloc(ctx, M);
  if (!d_sites || !d_flags) { dfree(ctx, d_sites); dfree(ctx, d_flags); return fail(ctx, CE_ERR_OOM, "NN set-up"); }
  CE_CUDA_TRY(cudaMemcpyAsync(d_sites, xy_host, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemsetAsync(d_flags, 0, M, s));
  nn_select_kernel<<<(n + 127) / 128, 128, 0, s>>>(g, d_sites, n, k, d_flags);
  CE_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned char> flags(M);
  CE_CUDA_TRY(cudaMemcpyAsync(flags.data(), d_flags, M, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, d_flags);
  std::vector<int> J;   // union, increasing flat index
  for (long long e = 0; e < M; ++e) if (flags[e]) J.push_back((int)e);
  const int nN = (int)J.size();
  if ((st = alloc_rows(ctx, nN, 1))) { dfree(ctx, d_sites); return st; }
  ctx->n = n;
  std::vector<double> gx(nN), gy(nN);
  for (int q = 0; q < nN; ++q) { gx[q] = J[q] % ctx->m; gy[q] = J[q] / ctx->m; }
  const std::vector<int> perm = morton_order(gx, gy, ctx->m);
  std::vector<int> Jint(nN);
  for (int q = 0; q < nN; ++q) Jint[q] = J[perm[q]];
  ctx->J = (int*)dalloc(ctx, sizeof(int) * nN);
  ctx->WN = (float*)dalloc(ctx, sizeof(float) * (size_t)nN * n);
  int* d_Jint = (int*)dalloc(ctx, sizeof(int) * nN);
  double* d_nxy = (double*)dalloc(ctx, sizeof(double) * 2 * nN);
  double* d_A = (double*)dalloc(ctx, sizeof(double) * (size_t)n * n);
  double* d_G = (double*)dalloc(ctx, sizeof(double) * (size_t)nN * n);
  double* d_C = (double*)dalloc(ctx, sizeof(double) * (size_t)nN * n);
  double* d_sig = (double*)dalloc(ctx, sizeof(double) * nN);
  double* d_AN = (double*)dalloc(ctx, sizeof(double) * (size_t)nN * nN);
  auto cleanup = [&]() {
    dfree(ctx, d_sites); dfree(ctx, d_Jint); dfree(ctx, d_nxy); dfree(ctx, d_A); dfree(ctx, d_G);
    dfree(ctx, d_C); dfree(ctx, d_sig); dfree(ctx, d_AN);
  };
  if (!ctx->J || !ctx->WN || !d_Jint || !d_nxy || !d_A || !d_G || !d_C || !d_sig || !d_AN) { cleanup(); return fail(ctx, CE_ERR_OOM, "NN set-up"); }
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->J, J.data(), sizeof(int) * nN, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemcpyAsync(ctx->perm, perm.data(), sizeof(int) * nN, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemcpyAsync(d_Jint, Jint.data(), sizeof(int) * nN, cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemsetAsync(ctx->obs, 0, sizeof(float4) * ctx->nobs_pad, s));
  nn_fill_kernel<<<(nN + 127) / 128, 128, 0, s>>>(d_Jint, nN, ctx->m, ctx->x0, ctx->y0, ctx->h, ctx->idx, ctx->W, ctx->obs, d_nxy);
  // A = K_oo + tau^2 I  and its FP64 inverse
  cov_matrix_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(g, d_sites, n, d_sites, n, ctx->tau2, nullptr, d_A);
  CE_CUDA_TRY(cudaGetLastError());
  double* Ainv = nullptr;
  if ((st = chol_inverse_f64(ctx, d_A, n, s, &Ainv))) { cleanup(); return st; }
  // G = K_No (internal rows), C = -G A^-1, sigma_N^2, WN
  cov_matrix_kernel<<<(unsigned)(((long long)nN * n + 255) / 256), 256, 0, s>>>(g, d_nxy, nN, d_sites, n, 0.0, nullptr, d_G);
  CE_CUDA_TRY(cudaMemsetAsync(d_C, 0, sizeof(double) * (size_t)nN * n, s));
  gemm64_nn_sub(d_G, n, Ainv, n, d_C, n, nN, n, n, s);
  nn_finish_kernel<<<(nN + 7) / 8, 256, 0, s>>>(d_C, d_G, nN, n, g.sigma2, ctx->WN, d_sig);
  nn_phi_kernel<<<(nN + 127) / 128, 128, 0, s>>>(d_sig, nN, ctx->tau2, ctx->phi);
  // A_N = K_NN + diag(tau^2 + sigma_N^2)
  cov_matrix_kernel<<<(unsigned)(((long long)nN * nN + 255) / 256), 256, 0, s>>>(g, d_nxy, nN, d_nxy, nN, ctx->tau2, d_sig, d_AN);
  CE_CUDA_TRY(cudaGetLastError());
  dfree(ctx, Ainv);
  st = chol_inverse_f64(ctx, d_AN, nN, s, nullptr);
  cleanup();
  if (st) return st;
  ctx->mode = CE_NN;
  ctx->knn = k;
  return CE_OK;
}

int krige_local_derivatives(ce_ctx* ctx, cudaStream_t s) {
  if (ctx->mode != CE_LOCAL || !ctx->sites64) return fail(ctx, CE_ERR_STATE, "gradient needs local Kriging set-up");
  const GridC g = gridc(ctx);
  const int np = ctx->np, K = ctx->K, n = ctx->nobs;
  double* d_kinv = (double*)dalloc(ctx, sizeof(double) * KMAX * KMAX);
  double* d_dk = (double*)dalloc(ctx, sizeof(double) * KMAX * KMAX);
  if (!ctx->dW) ctx->dW = (float*)dalloc(ctx, sizeof(float) * (size_t)n * K);
  if (!ctx->dphi) ctx->dphi = (float*)dalloc(ctx, sizeof(float) * 3 * (size_t)n);
  if (!d_kinv || !d_dk || !ctx->dW || !ctx->dphi) { dfree(ctx, d_kinv); dfree(ctx, d_dk); return fail(ctx, CE_ERR_OOM, "derivatives"); }
  k11_inverse_kernel<<<1, 256, 0, s>>>(g, np, d_kinv);
  dk11_kernel<<<1, 256, 0, s>>>(g, np, d_dk);
  local_deriv_kernel<<<(n + 63) / 64, 64, 0, s>>>(g, np, ctx->sites64, n, d_kinv, d_dk, ctx->tau2, ctx->dW, ctx->dphi);
  CE_CUDA_TRY(cudaGetLastError());
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, d_kinv);
  dfree(ctx, d_dk);
  return CE_OK;
}

void launch_residuals(ce_ctx* ctx, const float* y, const float* zint, int R, uint64_t seed, uint64_t r_offset, float* E,
                      cudaStream_t s) {
  const long long tot = (long long)R * ctx->nobs;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  if (ctx->box_joint > 0) {
    residual_kernel<true><<<blocks, 256, 0, s>>>(y, (long long)ctx->m * ctx->m, ctx->idx, ctx->W, ctx->K, ctx->phi, zint, ctx->perm,
                                                 ctx->nobs, R, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                 (uint32_t)r_offset, ctx->box_cnt, ctx->box_mem, ctx->box_L, E);
  } else {
    residual_kernel<false><<<blocks, 256, 0, s>>>(y, (long long)ctx->m * ctx->m, ctx->idx, ctx->W, ctx->K, ctx->phi, zint, ctx->perm,
                                                  ctx->nobs, R, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                  (uint32_t)r_offset, nullptr, nullptr, nullptr, E);
  }
}

void launch_permute_rows(const float* src, float* dst, const int* perm, int R, int nobs, int ld_src, int ld_dst, bool to_caller,
                         cudaStream_t s) {
  const long long tot = (long long)R * nobs;
  permute_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, perm, R, nobs, ld_src, ld_dst, to_caller ? 1 : 0);
}

}  // namespace ce

using namespace ce;

extern "C" int ce_set_box_joint(ce_ctx* ctx, int on, int* n_boxes) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (n_boxes) *n_boxes = 0;
  if (on != 0 && on != 1) return fail(ctx, CE_ERR_ARG, "on must be 0 or 1");
  if (ctx->mode != CE_LOCAL || !ctx->sites64) {
    return fail(ctx, CE_ERR_STATE, "joint grid-box draws need local Kriging weights (ce_krige_weights with CE_LOCAL)");
  }
  cudaStream_t s = ctx->setup_stream;
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  free_boxes(ctx);
  if (!on) return CE_OK;
  const int n = ctx->nobs, m = ctx->m;
  std::vector<double> xy(2 * (size_t)n);
  std::vector<int> perm(n);
  CE_CUDA_TRY(cudaMemcpyAsync(xy.data(), ctx->sites64, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaMemcpyAsync(perm.data(), ctx->perm, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  // grid box of every row (the floor of its grid coordinates, as for the window), then
  // the rows grouped by box, ascending caller index within a box
  std::vector<std::pair<long long, int>> key(n);   // (box, caller index)
  std::vector<int> row_of(n);
  for (int q = 0; q < n; ++q) {
    const double u = (xy[2 * q] - ctx->x0) / ctx->h, v = (xy[2 * q + 1] - ctx->y0) / ctx->h;
    key[q] = {(long long)std::floor(v) * m + (long long)std::floor(u), perm[q]};
    row_of[perm[q]] = q;
  }
  std::sort(key.begin(), key.end());
  std::vector<int> boff{0}, bq;
  for (int a = 0; a < n;) {
    int e = a + 1;
    while (e < n && key[e].first == key[a].first) ++e;
    if (e - a > kBoxMax) {
      return fail(ctx, CE_ERR_ARG, "grid box with " + std::to_string(e - a) + " sites (at most " + std::to_string(kBoxMax) +
                                       " are drawn jointly; refine the grid)");
    }
    if (e - a >= 2) {
      for (int t = a; t < e; ++t) bq.push_back(row_of[key[t].second]);
      boff.push_back((int)bq.size());
    }
    a = e;
  }
  const int nbox = (int)boff.size() - 1;
  if (n_boxes) *n_boxes = nbox;
  if (nbox == 0) return CE_OK;   // every site is alone in its box: the draws are the independent ones
  ctx->box_cnt = (int*)dalloc(ctx, sizeof(int) * n);
  ctx->box_mem = (int*)dalloc(ctx, sizeof(int) * (size_t)n * kBoxMax);
  ctx->box_L = (float*)dalloc(ctx, sizeof(float) * (size_t)n * kBoxMax);
  int* d_boff = (int*)dalloc(ctx, sizeof(int) * boff.size());
  int* d_bq = (int*)dalloc(ctx, sizeof(int) * bq.size());
  double* d_kinv = (double*)dalloc(ctx, sizeof(double) * KMAX * KMAX);
  int* d_status = (int*)dalloc(ctx, sizeof(int));
  auto release = [&]() { dfree(ctx, d_boff); dfree(ctx, d_bq); dfree(ctx, d_kinv); dfree(ctx, d_status); };
  if (!ctx->box_cnt || !ctx->box_mem || !ctx->box_L || !d_boff || !d_bq || !d_kinv || !d_status) {
    release();
    free_boxes(ctx);
    return fail(ctx, CE_ERR_OOM, "grid-box noise factors");
  }
  CE_CUDA_TRY(cudaMemsetAsync(ctx->box_cnt, 0, sizeof(int) * n, s));
  CE_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  CE_CUDA_TRY(cudaMemcpyAsync(d_boff, boff.data(), sizeof(int) * boff.size(), cudaMemcpyHostToDevice, s));
  CE_CUDA_TRY(cudaMemcpyAsync(d_bq, bq.data(), sizeof(int) * bq.size(), cudaMemcpyHostToDevice, s));
  const GridC g = gridc(ctx);
  k11_inverse_kernel<<<1, 256, 0, s>>>(g, ctx->np, d_kinv);
  box_factor_kernel<<<(nbox + 31) / 32, 32, 0, s>>>(g, ctx->np, ctx->sites64, d_kinv, d_boff, d_bq, nbox, ctx->perm, ctx->tau2,
                                                    ctx->box_cnt, ctx->box_mem, ctx->box_L, d_status);
  CE_CUDA_TRY(cudaGetLastError());
  int status = 0;
  CE_CUDA_TRY(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  release();
  if (status) {
    free_boxes(ctx);
    return fail(ctx, CE_ERR_NOT_SPD, "conditional covariance of a grid box is not positive definite (coincident sites without nugget?)");
  }
  ctx->box_joint = nbox;
  return CE_OK;
}
