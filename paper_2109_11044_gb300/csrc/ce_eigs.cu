// Circulant-embedding set-up in FP64 (Section 1 with Wood & Chan's embedding;
// Section 2.1 step (a)): the first row of the block-circulant covariance on a
// P x P torus, its 2-D DFT, the nonnegativity check with embedding growth, and
// the FP32 spectral weights sqrt(lambda / P^2) used by the unconditional sampler.
#include <cmath>
#include <cstdio>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

// c[a][b] = C(h sqrt(min(a,P-a)^2 + min(b,P-b)^2)) as a complex value with zero imaginary part.
// Anisotropic: C of the signed torus lag (row lag a, column lag b, each in (-P/2, P/2]),
// averaged with the entry of the mirrored lag (-a, -b), which differs only where a lag
// is P/2: c is then even on the torus (lambda real), and no grid lag is changed.
__global__ void embed_kernel(double2* __restrict__ buf, int P, double h, double sigma2, double theta, int nu3, Aniso an) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)P * P) return;
  const int a = (int)(e / P), b = (int)(e % P);
  if (!an.on) {
    const double wa = (double)min(a, P - a), wb = (double)min(b, P - b);
    buf[e] = make_double2(matern_d(h * sqrt(wa * wa + wb * wb), sigma2, theta, nu3), 0.0);
    return;
  }
  const int la = a <= P / 2 ? a : a - P, lb = b <= P / 2 ? b : b - P;
  const int ma = (P - a) % P, mb = (P - b) % P;   // the mirrored entry's indices
  const int lma = ma <= P / 2 ? ma : ma - P, lmb = mb <= P / 2 ? mb : mb - P;
  const double c1 = matern_d(aniso_dist(h * lb, h * la, an), sigma2, theta, nu3);
  const double c2 = matern_d(aniso_dist(h * lmb, h * lma, an), sigma2, theta, nu3);
  buf[e] = make_double2(0.5 * (c1 + c2), 0.0);
}

// One radix-2 Stockham FFT (forward, unnormalised) of length P per block, in
// shared memory.  Line `blockIdx.x` starts at buf + blockIdx.x * line_stride and
// its elements are elem_stride apart.  Each stage reads all of a thread's
// butterfly inputs into registers before any thread overwrites the line.
constexpr int kFft64Threads = 1024;
constexpr int kFft64MaxB = 4;   // P <= 8192

__global__ void __launch_bounds__(kFft64Threads)
fft64_lines(double2* __restrict__ buf, int P, long long line_stride, long long elem_stride) {
  extern __shared__ double2 sm64[];
  double2* line = buf + (long long)blockIdx.x * line_stride;
  for (int e = threadIdx.x; e < P; e += blockDim.x) sm64[e] = line[(long long)e * elem_stride];
  __syncthreads();
  const int half = P / 2;
  for (int Ns = 1; Ns < P; Ns *= 2) {
    double2 v0[kFft64MaxB], v1[kFft64MaxB];
    int nb = 0;
    for (int j = threadIdx.x; j < half; j += blockDim.x, ++nb) {
      const int k = j % Ns;
      const double2 a = sm64[j], b = sm64[j + half];
      double s, c;
      sincospi(-(double)k / (double)Ns, &s, &c);   // e^{-2 pi i k / (2 Ns)}
      const double2 bw = make_double2(b.x * c - b.y * s, b.x * s + b.y * c);
      v0[nb] = make_double2(a.x + bw.x, a.y + bw.y);
      v1[nb] = make_double2(a.x - bw.x, a.y - bw.y);
    }
    __syncthreads();
    nb = 0;
    for (int j = threadIdx.x; j < half; j += blockDim.x, ++nb) {
      const int k = j % Ns;
      const int base = (j / Ns) * 2 * Ns + k;
      sm64[base] = v0[nb];
      sm64[base + Ns] = v1[nb];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < P; e += blockDim.x) line[(long long)e * elem_stride] = sm64[e];
}

// Per-block min and max of the real parts.
__global__ void minmax_kernel(const double2* __restrict__ buf, long long N, double* __restrict__ out) {
  __shared__ double smin[32], smax[32];
  double lo = INFINITY, hi = -INFINITY;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const double v = buf[e].x;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  for (int o = 16; o; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) { smin[threadIdx.x >> 5] = lo; smax[threadIdx.x >> 5] = hi; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    lo = threadIdx.x < nw ? smin[threadIdx.x] : INFINITY;
    hi = threadIdx.x < nw ? smax[threadIdx.x] : -INFINITY;
    for (int o = 16; o; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (threadIdx.x == 0) { out[2 * blockIdx.x] = lo; out[2 * blockIdx.x + 1] = hi; }
  }
}

// sqrt(max(lambda, 0) / N) in FP32; counts and sums the clipped negatives.
__global__ void finalize_kernel(const double2* __restrict__ buf, long long N, float* __restrict__ sq,
                                unsigned long long* __restrict__ nclip, double* __restrict__ clipmass) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double l = buf[e].x;
  if (l < 0.0) {
    atomicAdd(nclip, 1ull);
    atomicAdd(clipmass, -l);
  }
  sq[e] = (float)sqrt(fmax(l, 0.0) / (double)N);
}

// t[b][a] = s[a][b] (P x P), through 32 x 32 shared-memory tiles (P of any size).
__global__ void transpose_kernel(const float* __restrict__ s, float* __restrict__ t, int P) {
  __shared__ float tile[32][33];
  const int b0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  const int x = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    if (a0 + r < P && b0 + x < P) tile[r][x] = s[(long long)(a0 + r) * P + b0 + x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    if (b0 + r < P && a0 + x < P) t[(long long)(b0 + r) * P + a0 + x] = tile[x][r];
}

// c and d c / d theta on the torus, as two complex arrays.
__global__ void embed_pair_kernel(double2* __restrict__ c, double2* __restrict__ dc, int P, double h, double sigma2,
                                  double theta, int nu3) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)P * P) return;
  const int a = (int)(e / P), b = (int)(e % P);
  const double wa = (double)min(a, P - a), wb = (double)min(b, P - b);
  const double d = h * sqrt(wa * wa + wb * wb);
  c[e] = make_double2(matern_d(d, sigma2, theta, nu3), 0.0);
  dc[e] = make_double2(matern_dtheta_d(d, sigma2, theta, nu3), 0.0);
}

// d sqrt(lambda / N) / d theta = (d lambda / d theta) / (2 sqrt(N lambda)), 0 where lambda <= 0.
__global__ void dsqrt_kernel(const double2* __restrict__ lam, const double2* __restrict__ dlam, long long N,
                             float* __restrict__ ds) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const double l = lam[e].x;
  ds[e] = l > 0.0 ? (float)(dlam[e].x / (2.0 * sqrt((double)N * l))) : 0.0f;
}

__global__ void twiddle_kernel(float2* __restrict__ tw, int P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)P, &s, &c);
  tw[k] = make_float2((float)c, (float)s);
}

// The twiddles of the 1024-point register transforms as a 32 x 32 matrix,
// tw32[k][t] = e^{-2 pi i t k / 1024}: lane t of a warp reads row k contiguously.
__global__ void twiddle32_kernel(float2* __restrict__ tw32) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 1024) return;
  const int k = e >> 5, t = e & 31;
  double s, c;
  sincospi(-2.0 * (double)(t * k) / 1024.0, &s, &c);
  tw32[e] = make_float2((float)c, (float)s);
}

}  // namespace

// d sqrt(lambda / N) / d theta on the context's embedding (FP64, stored as FP32).
int eigs_dsqrt_dtheta(ce_ctx* ctx, float* ds, cudaStream_t s) {
  const int P = ctx->P;
  const long long N = (long long)P * P;
  double2* lam = (double2*)dalloc(ctx, sizeof(double2) * N);
  double2* dlam = (double2*)dalloc(ctx, sizeof(double2) * N);
  if (!lam || !dlam) { dfree(ctx, lam); dfree(ctx, dlam); return fail(ctx, CE_ERR_OOM, "embedding derivative"); }
  embed_pair_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(lam, dlam, P, ctx->h, ctx->sigma * ctx->sigma, ctx->range,
                                                               ctx->nu == 1.5 ? 1 : 0);
  const size_t shm = sizeof(double2) * P;
  CE_CUDA_TRY(cudaFuncSetAttribute(fft64_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const int thr = P / 2 < kFft64Threads ? P / 2 : kFft64Threads;
  for (double2* buf : {lam, dlam}) {
    fft64_lines<<<P, thr, shm, s>>>(buf, P, P, 1);
    fft64_lines<<<P, thr, shm, s>>>(buf, P, 1, P);
  }
  dsqrt_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(lam, dlam, N, ds);
  CE_CUDA_TRY(cudaGetLastError());
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, lam);
  dfree(ctx, dlam);
  return CE_OK;
}

int eigs_setup(ce_ctx* ctx, int max_growth, cudaStream_t s) {
  int P = 1;
  while (P < 2 * ctx->m) P *= 2;
  const double sigma2 = ctx->sigma * ctx->sigma;
  const int nu3 = ctx->nu == 1.5 ? 1 : 0;
  for (int g = 0; g <= max_growth; ++g, P *= 2) {
    if (P > 8192) return fail(ctx, CE_ERR_EMBED, "embedding would exceed 8192 x 8192");
    const long long N = (long long)P * P;
    double2* buf = (double2*)dalloc(ctx, sizeof(double2) * N);
    double* mm = (double*)dalloc(ctx, sizeof(double) * 2 * 1024);
    if (!buf || !mm) { dfree(ctx, buf); dfree(ctx, mm); return fail(ctx, CE_ERR_OOM, "embedding buffer"); }
    embed_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(buf, P, ctx->h, sigma2, ctx->range, nu3,
                                                              make_aniso(ctx->aniso_ratio, ctx->aniso_angle));
    const size_t shm = sizeof(double2) * P;
    CE_CUDA_TRY(cudaFuncSetAttribute(fft64_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const int thr = P / 2 < kFft64Threads ? P / 2 : kFft64Threads;
    fft64_lines<<<P, thr, shm, s>>>(buf, P, P, 1);   // rows
    fft64_lines<<<P, thr, shm, s>>>(buf, P, 1, P);   // columns
    minmax_kernel<<<1024, 256, 0, s>>>(buf, N, mm);
    CE_CUDA_TRY(cudaGetLastError());
    std::vector<double> h_mm(2 * 1024);
    CE_CUDA_TRY(cudaMemcpyAsync(h_mm.data(), mm, sizeof(double) * 2 * 1024, cudaMemcpyDeviceToHost, s));
    CE_CUDA_TRY(cudaStreamSynchronize(s));
    double lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < 1024; ++b) { lo = std::fmin(lo, h_mm[2 * b]); hi = std::fmax(hi, h_mm[2 * b + 1]); }
    if (!(lo >= -1e-6 * hi)) {   // indefinite: grow
      dfree(ctx, buf);
      dfree(ctx, mm);
      continue;
    }
    ctx->P = P;
    ctx->growth = g;
    ctx->lambda_min = lo;
    ctx->lambda_max = hi;
    ctx->sqrt_lam = (float*)dalloc(ctx, sizeof(float) * N);
    ctx->twiddle = (float2*)dalloc(ctx, sizeof(float2) * P);
    if (P >= 1024) ctx->tw32 = (float2*)dalloc(ctx, sizeof(float2) * 1024);
    if (!ctx->sqrt_lam || !ctx->twiddle || (P >= 1024 && !ctx->tw32)) {
      dfree(ctx, buf);
      dfree(ctx, mm);
      return fail(ctx, CE_ERR_OOM, "spectral weights");
    }
    unsigned long long* nclip = (unsigned long long*)mm;
    double* cmass = mm + 1;
    CE_CUDA_TRY(cudaMemsetAsync(mm, 0, 2 * sizeof(double), s));
    finalize_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(buf, N, ctx->sqrt_lam, nclip, cmass);
    // the column passes read the weights of a torus column contiguously: the transpose,
    // which is the array itself when lambda is symmetric (isotropic covariance)
    if (make_aniso(ctx->aniso_ratio, ctx->aniso_angle).on) {
      ctx->sqrt_lam_t = (float*)dalloc(ctx, sizeof(float) * N);
      if (!ctx->sqrt_lam_t) { dfree(ctx, buf); dfree(ctx, mm); return fail(ctx, CE_ERR_OOM, "spectral weights"); }
      transpose_kernel<<<dim3((P + 31) / 32, (P + 31) / 32), dim3(32, 8), 0, s>>>(ctx->sqrt_lam, ctx->sqrt_lam_t, P);
    } else {
      ctx->sqrt_lam_t = ctx->sqrt_lam;
    }
    twiddle_kernel<<<(P + 255) / 256, 256, 0, s>>>(ctx->twiddle, P);
    if (P >= 1024) twiddle32_kernel<<<4, 256, 0, s>>>(ctx->tw32);
    CE_CUDA_TRY(cudaGetLastError());
    unsigned long long hc = 0;
    double hm = 0;
    CE_CUDA_TRY(cudaMemcpyAsync(&hc, nclip, sizeof(hc), cudaMemcpyDeviceToHost, s));
    CE_CUDA_TRY(cudaMemcpyAsync(&hm, cmass, sizeof(hm), cudaMemcpyDeviceToHost, s));
    CE_CUDA_TRY(cudaStreamSynchronize(s));
    ctx->clipped = (long long)hc;
    ctx->clipped_mass = hm;
    dfree(ctx, buf);
    dfree(ctx, mm);
    return CE_OK;
  }
  return fail(ctx, CE_ERR_EMBED, "circulant embedding indefinite after growth");
}

}  // namespace ce
