// Unconditional circulant-embedding ensemble (Section 2.1 step (a); Section 1):
// for each realization pair p, w = DFT2(sqrt(lambda / N) (eps1 + i eps2)) on the
// P x P torus, realization 2p = Re w and 2p+1 = Im w on the m x m grid.
//
// Two passes per chunk of pairs, sized so the chunk's intermediate stays in L2:
//  rows:    Philox noise generated in registers, scaled by sqrt(lambda/N),
//           P-point FFT of every torus row, first m outputs kept -> T[pair][a][k2];
//  columns: CB adjacent columns of T per block, P-point FFT down each column,
//           first m outputs written as the Re/Im realizations.
// The FFT is a shared-memory Stockham radix-4 (final radix-2 stage when log2 P
// is odd) with twiddles from a table computed in FP64 at set-up.
#include <algorithm>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// LINES independent forward FFTs of length P stored back to back in `sm`,
// computed cooperatively by NT threads.  Result in natural order.
template <int P, int LINES, int NT>
__device__ __forceinline__ void fft_lines_smem(float2* sm, const float2* __restrict__ tw) {
  constexpr int Q = P / 4;
  constexpr int BPT = LINES * Q / NT;
  static_assert(LINES * Q % NT == 0 && BPT >= 1, "butterflies must divide evenly");
  constexpr int L = ilog2(P);
  constexpr int N4 = L / 2;
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < N4; ++s) {
    float2 v[BPT][4];
    const int step = Q / Ns;
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int bf = threadIdx.x + t * NT;
      const int line = bf / Q, j = bf % Q;
      const float2* x = sm + line * P;
      float2 a0 = x[j], a1 = x[j + Q], a2 = x[j + 2 * Q], a3 = x[j + 3 * Q];
      if (s > 0) {
        const int k = j & (Ns - 1);
        a1 = cmul(a1, __ldg(tw + k * step));
        a2 = cmul(a2, __ldg(tw + 2 * k * step));
        a3 = cmul(a3, __ldg(tw + 3 * k * step));
      }
      const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y);
      const float2 d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
      const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y);
      const float2 d13 = make_float2(a1.y - a3.y, a3.x - a1.x);   // -i (a1 - a3)
      v[t][0] = make_float2(s02.x + s13.x, s02.y + s13.y);
      v[t][1] = make_float2(d02.x + d13.x, d02.y + d13.y);
      v[t][2] = make_float2(s02.x - s13.x, s02.y - s13.y);
      v[t][3] = make_float2(d02.x - d13.x, d02.y - d13.y);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int bf = threadIdx.x + t * NT;
      const int line = bf / Q, j = bf % Q;
      const int k = j & (Ns - 1);
      float2* y = sm + line * P + (j / Ns) * 4 * Ns + k;
      y[0] = v[t][0];
      y[Ns] = v[t][1];
      y[2 * Ns] = v[t][2];
      y[3 * Ns] = v[t][3];
    }
    __syncthreads();
    Ns *= 4;
  }
  if constexpr (L & 1) {
    constexpr int H = P / 2;
    constexpr int B2 = LINES * H / NT;
    float2 v0[B2], v1[B2];
    const int step = H / Ns;
#pragma unroll
    for (int t = 0; t < B2; ++t) {
      const int bf = threadIdx.x + t * NT;
      const int line = bf / H, j = bf % H;
      const int k = j & (Ns - 1);
      const float2* x = sm + line * P;
      const float2 a = x[j];
      const float2 b = cmul(x[j + H], __ldg(tw + k * step));
      v0[t] = make_float2(a.x + b.x, a.y + b.y);
      v1[t] = make_float2(a.x - b.x, a.y - b.y);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < B2; ++t) {
      const int bf = threadIdx.x + t * NT;
      const int line = bf / H, j = bf % H;
      const int k = j & (Ns - 1);
      float2* y = sm + line * P + (j / Ns) * 2 * Ns + k;
      y[0] = v0[t];
      y[Ns] = v1[t];
    }
    __syncthreads();
  }
}

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

template <int P>
struct FftShape {
  static constexpr int ROWS = P >= 2048 ? 1 : cmin(P, 2048 / P);   // torus rows per block, row pass
  static constexpr int NT_ROWS = cmin(256, ROWS * P / 4);
  static constexpr int CB = P >= 4096 ? 2 : (P >= 2048 ? 4 : 8);   // columns per block, column pass
  static constexpr int NT_COLS = cmin(256, CB * P / 4);
};

// Row pass.  grid.x = P / ROWS, grid.y = pairs in this chunk.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_ROWS)
fft_rows_kernel(const float* __restrict__ sqrt_lam, const float2* __restrict__ tw, int m,
                uint32_t k0, uint32_t k1, uint32_t pair0, uint32_t event, float2* __restrict__ T) {
  constexpr int ROWS = FftShape<P>::ROWS;
  constexpr int kNT = FftShape<P>::NT_ROWS;
  extern __shared__ __align__(16) float2 sm[];
  const int a0 = blockIdx.x * ROWS;
  const int pl = blockIdx.y;
  const uint32_t pair = pair0 + (uint32_t)pl;
  // noise: group g covers torus elements 2g and 2g+1 of the flattened P x P array
  for (int t = threadIdx.x; t < ROWS * P / 2; t += kNT) {
    const int row = t / (P / 2), b = 2 * (t % (P / 2));
    const int a = a0 + row;
    const uint32_t g = (uint32_t)(((long long)a * P + b) >> 1);
    const uint4 x = philox4x32_10(make_uint4(g, pair, 0u, event), k0, k1);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float2 s = *reinterpret_cast<const float2*>(sqrt_lam + (long long)a * P + b);
    sm[row * P + b] = make_float2(s.x * z01.x, s.x * z01.y);
    sm[row * P + b + 1] = make_float2(s.y * z23.x, s.y * z23.y);
  }
  __syncthreads();
  fft_lines_smem<P, ROWS, kNT>(sm, tw);
  float2* dst = T + ((long long)pl * P + a0) * m;
  for (int t = threadIdx.x; t < ROWS * m; t += kNT) {
    const int row = t / m, k2 = t % m;
    dst[(long long)row * m + k2] = sm[row * P + k2];
  }
}

// Column pass.  grid.x = ceil(m / CB), grid.y = pairs in this chunk.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_COLS)
fft_cols_kernel(const float2* __restrict__ T, const float2* __restrict__ tw, int m, int R_local,
                int pair_local0, float* __restrict__ out) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int kNT = FftShape<P>::NT_COLS;
  extern __shared__ __align__(16) float2 smc[];
  const int c0 = blockIdx.x * CB;
  const int pl = blockIdx.y;
  const float2* src = T + (long long)pl * P * m;
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, a = e / CB;
    smc[c * P + a] = (c0 + c < m) ? src[(long long)a * m + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, CB, kNT>(smc, tw);
  const int r_re = 2 * (pair_local0 + pl);
  const bool has_im = r_re + 1 < R_local;
  const long long M = (long long)m * m;
  for (int e = threadIdx.x; e < CB * m; e += kNT) {
    const int c = e % CB, k1 = e / CB;
    if (c0 + c >= m) continue;
    const float2 w = smc[c * P + k1];
    const long long o = (long long)k1 * m + c0 + c;
    out[r_re * M + o] = w.x;
    if (has_im) out[(r_re + 1) * M + o] = w.y;
  }
}

template <int P>
int run_ensemble(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s) {
  const int m = ctx->m;
  const int pairs = (R + 1) / 2;
  const size_t per_pair = sizeof(float2) * (size_t)P * m;
  // chunk of pairs whose intermediate fits in about 48 MB of L2
  int chunk = (int)std::max<size_t>(1, (48u << 20) / per_pair);
  chunk = std::min(chunk, pairs);
  const int nchunks = (pairs + chunk - 1) / chunk;
  chunk = (pairs + nchunks - 1) / nchunks;
  if (ctx->Tpairs < chunk) {
    dfree(ctx, ctx->T);
    ctx->T = (float2*)dalloc(ctx, per_pair * chunk);
    if (!ctx->T) { ctx->Tpairs = 0; return fail(ctx, CE_ERR_OOM, "FFT intermediate"); }
    ctx->Tpairs = chunk;
  }
  constexpr int CB = FftShape<P>::CB;
  const size_t shm_cols = sizeof(float2) * CB * P;
  const size_t shm_rows = sizeof(float2) * FftShape<P>::ROWS * P;
  CE_CUDA_TRY(cudaFuncSetAttribute(fft_cols_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_cols));
  CE_CUDA_TRY(cudaFuncSetAttribute(fft_rows_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_rows));
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  const uint32_t pair_base = (uint32_t)(r_offset / 2);
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    dim3 grow(P / FftShape<P>::ROWS, np);
    fft_rows_kernel<P><<<grow, FftShape<P>::NT_ROWS, shm_rows, s>>>(ctx->sqrt_lam, ctx->twiddle, m, k0, k1, pair_base + p0, 0u, ctx->T);
    dim3 gcol((m + CB - 1) / CB, np);
    fft_cols_kernel<P><<<gcol, FftShape<P>::NT_COLS, shm_cols, s>>>(ctx->T, ctx->twiddle, m, R, p0, y);
    ctx->launches += 2;
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

__global__ void philox_kernel(const uint4* __restrict__ ctr, int count, uint32_t k0, uint32_t k1, uint4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void normals_kernel(const uint4* __restrict__ ctr, int count, uint32_t k0, uint32_t k1, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 x = philox4x32_10(ctr[i], k0, k1);
  const float2 a = box_muller(x.x, x.y), b = box_muller(x.z, x.w);
  out[i] = make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace

int fft_unconditional(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s) {
  switch (ctx->P) {
    case 16: return run_ensemble<16>(ctx, R, seed, r_offset, y, s);
    case 32: return run_ensemble<32>(ctx, R, seed, r_offset, y, s);
    case 64: return run_ensemble<64>(ctx, R, seed, r_offset, y, s);
    case 128: return run_ensemble<128>(ctx, R, seed, r_offset, y, s);
    case 256: return run_ensemble<256>(ctx, R, seed, r_offset, y, s);
    case 512: return run_ensemble<512>(ctx, R, seed, r_offset, y, s);
    case 1024: return run_ensemble<1024>(ctx, R, seed, r_offset, y, s);
    case 2048: return run_ensemble<2048>(ctx, R, seed, r_offset, y, s);
    case 4096: return run_ensemble<4096>(ctx, R, seed, r_offset, y, s);
    case 8192: return run_ensemble<8192>(ctx, R, seed, r_offset, y, s);
    default: return fail(ctx, CE_ERR_ARG, "unsupported embedding size");
  }
}

void launch_philox(const uint32_t* ctr, int count, uint64_t seed, uint32_t* out, cudaStream_t s) {
  if (count <= 0) return;
  philox_kernel<<<(count + 255) / 256, 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), count,
                                                    (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                    reinterpret_cast<uint4*>(out));
}

void launch_normals(const uint32_t* ctr, int count, uint64_t seed, float* out, cudaStream_t s) {
  if (count <= 0) return;
  normals_kernel<<<(count + 255) / 256, 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), count,
                                                     (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                     reinterpret_cast<float4*>(out));
}

}  // namespace ce

// ---------------------------------------------------------------------------
// The same row and column passes with the intermediate in a caller-supplied
// device buffer of T_bytes; nothing is allocated.  Pairs are processed in
// chunks that fit the buffer.
// ---------------------------------------------------------------------------
namespace ce {
namespace {

template <int P>
int run_ensemble_into(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s, float2* T,
                      size_t T_bytes) {
  const int m = ctx->m;
  const int pairs = (R + 1) / 2;
  const size_t per_pair = sizeof(float2) * (size_t)P * m;
  if (per_pair > T_bytes) return fail(ctx, CE_ERR_ARG, "one realization pair needs more scratch than the fixed buffer holds");
  const int chunk = (int)std::min<size_t>((size_t)pairs, T_bytes / per_pair);
  constexpr int CB = FftShape<P>::CB;
  const size_t shm_cols = sizeof(float2) * CB * P;
  const size_t shm_rows = sizeof(float2) * FftShape<P>::ROWS * P;
  CE_CUDA_TRY(cudaFuncSetAttribute(fft_cols_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_cols));
  CE_CUDA_TRY(cudaFuncSetAttribute(fft_rows_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_rows));
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  const uint32_t pair_base = (uint32_t)(r_offset / 2);
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    dim3 grow(P / FftShape<P>::ROWS, np);
    fft_rows_kernel<P><<<grow, FftShape<P>::NT_ROWS, shm_rows, s>>>(ctx->sqrt_lam, ctx->twiddle, m, k0, k1, pair_base + p0, 0u, T);
    dim3 gcol((m + CB - 1) / CB, np);
    fft_cols_kernel<P><<<gcol, FftShape<P>::NT_COLS, shm_cols, s>>>(T, ctx->twiddle, m, R, p0, y);
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace

int fft_unconditional_into(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s, void* T,
                           size_t T_bytes) {
  float2* t = static_cast<float2*>(T);
  switch (ctx->P) {
    case 16: return run_ensemble_into<16>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 32: return run_ensemble_into<32>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 64: return run_ensemble_into<64>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 128: return run_ensemble_into<128>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 256: return run_ensemble_into<256>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 512: return run_ensemble_into<512>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 1024: return run_ensemble_into<1024>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 2048: return run_ensemble_into<2048>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 4096: return run_ensemble_into<4096>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    case 8192: return run_ensemble_into<8192>(ctx, R, seed, r_offset, y, s, t, T_bytes);
    default: return fail(ctx, CE_ERR_ARG, "unsupported embedding size");
  }
}

}  // namespace ce
