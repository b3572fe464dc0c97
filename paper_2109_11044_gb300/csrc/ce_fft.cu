// Unconditional circulant-embedding ensemble (Section 2.1 step (a); Section 1):
// for each realization pair p, w = DFT2(sqrt(lambda / N) (eps1 + i eps2)) on the
// P x P torus, realization 2p = Re w and 2p+1 = Im w on the m x m grid.
//
// Two passes per chunk of pairs, sized so the chunk's intermediate stays in L2:
//  columns: Philox noise generated in registers, scaled by sqrt(lambda/N),
//           P-point FFT down every torus column, first m frequencies kept
//           -> T[pair][k1][b];
//  rows:    P-point FFT along every kept row of T, first m frequencies written
//           as the Re/Im realizations.
// For P = 1024 each line is one warp's: 32 points per lane in registers, two
// in-register 32-point FFTs around a shared-memory transpose.  Other sizes use
// a shared-memory Stockham radix-4 (final radix-2 stage when log2 P is odd).
// Twiddles come from a table computed in FP64 at set-up.
#include <algorithm>

#include "ce_common.cuh"
#include "ce_fft_lines.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

// Column pass with the noise.  grid.x = P / CB, grid.y = pairs in this chunk.
// Block: CB torus columns b0 .. b0+CB-1; counter (a P + b, pair, 0, event), a < P/2,
// gives the noise of elements (a, b) and (a + P/2, b).  The spectral weight of
// (a, b) is read from the transposed weights, sqrt_lam_t[b P + a] = sqrt_lam[a P + b],
// so the loads are contiguous in a.
// Output: T[pair][k1][b] for the first m column frequencies k1.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_COLS)
fft_colnoise_kernel(const float* __restrict__ sqrt_lam, const float2* __restrict__ tw, int m,
                    const __grid_constant__ PhiloxKeys keys, uint32_t pair0, uint32_t event, float2* __restrict__ T) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int kNT = FftShape<P>::NT_COLS;
  constexpr int H = P / 2;
  extern __shared__ __align__(16) float2 smc[];
  const int b0 = blockIdx.x * CB;
  const int pl = blockIdx.y;
  const uint32_t pair = pair0 + (uint32_t)pl;
  for (int e = threadIdx.x; e < CB * H; e += kNT) {
    const int a = e % H, c = e / H;
    const int b = b0 + c;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)(a * P + b), pair, 0u, event), keys);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float s0 = __ldg(sqrt_lam + (long long)b * P + a), s1 = __ldg(sqrt_lam + (long long)b * P + a + H);
    smc[c * P + a] = make_float2(s0 * z01.x, s0 * z01.y);
    smc[c * P + a + H] = make_float2(s1 * z23.x, s1 * z23.y);
  }
  __syncthreads();
  fft_lines_smem<P, CB, kNT>(smc, tw);
  float2* dst = T + (long long)pl * m * P;
  for (int e = threadIdx.x; e < CB * m; e += kNT) {
    const int c = e % CB, kk = e / CB;
    dst[(long long)kk * P + b0 + c] = smc[c * P + kk];
  }
}

// Row pass.  grid.x = ceil(m / ROWS), grid.y = pairs in this chunk.  Rows k1 of T
// are transformed along b; the first m frequencies are realization 2p (real
// part) and 2p+1 (imaginary part) at out[.][k1][k2].
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_ROWS)
fft_rowout_kernel(const float2* __restrict__ T, const float2* __restrict__ tw, int m, int R_local, int pair_local0,
                  float* __restrict__ out) {
  constexpr int ROWS = FftShape<P>::ROWS;
  constexpr int kNT = FftShape<P>::NT_ROWS;
  extern __shared__ __align__(16) float2 sm[];
  const int r0 = blockIdx.x * ROWS;
  const int pl = blockIdx.y;
  const float2* src = T + (long long)pl * m * P;
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, b = e % P;
    sm[e] = (r0 + row < m) ? src[(long long)(r0 + row) * P + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, ROWS, kNT>(sm, tw);
  const int r_re = 2 * (pair_local0 + pl);
  const bool has_im = r_re + 1 < R_local;
  const long long M = (long long)m * m;
  for (int e = threadIdx.x; e < ROWS * m; e += kNT) {
    const int row = e / m, k2 = e % m;
    if (r0 + row >= m) continue;
    const float2 w = sm[row * P + k2];
    const long long o = (long long)(r0 + row) * m + k2;
    out[r_re * M + o] = w.x;
    if (has_im) out[(r_re + 1) * M + o] = w.y;
  }
}

// ---------------------------------------------------------------------------
// P = 1024: one warp per line, 32 points per lane in registers.  A line x[a]
// is split as a = t + 32 k (lane t, register k); X[j + 32 l] =
// sum_t W32^{t l} W1024^{t j} sum_k x[t + 32 k] W32^{k j}: a 32-point FFT in
// each lane, the twiddles W1024^{t j}, a transpose through shared memory, and
// a second 32-point FFT in each lane.
// ---------------------------------------------------------------------------
// cos(pi q / 16)
__host__ __device__ constexpr float cospi16(int q) {
  q = ((q % 32) + 32) % 32;
  const int r = q <= 8 ? q : (q <= 16 ? 16 - q : (q <= 24 ? q - 16 : 32 - q));
  const float v = r == 0 ? 1.0f
                : r == 1 ? 0.980785280403230449126f
                : r == 2 ? 0.923879532511286756128f
                : r == 3 ? 0.831469612302545237079f
                : r == 4 ? 0.707106781186547524401f
                : r == 5 ? 0.555570233019602224743f
                : r == 6 ? 0.382683432365089771728f
                : r == 7 ? 0.195090322016128267848f
                : 0.0f;
  return (q > 8 && q < 24) ? -v : v;
}

// a * W32^q, W32 = exp(-2 pi i / 32)
__device__ __forceinline__ float2 mul_w32(float2 a, int q) {
  q &= 31;
  if (q == 0) return a;
  if (q == 8) return make_float2(a.y, -a.x);
  if (q == 16) return make_float2(-a.x, -a.y);
  if (q == 24) return make_float2(-a.y, a.x);
  const float c = cospi16(q), s = cospi16(q - 8);   // W32^q = c - i s
  return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

__host__ __device__ constexpr int brev5(int i) {
  return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// In-register 32-point forward DFT, natural order in and out (radix-2 DIT).
// HALF: only the outputs 0..15 are formed (the last stage's differences, which
// give 16..31, are skipped); v[16..31] are left undefined.
template <bool HALF = false>
__device__ __forceinline__ void fft32_reg(float2 (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int j = brev5(i);
    if (i < j) { const float2 t = v[i]; v[i] = v[j]; v[j] = t; }
  }
#pragma unroll
  for (int half = 1; half < 32; half *= 2) {
#pragma unroll
    for (int s0 = 0; s0 < 32; s0 += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 a = v[s0 + k];
        const float2 b = mul_w32(v[s0 + k + half], k * (16 / half));
        v[s0 + k] = make_float2(a.x + b.x, a.y + b.y);
        if (!(HALF && half == 16)) v[s0 + k + half] = make_float2(a.x - b.x, a.y - b.y);
      }
    }
  }
}

// Second half of the line transform: twiddle, transpose through `buf`
// (32 x 33 float2, this warp's), second 32-point FFT.  On return lane j holds
// X[j + 32 l] in v[l] (HALF: for l < 16 only).  `tw32` is the 32 x 32 twiddle
// matrix, tw32[k][t] = W1024^{t k}: each of the 31 loads of a lane reads one row
// of it contiguously across the warp.
template <bool HALF = false>
__device__ __forceinline__ void fft1024_finish(float2 (&v)[32], float2* buf, const float2* __restrict__ tw32, int lane) {
#pragma unroll
  for (int k = 1; k < 32; ++k) v[k] = cmul(v[k], __ldg(tw32 + k * 32 + lane));
#pragma unroll
  for (int k = 0; k < 32; ++k) buf[k * 33 + lane] = v[k];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = buf[lane * 33 + t];
  __syncwarp();
  fft32_reg<HALF>(v);
}

constexpr int kFastWarps = 8;

// One warp stages `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global memory into its shared buffer with one bulk asynchronous copy completing
// on the warp's own mbarrier (phase 0: each barrier serves one copy per launch).
// The wait is bounded; on expiry it returns false in every lane after giving the
// copy in flight one more bounded wait and setting CE_ERR_TIMEOUT in *status.
__device__ __forceinline__ bool warp_bulk_stage(void* dst, const void* src, uint32_t bytes, uint64_t* bar_ptr, int lane,
                                                int* __restrict__ status) {
  const uint32_t bar = static_cast<uint32_t>(__cvta_generic_to_shared(bar_ptr));
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
  }
  __syncwarp();
  auto arrived_within = [&](uint32_t limit) {
    bool done = false;
    for (uint32_t it = 0; it < limit && !done; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(bar)
          : "memory");
      done = ok != 0;
    }
    return done;
  };
  if (__all_sync(0xffffffffu, arrived_within(1u << 22))) return true;
  if (lane == 0) atomicExch(status, CE_ERR_TIMEOUT);
  arrived_within(1u << 22);
  return false;
}

// Column pass with noise, P = 1024.  grid.x = 1024 / 8, grid.y = pairs.
__global__ void __launch_bounds__(32 * kFastWarps, 3)
fft1024_colnoise_kernel(const float* __restrict__ sqrt_lam, const float2* __restrict__ tw32, int m,
                        const __grid_constant__ PhiloxKeys keys, uint32_t pair0, uint32_t event, float2* __restrict__ T,
                        int* __restrict__ status) {
  constexpr int P = 1024;
  extern __shared__ __align__(16) float2 smf[];
  __shared__ __align__(8) uint64_t col_bar[kFastWarps];
  float2* buf = smf + (threadIdx.x >> 5) * (32 * 33);
  float2* stage = smf;   // [k1][8 columns], reusing the transpose buffers after a barrier
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * kFastWarps + w;
  const int pl = blockIdx.y;
  const uint32_t pair = pair0 + (uint32_t)pl;
  // the column's 4 KB of weights, staged in the warp's transpose buffer by one bulk copy
  const float* sl = reinterpret_cast<const float*>(buf);
  const bool staged = warp_bulk_stage(buf, sqrt_lam + (long long)b * P, P * sizeof(float), &col_bar[w], lane, status);
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int a = lane + 32 * k;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)(a * P + b), pair, 0u, event), keys);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float s0 = staged ? sl[a] : 0.f, s1 = staged ? sl[a + P / 2] : 0.f;
    v[k] = make_float2(s0 * z01.x, s0 * z01.y);
    v[k + 16] = make_float2(s1 * z23.x, s1 * z23.y);
  }
  __syncwarp();   // every lane has read its weights before the transpose reuses the buffer
  fft32_reg(v);
  fft1024_finish<true>(v, buf, tw32, lane);   // outputs kk < m <= 512: l < 16
  __syncthreads();   // every warp is done with its transpose buffer
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const int kk = lane + 32 * l;
    if (kk < m) stage[kk * kFastWarps + w] = v[l];
  }
  __syncthreads();
  float2* dst = T + (long long)pl * m * P + blockIdx.x * kFastWarps;
  for (int e = threadIdx.x; e < m * kFastWarps; e += 32 * kFastWarps) {
    const int kk = e / kFastWarps, c = e % kFastWarps;
    dst[(long long)kk * P + c] = stage[e];
  }
}

// Row pass, P = 1024.  grid.x = ceil(m / 8), grid.y = pairs.  Each warp's row
// (8 KB) arrives in its transpose buffer by one bulk asynchronous copy, so the
// load path carries one instruction per row instead of 32 per lane.  The wait
// is bounded: on expiry the warp sets CE_ERR_TIMEOUT in *status and skips its row.
// ACC: add the real parts to realization 2p and subtract the imaginary parts from
// 2p + 1 (the circulant correction's final conjugation) instead of storing them.
template <bool ACC = false>
__global__ void __launch_bounds__(32 * kFastWarps, 3)
fft1024_rowout_kernel(const float2* __restrict__ T, const float2* __restrict__ tw32, int m, int R_local, int pair_local0,
                      float* __restrict__ out, int* __restrict__ status) {
  constexpr int P = 1024;
  extern __shared__ __align__(16) float2 smf[];
  __shared__ __align__(8) uint64_t row_bar[kFastWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* buf = smf + w * (32 * 33);
  const int row = blockIdx.x * kFastWarps + w;
  if (row >= m) return;
  const int pl = blockIdx.y;
  const float2* src = T + ((long long)pl * m + row) * P;
  if (!warp_bulk_stage(buf, src, P * sizeof(float2), &row_bar[w], lane, status)) return;
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = buf[lane + 32 * k];
  __syncwarp();   // every lane has its inputs before the transpose reuses the buffer
  fft32_reg(v);
  fft1024_finish<true>(v, buf, tw32, lane);   // outputs k2 < m <= 512: l < 16
  const int r_re = 2 * (pair_local0 + pl);
  const bool has_im = r_re + 1 < R_local;
  const long long M = (long long)m * m;
  float* o_re = out + r_re * M + (long long)row * m;
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const int k2 = lane + 32 * l;
    if (k2 < m) {
      if (ACC) {
        o_re[k2] += v[l].x;
        if (has_im) o_re[M + k2] -= v[l].y;
      } else {
        o_re[k2] = v[l].x;
        if (has_im) o_re[M + k2] = v[l].y;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// P = 2048: two warps per torus line.  The warp of parity q transforms
// x_q[t] = x[2t + q], t < 1024, as a 1024-point transform in registers (the
// code above, with the same 32 x 32 matrix of W1024 twiddles);
// the line's transform is X[k] = E[k] + W2048^k O[k] for k < 1024, and only the
// k < m <= 1024 that the crop keeps are formed.  The noise of element a < 1024
// and a + 1024 comes from one counter (same parity, same warp).
// ---------------------------------------------------------------------------
constexpr int kLines2048 = 4;   // torus lines per block of 8 warps

__global__ void __launch_bounds__(256, 2)
fft2048_colnoise_kernel(const float* __restrict__ sqrt_lam, const float2* __restrict__ tw,
                        const float2* __restrict__ tw32, int m,
                        const __grid_constant__ PhiloxKeys keys, uint32_t pair0, uint32_t event, float2* __restrict__ T) {
  constexpr int P = 2048;
  extern __shared__ __align__(16) float2 smf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* buf = smf + w * (32 * 33);
  float2* odd = smf + 8 * 32 * 33;   // [line][1024]: W^k O[k]
  float2* stage = smf;               // [k][line], over the transpose buffers after a barrier
  const int c = w >> 1, par = w & 1;
  const int b = blockIdx.x * kLines2048 + c;
  const int pl = blockIdx.y;
  const uint32_t pair = pair0 + (uint32_t)pl;
  const float* sl = sqrt_lam + (long long)b * P;
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int a = 2 * (lane + 32 * k) + par;   // < 1024; a + 1024 is element t + 512
    const uint4 x = philox4x32_10(make_uint4((uint32_t)(a * P + b), pair, 0u, event), keys);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float s0 = __ldg(sl + a), s1 = __ldg(sl + a + P / 2);
    v[k] = make_float2(s0 * z01.x, s0 * z01.y);
    v[k + 16] = make_float2(s1 * z23.x, s1 * z23.y);
  }
  fft32_reg(v);
  fft1024_finish(v, buf, tw32, lane);   // lane j holds the transform at j + 32 l in v[l]
  if (par) {
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int k = lane + 32 * l;
      if (k < m) odd[c * 1024 + k] = cmul(v[l], __ldg(tw + k));
    }
  }
  __syncthreads();
  if (!par) {
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int k = lane + 32 * l;
      if (k < m) {
        const float2 o = odd[c * 1024 + k];
        stage[k * kLines2048 + c] = make_float2(v[l].x + o.x, v[l].y + o.y);
      }
    }
  }
  __syncthreads();
  float2* dst = T + (long long)pl * m * P + blockIdx.x * kLines2048;
  for (int e = threadIdx.x; e < m * kLines2048; e += 256) {
    const int k = e / kLines2048, cc = e % kLines2048;
    dst[(long long)k * P + cc] = stage[e];
  }
}

// Row pass, P = 2048: rows k1 < m of T, two warps per row; the first m
// frequencies go to realizations 2p (real part) and 2p + 1 (imaginary part).
__global__ void __launch_bounds__(256, 2)
fft2048_rowout_kernel(const float2* __restrict__ T, const float2* __restrict__ tw, const float2* __restrict__ tw32,
                      int m, int R_local, int pair_local0,
                      float* __restrict__ out) {
  constexpr int P = 2048;
  extern __shared__ __align__(16) float2 smf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* buf = smf + w * (32 * 33);
  float2* odd = smf + 8 * 32 * 33;
  const int c = w >> 1, par = w & 1;
  const int row = blockIdx.x * kLines2048 + c;
  const bool live = row < m;   // every warp reaches the barrier
  const int pl = blockIdx.y;
  const float2* src = T + ((long long)pl * m + (live ? row : 0)) * P;
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = live ? src[2 * (lane + 32 * k) + par] : make_float2(0.f, 0.f);
  fft32_reg(v);
  fft1024_finish(v, buf, tw32, lane);
  if (par) {
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int k = lane + 32 * l;
      if (k < m) odd[c * 1024 + k] = cmul(v[l], __ldg(tw + k));
    }
  }
  __syncthreads();
  if (!par && live) {
    const int r_re = 2 * (pair_local0 + pl);
    const bool has_im = r_re + 1 < R_local;
    const long long M = (long long)m * m;
    float* o_re = out + r_re * M + (long long)row * m;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int k = lane + 32 * l;
      if (k < m) {
        const float2 o = odd[c * 1024 + k];
        o_re[k] = v[l].x + o.x;
        if (has_im) o_re[M + k] = v[l].y + o.y;
      }
    }
  }
}

// Launch the two passes for every chunk of pairs, the intermediate in T.
template <int P>
int launch_ensemble(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s, float2* T, int chunk) {
  const int m = ctx->m;
  const int pairs = (R + 1) / 2;
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  const uint32_t pair_base = (uint32_t)(r_offset / 2);
  const PhiloxKeys keys = philox_round_keys(k0, k1);
  if (P == 2048) {
    // transpose buffers (8 warps) + the odd halves of 4 lines; the output stage reuses the former
    const size_t shm = sizeof(float2) * ((size_t)8 * 32 * 33 + (size_t)kLines2048 * 1024);
    CE_CUDA_TRY(cudaFuncSetAttribute(fft2048_colnoise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    CE_CUDA_TRY(cudaFuncSetAttribute(fft2048_rowout_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    for (int p0 = 0; p0 < pairs; p0 += chunk) {
      const int np = std::min(chunk, pairs - p0);
      fft2048_colnoise_kernel<<<dim3(P / kLines2048, np), 256, shm, s>>>(ctx->sqrt_lam_t, ctx->twiddle, ctx->tw32, m, keys,
                                                                          pair_base + p0, 0u, T);
      fft2048_rowout_kernel<<<dim3((m + kLines2048 - 1) / kLines2048, np), 256, shm, s>>>(T, ctx->twiddle, ctx->tw32, m,
                                                                                            R, p0, y);
      ctx->launches += 2;
    }
  } else if (P == 1024) {
    // m <= P / 2, so the staged columns fit in the transpose buffers; 3 blocks per SM
    const size_t shm_c = sizeof(float2) * std::max((size_t)kFastWarps * 32 * 33, (size_t)m * kFastWarps);
    const size_t shm_r = sizeof(float2) * (size_t)kFastWarps * 32 * 33;
    CE_CUDA_TRY(cudaFuncSetAttribute(fft1024_colnoise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_c));
    CE_CUDA_TRY(cudaFuncSetAttribute(fft1024_rowout_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_r));
    for (int p0 = 0; p0 < pairs; p0 += chunk) {
      const int np = std::min(chunk, pairs - p0);
      fft1024_colnoise_kernel<<<dim3(P / kFastWarps, np), 32 * kFastWarps, shm_c, s>>>(ctx->sqrt_lam_t, ctx->tw32, m, keys,
                                                                                       pair_base + p0, 0u, T, ctx->dev_status);
      fft1024_rowout_kernel<false><<<dim3((m + kFastWarps - 1) / kFastWarps, np), 32 * kFastWarps, shm_r, s>>>(
          T, ctx->tw32, m, R, p0, y, ctx->dev_status);
      ctx->launches += 2;
    }
  } else {
    constexpr int CB = FftShape<P>::CB;
    constexpr int ROWS = FftShape<P>::ROWS;
    const size_t shm_c = sizeof(float2) * CB * P;
    const size_t shm_r = sizeof(float2) * ROWS * P;
    CE_CUDA_TRY(cudaFuncSetAttribute(fft_colnoise_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_c));
    CE_CUDA_TRY(cudaFuncSetAttribute(fft_rowout_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_r));
    for (int p0 = 0; p0 < pairs; p0 += chunk) {
      const int np = std::min(chunk, pairs - p0);
      fft_colnoise_kernel<P><<<dim3(P / CB, np), FftShape<P>::NT_COLS, shm_c, s>>>(ctx->sqrt_lam_t, ctx->twiddle, m, keys,
                                                                                   pair_base + p0, 0u, T);
      fft_rowout_kernel<P><<<dim3((m + ROWS - 1) / ROWS, np), FftShape<P>::NT_ROWS, shm_r, s>>>(T, ctx->twiddle, m, R,
                                                                                             p0, y);
      ctx->launches += 2;
    }
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

// Pairs per chunk: as many as keep the chunk's intermediate within fft_chunk_mb (64 MB
// of the 129 MB L2 by default; ce_autotune may pick another budget), balanced over the
// chunks (fewer, larger chunks also fill the last wave of the row pass better: 10 pairs
// of 512 rows are 1.4 waves of 24 warps per SM).
int ensemble_chunk(const ce_ctx* ctx, int R) {
  const int pairs = (R + 1) / 2;
  const size_t per_pair = sizeof(float2) * (size_t)ctx->P * ctx->m;
  int chunk = (int)std::max<size_t>(1, ((size_t)ctx->fft_chunk_mb << 20) / per_pair);
  chunk = std::min(chunk, pairs);
  const int nchunks = (pairs + chunk - 1) / chunk;
  return (pairs + nchunks - 1) / nchunks;
}

template <int P>
int run_ensemble(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y, cudaStream_t s) {
  const int st = ensure_fft_buffer(ctx, R);
  if (st) return st;
  return launch_ensemble<P>(ctx, R, seed, r_offset, y, s, ctx->T, ensemble_chunk(ctx, R));
}


// ---------------------------------------------------------------------------
// Adjoint of the ensemble through the spectral weights (gradient): for every
// realization pair p, Y = DFT2(h_{2p} - i h_{2p+1}) with h embedded in the
// m x m corner of the P x P torus, then acc[0] += sum_a dsdt_a Re(eps_a Y_a) and
// acc[1] += sum_a (s_a / sigma) Re(eps_a Y_a), eps the same complex noise as the
// forward pass.  Columns first (only the m nonzero columns), then every row.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_COLS)
adj_cols_kernel(const float* __restrict__ H, int m, int R_local, int pair_local0, const float2* __restrict__ tw,
                float2* __restrict__ T) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int kNT = FftShape<P>::NT_COLS;
  extern __shared__ __align__(16) float2 smc[];
  const int b0 = blockIdx.x * CB;
  const int pl = blockIdx.y;
  const int r_re = 2 * (pair_local0 + pl);
  const bool has_im = r_re + 1 < R_local;
  const long long M = (long long)m * m;
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, a = e / CB;
    float2 x = make_float2(0.f, 0.f);
    if (a < m && b0 + c < m) {
      const long long o = (long long)a * m + b0 + c;
      x.x = H[r_re * M + o];
      if (has_im) x.y = -H[(r_re + 1) * M + o];
    }
    smc[c * P + a] = x;
  }
  __syncthreads();
  fft_lines_smem<P, CB, kNT>(smc, tw);
  float2* dst = T + (long long)pl * P * m;
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, kk = e / CB;
    if (b0 + c < m) dst[(long long)kk * m + b0 + c] = smc[c * P + kk];
  }
}

template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_ROWS)
adj_rows_kernel(const float2* __restrict__ T, int m, const float2* __restrict__ tw, const float* __restrict__ sqrt_lam,
                const float* __restrict__ dsdt, float inv_sigma, uint32_t k0, uint32_t k1, uint32_t pair0,
                double* __restrict__ acc) {
  constexpr int ROWS = FftShape<P>::ROWS;
  constexpr int kNT = FftShape<P>::NT_ROWS;
  extern __shared__ __align__(16) float2 sm[];
  __shared__ double red[2][32];
  const int a0 = blockIdx.x * ROWS;
  const int pl = blockIdx.y;
  const uint32_t pair = pair0 + (uint32_t)pl;
  const float2* src = T + (long long)pl * P * m;
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, b = e % P;
    sm[e] = (b < m) ? src[(long long)(a0 + row) * m + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, ROWS, kNT>(sm, tw);
  double st = 0.0, ss = 0.0;
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, b = e % P;
    const int a = a0 + row;
    const int ah = a < P / 2 ? a : a - P / 2;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)(ah * P + b), pair, 0u, 0u), k0, k1);
    const float2 z = a < P / 2 ? box_muller(x.x, x.y) : box_muller(x.z, x.w);
    const float2 y = sm[e];
    const float re = z.x * y.x - z.y * y.y;
    const long long o = (long long)a * P + b;
    st += (double)dsdt[o] * re;
    ss += (double)(sqrt_lam[o] * inv_sigma) * re;
  }
  for (int o = 16; o; o >>= 1) {
    st += __shfl_xor_sync(0xffffffffu, st, o);
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = st; red[1][threadIdx.x >> 5] = ss; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < (kNT + 31) / 32; ++w) { t0 += red[0][w]; t1 += red[1][w]; }
    atomicAdd(acc + 0, t0);
    atomicAdd(acc + 1, t1);
  }
}

template <int P>
int run_adjoint(ce_ctx* ctx, const float* H, int R, uint64_t seed, uint64_t r_offset, double* acc, cudaStream_t s) {
  const int m = ctx->m;
  const int pairs = (R + 1) / 2;
  int st = ensure_fft_buffer(ctx, R);
  if (st) return st;
  const int chunk = ensemble_chunk(ctx, R);
  constexpr int CB = FftShape<P>::CB;
  constexpr int ROWS = FftShape<P>::ROWS;
  const size_t shm_c = sizeof(float2) * CB * P;
  const size_t shm_r = sizeof(float2) * ROWS * P;
  CE_CUDA_TRY(cudaFuncSetAttribute(adj_cols_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_c));
  CE_CUDA_TRY(cudaFuncSetAttribute(adj_rows_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_r));
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  const float inv_sigma = (float)(1.0 / ctx->sigma);
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    adj_cols_kernel<P><<<dim3((m + CB - 1) / CB, np), FftShape<P>::NT_COLS, shm_c, s>>>(H, m, R, p0, ctx->twiddle, ctx->T);
    adj_rows_kernel<P><<<dim3(P / ROWS, np), FftShape<P>::NT_ROWS, shm_r, s>>>(
        ctx->T, m, ctx->twiddle, ctx->sqrt_lam, ctx->ds_theta, inv_sigma, k0, k1, (uint32_t)(r_offset / 2) + p0, acc);
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

// ---------------------------------------------------------------------------
// The circulant NN correction at P = 1024 (the convolution of Section 2.1 (a)
// applied to the weights scattered on the torus), in three register passes of
// one warp per line: rows forward (inputs past column m are zero), columns
// forward, times lambda / N, conjugated, and forward again keeping the first m
// outputs (one kernel, the column stays in registers), rows forward keeping the
// first m outputs, added to the fields with the final conjugation
// (fft1024_rowout_kernel<true>).
// ---------------------------------------------------------------------------

// S: pairs x m x m scatter of the weights (pair p: B[2p] + i B[2p+1]); zero first.
__global__ void circ1024_scatter_kernel(const float* __restrict__ B, int ldb, int R, int nobs, const int* __restrict__ node,
                                        int m, int pair0, float2* __restrict__ S) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int pl = blockIdx.y;
  if (q >= nobs) return;
  const int r = 2 * (pair0 + pl);
  const float re = B[(long long)r * ldb + q];
  const float im = r + 1 < R ? B[(long long)(r + 1) * ldb + q] : 0.f;
  S[(long long)pl * m * m + node[q]] = make_float2(re, im);
}

// Rows i < m of S, zero-padded to 1024 points: all 1024 outputs to T (pairs x m x 1024).
__global__ void __launch_bounds__(32 * kFastWarps, 3)
circ1024_rowfwd_kernel(const float2* __restrict__ S, int m, const float2* __restrict__ tw32, float2* __restrict__ T) {
  extern __shared__ __align__(16) float2 smf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* buf = smf + w * (32 * 33);
  const int row = blockIdx.x * kFastWarps + w;
  if (row >= m) return;   // no block barrier below
  const int pl = blockIdx.y;
  const float2* src = S + ((long long)pl * m + row) * m;
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int a = lane + 32 * k;
    v[k] = a < m ? src[a] : make_float2(0.f, 0.f);
  }
  fft32_reg(v);
  fft1024_finish(v, buf, tw32, lane);
  float2* dst = T + ((long long)pl * m + row) * 1024;
#pragma unroll
  for (int l = 0; l < 32; ++l) dst[lane + 32 * l] = v[l];
}

// Columns c0 .. c0 + 7 of T (rows i < m; rows past m are zero): forward transform,
// times lambda / N = sqrt_lam^2 (the column's weights read from the transposed copy),
// conjugated, forward transform again, first m outputs written back in place.
// two blocks per SM: with two transforms in flight the line needs more than 80 registers
__global__ void __launch_bounds__(32 * kFastWarps, 2)
circ1024_col_kernel(float2* __restrict__ T, int m, const float* __restrict__ sqrt_lam_t, const float2* __restrict__ tw32) {
  constexpr int P = 1024, LD = kFastWarps + 1;   // stage row stride (padded against bank conflicts)
  extern __shared__ __align__(16) float2 smf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* buf = smf + w * (32 * 33);
  float2* stage = smf;   // [row][LD], over the transpose buffers between barriers
  const int c0 = blockIdx.x * kFastWarps;
  float2* Tp = T + (long long)blockIdx.y * m * P;
  for (int e = threadIdx.x; e < m * kFastWarps; e += 32 * kFastWarps) {
    const int i = e / kFastWarps, c = e % kFastWarps;
    stage[i * LD + c] = Tp[(long long)i * P + c0 + c];
  }
  __syncthreads();
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int a = lane + 32 * k;
    v[k] = a < m ? stage[a * LD + w] : make_float2(0.f, 0.f);
  }
  __syncthreads();   // every warp has its column before the transposes reuse the stage
  fft32_reg(v);
  fft1024_finish(v, buf, tw32, lane);   // lane j: frequency j + 32 l in v[l]
  const float* sl = sqrt_lam_t + (long long)(c0 + w) * P;
  // in groups of eight, each behind a compiler barrier, so that the weights' loads are not
  // all hoisted beside the 64 registers of the line
#pragma unroll
  for (int l0 = 0; l0 < 32; l0 += 8) {
    asm volatile("" ::: "memory");
#pragma unroll
    for (int l = l0; l < l0 + 8; ++l) {
      const float sv = sl[lane + 32 * l];
      const float lam = sv * sv;
      v[l] = make_float2(lam * v[l].x, -lam * v[l].y);
    }
  }
  asm volatile("" ::: "memory");
  fft32_reg(v);
  fft1024_finish<true>(v, buf, tw32, lane);   // outputs j + 32 l < m <= 512: l < 16
  __syncthreads();   // every warp is done with its transpose buffer
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const int a = lane + 32 * l;
    if (a < m) stage[a * LD + w] = v[l];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * kFastWarps; e += 32 * kFastWarps) {
    const int i = e / kFastWarps, c = e % kFastWarps;
    Tp[(long long)i * P + c0 + c] = stage[i * LD + c];
  }
}

}  // namespace

int ensure_fft_buffer(ce_ctx* ctx, int R) {
  const int chunk = ensemble_chunk(ctx, R);
  if (ctx->Tpairs >= chunk) return CE_OK;
  dfree(ctx, ctx->T);
  ctx->T = (float2*)dalloc(ctx, sizeof(float2) * (size_t)ctx->P * ctx->m * chunk);
  if (!ctx->T) { ctx->Tpairs = 0; return fail(ctx, CE_ERR_OOM, "FFT intermediate"); }
  ctx->Tpairs = chunk;
  return CE_OK;
}

// The circulant NN correction at P = 1024 on the chunk buffer ctx->Xc (per pair
// m x m scatter + m x 1024 rows, within the P x P complex the buffer holds per pair).
int circulant_correct_1024(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  constexpr int P = 1024;
  const int m = ctx->m;
  if (ctx->P != P || m > P / 2) return fail(ctx, CE_ERR_ARG, "register circulant correction: P = 1024 only");
  const int pairs = (R + 1) / 2;
  const int chunk = ctx->circ_pairs;
  const size_t shm = sizeof(float2) * std::max((size_t)kFastWarps * 32 * 33, (size_t)m * (kFastWarps + 1));
  CE_CUDA_TRY(cudaFuncSetAttribute(circ1024_rowfwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  CE_CUDA_TRY(cudaFuncSetAttribute(circ1024_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  CE_CUDA_TRY(cudaFuncSetAttribute(fft1024_rowout_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    float2* S = ctx->Xc;
    float2* T = S + ((size_t)np * m * m + 1) / 2 * 2;   // 16-byte aligned rows for the bulk copies
    CE_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(float2) * (size_t)np * m * m, s));
    circ1024_scatter_kernel<<<dim3((ctx->nobs + 255) / 256, np), 256, 0, s>>>(B, ctx->nobs_pad, R, ctx->nobs, ctx->idx, m,
                                                                              p0, S);
    circ1024_rowfwd_kernel<<<dim3((m + kFastWarps - 1) / kFastWarps, np), 32 * kFastWarps, shm, s>>>(S, m, ctx->tw32, T);
    circ1024_col_kernel<<<dim3(P / kFastWarps, np), 32 * kFastWarps, shm, s>>>(T, m, ctx->sqrt_lam_t, ctx->tw32);
    fft1024_rowout_kernel<true><<<dim3((m + kFastWarps - 1) / kFastWarps, np), 32 * kFastWarps, shm, s>>>(
        T, ctx->tw32, m, R, p0, y, ctx->dev_status);
    ctx->launches += 4;
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

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

int launch_adjoint_ensemble(ce_ctx* ctx, const float* H, int R, uint64_t seed, uint64_t r_offset, double* acc,
                            cudaStream_t s) {
  switch (ctx->P) {
    case 16: return run_adjoint<16>(ctx, H, R, seed, r_offset, acc, s);
    case 32: return run_adjoint<32>(ctx, H, R, seed, r_offset, acc, s);
    case 64: return run_adjoint<64>(ctx, H, R, seed, r_offset, acc, s);
    case 128: return run_adjoint<128>(ctx, H, R, seed, r_offset, acc, s);
    case 256: return run_adjoint<256>(ctx, H, R, seed, r_offset, acc, s);
    case 512: return run_adjoint<512>(ctx, H, R, seed, r_offset, acc, s);
    case 1024: return run_adjoint<1024>(ctx, H, R, seed, r_offset, acc, s);
    case 2048: return run_adjoint<2048>(ctx, H, R, seed, r_offset, acc, s);
    case 4096: return run_adjoint<4096>(ctx, H, R, seed, r_offset, acc, s);
    case 8192: return run_adjoint<8192>(ctx, H, R, seed, r_offset, acc, s);
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
  const int pairs = (R + 1) / 2;
  const size_t per_pair = sizeof(float2) * (size_t)P * ctx->m;
  if (per_pair > T_bytes) return fail(ctx, CE_ERR_ARG, "one realization pair needs more scratch than the fixed buffer holds");
  const int chunk = (int)std::min<size_t>((size_t)pairs, T_bytes / per_pair);
  return launch_ensemble<P>(ctx, R, seed, r_offset, y, s, T, chunk);
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
