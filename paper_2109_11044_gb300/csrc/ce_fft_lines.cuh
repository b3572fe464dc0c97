// Shared-memory FFT building blocks used by the ensemble (ce_fft.cu) and by the
// circulant correction of NN Kriging (ce_circulant.cu): LINES forward FFTs of
// length P (a power of two) held back to back in shared memory, radix-4
// Stockham stages with one radix-2 stage when log2 P is odd, and the block
// shapes of the column and row passes.
#pragma once

#include <cuda_runtime.h>

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


}  // namespace
}  // namespace ce
