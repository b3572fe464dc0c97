// Kriging correction for nearest-neighbour Kriging as a circulant convolution.
//
// In NN mode (Section 2.2, Section 3.2) the surrogate data sit on grid nodes, so for a
// grid node g and a surrogate node s both inside the m x m grid,
// C(g, s) = c[(g - s) mod P] with c the first row of the block-circulant
// embedding on the P x P torus: every lag inside the grid is below m <= P/2,
// so the torus distance is the true distance.  Hence
//   K_gN B_r = (c * b_r) restricted to the grid,
// with b_r the weights of realization r scattered onto the torus and * the 2-D
// circular convolution, and c * b = F^-1(lambda . F(b)) = (1/N) conj F conj
// (lambda . F(b)), lambda = F(c) the embedding eigenvalues of Section 2.1 (a).
// Realizations 2p and 2p+1 travel together as the real and imaginary parts of
// one complex field (c and lambda are real), as in the unconditional ensemble.
// The transform uses the eigenvalues as stored for the ensemble (negative ones
// clipped to zero), so it reproduces the embedding's covariance, which equals
// C on the grid up to the clipped part.
//
// Per chunk of pairs, on a P x P complex buffer X per pair:
//   1. zero X, scatter (B[2p][q], B[2p+1][q]) to the node of surrogate q;
//   2. column transforms of the m columns that can be non-zero, all P outputs;
//   3. row transforms of all P rows, times lambda / N, conjugated;
//   4. column transforms of all P columns, only the m rows the grid needs;
//   5. row transforms of those m rows; y[2p] += Re, y[2p+1] -= Im of the
//      first m outputs (the final conjugation).
#include <algorithm>

#include "ce_common.cuh"
#include "ce_fft_lines.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

__global__ void circ_scatter_kernel(const float* __restrict__ B, int ldb, int R, int nobs, const int* __restrict__ node,
                                    int m, int P, int pair0, float2* __restrict__ X) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int pl = blockIdx.y;
  if (q >= nobs) return;
  const int r = 2 * (pair0 + pl);
  const float re = B[(long long)r * ldb + q];
  const float im = r + 1 < R ? B[(long long)(r + 1) * ldb + q] : 0.f;
  const int g = node[q], i = g / m, j = g % m;
  X[((long long)pl * P + i) * P + j] = make_float2(re, im);
}

// Columns j0 .. j0+CB-1 (< m) of pair pl: rows >= m are zero on input.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_COLS)
circ_colfwd_kernel(float2* __restrict__ X, int m, const float2* __restrict__ tw) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int kNT = FftShape<P>::NT_COLS;
  extern __shared__ __align__(16) float2 smx[];
  const int j0 = blockIdx.x * CB;
  float2* Xp = X + (long long)blockIdx.y * P * P;
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, a = e / CB;
    smx[c * P + a] = (a < m && j0 + c < m) ? Xp[(long long)a * P + j0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, CB, kNT>(smx, tw);
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, a = e / CB;
    if (j0 + c < m) Xp[(long long)a * P + j0 + c] = smx[c * P + a];
  }
}

// Rows r0 .. r0+ROWS-1 of pair pl (columns >= m are zero on input); the
// spectrum is multiplied by lambda / N = sqrt_lam^2 and conjugated.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_ROWS)
circ_rowfwd_kernel(float2* __restrict__ X, int m, const float* __restrict__ sqrt_lam, const float2* __restrict__ tw) {
  constexpr int ROWS = FftShape<P>::ROWS;
  constexpr int kNT = FftShape<P>::NT_ROWS;
  extern __shared__ __align__(16) float2 smx[];
  const int r0 = blockIdx.x * ROWS;
  float2* Xp = X + (long long)blockIdx.y * P * P;
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, b = e % P;
    smx[e] = b < m ? Xp[(long long)(r0 + row) * P + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, ROWS, kNT>(smx, tw);
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, k = e % P;
    const float s = sqrt_lam[(long long)(r0 + row) * P + k];
    const float l = s * s;
    const float2 w = smx[e];
    Xp[(long long)(r0 + row) * P + k] = make_float2(l * w.x, -l * w.y);
  }
}

// All P columns of pair pl; only the first m outputs of each are kept.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_COLS)
circ_colinv_kernel(float2* __restrict__ X, int m, const float2* __restrict__ tw) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int kNT = FftShape<P>::NT_COLS;
  extern __shared__ __align__(16) float2 smx[];
  const int j0 = blockIdx.x * CB;
  float2* Xp = X + (long long)blockIdx.y * P * P;
  for (int e = threadIdx.x; e < CB * P; e += kNT) {
    const int c = e % CB, a = e / CB;
    smx[c * P + a] = Xp[(long long)a * P + j0 + c];
  }
  __syncthreads();
  fft_lines_smem<P, CB, kNT>(smx, tw);
  for (int e = threadIdx.x; e < CB * m; e += kNT) {
    const int c = e % CB, a = e / CB;
    Xp[(long long)a * P + j0 + c] = smx[c * P + a];
  }
}

// Rows i < m of pair pl: y[2p][i][k] += Re, y[2p+1][i][k] -= Im for k < m.
template <int P>
__global__ void __launch_bounds__(FftShape<P>::NT_ROWS)
circ_rowinv_add_kernel(const float2* __restrict__ X, int m, int R, int pair0, const float2* __restrict__ tw,
                       float* __restrict__ y) {
  constexpr int ROWS = FftShape<P>::ROWS;
  constexpr int kNT = FftShape<P>::NT_ROWS;
  extern __shared__ __align__(16) float2 smx[];
  const int r0 = blockIdx.x * ROWS;
  const int pl = blockIdx.y;
  const float2* Xp = X + (long long)pl * P * P;
  for (int e = threadIdx.x; e < ROWS * P; e += kNT) {
    const int row = e / P, b = e % P;
    smx[e] = r0 + row < m ? Xp[(long long)(r0 + row) * P + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_lines_smem<P, ROWS, kNT>(smx, tw);
  const int r = 2 * (pair0 + pl);
  const bool has_im = r + 1 < R;
  const long long M = (long long)m * m;
  for (int e = threadIdx.x; e < ROWS * m; e += kNT) {
    const int row = e / m, k = e % m;
    if (r0 + row >= m) continue;
    const float2 w = smx[row * P + k];
    const long long o = (long long)(r0 + row) * m + k;
    y[r * M + o] += w.x;
    if (has_im) y[(r + 1) * M + o] -= w.y;
  }
}

template <int P>
int run_circulant(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  constexpr int CB = FftShape<P>::CB;
  constexpr int ROWS = FftShape<P>::ROWS;
  const int m = ctx->m;
  const int pairs = (R + 1) / 2;
  const int chunk = ctx->circ_pairs;
  const size_t shm_c = sizeof(float2) * CB * P, shm_r = sizeof(float2) * ROWS * P;
  CE_CUDA_TRY(cudaFuncSetAttribute(circ_colfwd_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_c));
  CE_CUDA_TRY(cudaFuncSetAttribute(circ_colinv_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_c));
  CE_CUDA_TRY(cudaFuncSetAttribute(circ_rowfwd_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_r));
  CE_CUDA_TRY(cudaFuncSetAttribute(circ_rowinv_add_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_r));
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    CE_CUDA_TRY(cudaMemsetAsync(ctx->Xc, 0, sizeof(float2) * (size_t)np * P * P, s));
    circ_scatter_kernel<<<dim3((ctx->nobs + 255) / 256, np), 256, 0, s>>>(B, ctx->nobs_pad, R, ctx->nobs, ctx->idx, m, P,
                                                                          p0, ctx->Xc);
    circ_colfwd_kernel<P><<<dim3((m + CB - 1) / CB, np), FftShape<P>::NT_COLS, shm_c, s>>>(ctx->Xc, m, ctx->twiddle);
    circ_rowfwd_kernel<P><<<dim3(P / ROWS, np), FftShape<P>::NT_ROWS, shm_r, s>>>(ctx->Xc, m, ctx->sqrt_lam, ctx->twiddle);
    circ_colinv_kernel<P><<<dim3(P / CB, np), FftShape<P>::NT_COLS, shm_c, s>>>(ctx->Xc, m, ctx->twiddle);
    circ_rowinv_add_kernel<P><<<dim3((m + ROWS - 1) / ROWS, np), FftShape<P>::NT_ROWS, shm_r, s>>>(ctx->Xc, m, R, p0,
                                                                                               ctx->twiddle, y);
    ctx->launches += 5;
  }
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

}  // namespace

// Pairs per chunk: as many as keep the chunk's P x P buffers within about 64 MB.
int ensure_circulant_buffer(ce_ctx* ctx, int R) {
  const int pairs = (R + 1) / 2;
  const size_t per_pair = sizeof(float2) * (size_t)ctx->P * ctx->P;
  const int chunk = (int)std::min<size_t>((size_t)pairs, std::max<size_t>(1, (64u << 20) / per_pair));
  if (ctx->Xc && ctx->circ_pairs >= chunk) return CE_OK;
  dfree(ctx, ctx->Xc);
  ctx->Xc = (float2*)dalloc(ctx, per_pair * chunk);
  ctx->circ_pairs = ctx->Xc ? chunk : 0;
  if (!ctx->Xc) return fail(ctx, CE_ERR_OOM, "circulant correction buffer");
  return CE_OK;
}

int launch_correct_circulant(ce_ctx* ctx, const float* B, int R, float* y, cudaStream_t s) {
  int st = ensure_circulant_buffer(ctx, R);
  if (st) return st;
  switch (ctx->P) {
    case 16: return run_circulant<16>(ctx, B, R, y, s);
    case 32: return run_circulant<32>(ctx, B, R, y, s);
    case 64: return run_circulant<64>(ctx, B, R, y, s);
    case 128: return run_circulant<128>(ctx, B, R, y, s);
    case 256: return run_circulant<256>(ctx, B, R, y, s);
    case 512: return run_circulant<512>(ctx, B, R, y, s);
    case 1024: return circulant_correct_1024(ctx, B, R, y, s);   // register passes
    case 2048: return run_circulant<2048>(ctx, B, R, y, s);
    case 4096: return run_circulant<4096>(ctx, B, R, y, s);
    case 8192: return run_circulant<8192>(ctx, B, R, y, s);
    default: return fail(ctx, CE_ERR_ARG, "unsupported embedding size");
  }
}

}  // namespace ce
