// Dense linear algebra of the Kriging step (Eq. (condmvn); Section 3.1).
//  - FP64, once per site set: blocked right-looking Cholesky A = L L^T of the
//    prediction matrix, then A^-1 by two blocked triangular solves with the
//    identity as right-hand side, stored as an FP32 pair hi + lo.
//  - FP32, per call: B = E (A^-1_hi + A^-1_lo) for the R x n residual block E
//    (A^-1 is symmetric, so this is (A^-1 E^T)^T).  Sums run over 32-term
//    chunks whose partial results are added with Kahan compensation.
#include <cmath>
#include <vector>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int NB = 32;   // diagonal block size

// Cholesky of the nb x nb diagonal block at (kb, kb), in place (lower part).
__global__ void __launch_bounds__(256) potrf_diag(double* __restrict__ A, int n, int kb, int nb, int* __restrict__ status) {
  __shared__ double s[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    s[i][j] = A[(long long)(kb + i) * n + kb + j];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = s[j][j];
      if (!(d > 0.0)) { atomicExch(status, CE_ERR_NOT_SPD); s[j][j] = 1.0; }
      else s[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][j] /= s[j][j];
    __syncthreads();
    for (int e = threadIdx.x; e < (nb - j - 1) * (nb - j - 1); e += blockDim.x) {
      const int i = j + 1 + e / (nb - j - 1), c = j + 1 + e % (nb - j - 1);
      if (c <= i) s[i][c] -= s[i][j] * s[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    A[(long long)(kb + i) * n + kb + j] = j <= i ? s[i][j] : 0.0;
  }
}

// Panel below the diagonal block: rows i >= kb+nb solve x L11^T = a_i.
__global__ void __launch_bounds__(128) trsm_panel(double* __restrict__ A, int n, int kb, int nb) {
  __shared__ double L[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) L[e / nb][e % nb] = A[(long long)(kb + e / nb) * n + kb + e % nb];
  __syncthreads();
  const int i = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[NB];
  double* row = A + (long long)i * n + kb;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nb) {
      double v = row[j];
      for (int t = 0; t < j; ++t) v -= x[t] * L[j][t];
      x[j] = v / L[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) if (j < nb) row[j] = x[j];
}

// C (M x N, ldc) -= opA(A) (M x K) * opB(B) (K x N).  TA: A stored K x M (lda).
// TB: B stored N x K (ldb).  LOWER: only tiles with row block >= column block,
// and only elements with row >= column.  64 x 64 tiles, 256 threads, 4 x 4 each.
template <bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(256) gemm64_sub(const double* __restrict__ A, int lda, const double* __restrict__ B, int ldb,
                                                  double* __restrict__ C, int ldc, int M, int N, int K) {
  const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
  if (LOWER && bn > bm + 63) return;
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int gm = bm + mm, gk = k0 + kk;
      double va = 0.0;
      if (gm < M && gk < K) va = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = va;
      const int gn = bn + mm;
      double vb = 0.0;
      if (gn < N && gk < K) vb = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][mm] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty + 16 * i]; b[i] = Bs[kk][tx + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = bm + ty + 16 * i, gn = bn + tx + 16 * j;
      if (gm < M && gn < N && (!LOWER || gn <= gm)) C[(long long)gm * ldc + gn] -= acc[i][j];
    }
}

// Forward solve of a diagonal block for all right-hand-side columns:
// X[kb..kb+nb, c] = L_bb^-1 X[kb..kb+nb, c]  (LOWER=true), or the transposed
// back substitution X = L_bb^-T X (LOWER=false).  One thread per column.
template <bool FORWARD>
__global__ void __launch_bounds__(128) trsv_block(const double* __restrict__ L, int n, int kb, int nb, double* __restrict__ X,
                                                  int ldx, int ncols) {
  __shared__ double S[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) S[e / nb][e % nb] = L[(long long)(kb + e / nb) * n + kb + e % nb];
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = j < nb ? X[(long long)(kb + j) * ldx + c] : 0.0;
  if (FORWARD) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j < nb) {
        double v = x[j];
        for (int t = 0; t < j; ++t) v -= S[j][t] * x[t];
        x[j] = v / S[j][j];
      }
    }
  } else {
#pragma unroll
    for (int jj = NB - 1; jj >= 0; --jj) {
      if (jj < nb) {
        double v = x[jj];
        for (int t = jj + 1; t < nb; ++t) v -= S[t][jj] * x[t];
        x[jj] = v / S[jj][jj];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) if (j < nb) X[(long long)(kb + j) * ldx + c] = x[j];
}

__global__ void identity_kernel(double* __restrict__ X, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)n * n) X[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void diag_kernel(const double* __restrict__ L, int n, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = L[(long long)i * n + i];
}

// hi = fp32(X), lo = fp32(X - hi), into an ld-padded layout.
__global__ void split_kernel(const double* __restrict__ X, int n, float* __restrict__ hi, float* __restrict__ lo, int ld) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const double v = X[e];
  const float h = (float)v;
  hi[(long long)i * ld + j] = h;
  lo[(long long)i * ld + j] = (float)(v - (double)h);
}

// ---------------------------------------------------------------------------
// Per-call FP32 solve: Bout (R x ldb) = E (R x n) * (Ahi + Alo) (n x n, lda).
// Block tile: 32 rows of E x 64 columns, 128 threads with 4 x 4 outputs each;
// the K range is split over KSPLIT blocks whose partial results a second
// kernel adds.  The next 32-term chunk is copied into shared memory with
// cp.async while the current one is multiplied (two buffers).
// The rows of A^-1 alternate in sign and the sum cancels heavily, and the
// correction that follows amplifies every error of B by the cancellation of
// its own sum, so each output is a compensated dot product in the manner of
// Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput.
// 26, 2005): the running sum is updated by an error-free TwoSum (Knuth) and
// its rounding errors, with the lo products, gather in a second FP32
// accumulator.  Two hi products are first joined by one FMA (a rounding
// relative to two terms, not to the running sum), which halves the work of
// the compensated form for an error a little above one rounding of B.  Each
// partial result is written as that (sum, compensation) pair; the reduction
// joins the pairs as a float pair and rounds once.
// ---------------------------------------------------------------------------
constexpr int SV_TR = 32, SV_TC = 64, SV_KC = 32, SV_KSPLIT = kSolveKSplit;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 4- and 16-byte asynchronous copies; a copy marked invalid writes zeros and reads nothing.
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// CHAIN = 2 or 4: the hi products are summed in FP32 CHAIN at a time and each such partial
// joins the running sum by an error-free TwoSum (the error kept in the compensation with
// the lo products); CHAIN = 0: plain per-chunk sums joined with Kahan compensation.
template <int CHAIN>
__global__ void __launch_bounds__(128) solve_gemm_f32(const float* __restrict__ E, int R, int n,
                                                      const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                                      int lda, float* __restrict__ part) {
  __shared__ __align__(16) float Es[2][SV_TR][SV_KC + 1];
  __shared__ __align__(16) float Hs[2][SV_KC][SV_TC];
  __shared__ __align__(16) float Ls[2][SV_KC][SV_TC];
  const int c0 = blockIdx.x * SV_TC, r0 = blockIdx.y * SV_TR;
  const int kper = ((n + SV_KSPLIT - 1) / SV_KSPLIT + SV_KC - 1) / SV_KC * SV_KC;
  const int kbeg = blockIdx.z * kper, kend = min(n, kbeg + kper);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const bool live = r0 + ty * 4 < R;

  // Issue the copies of the chunk starting at k0 into buffer bf.
  auto load = [&](int bf, int k0) {
    for (int e = threadIdx.x; e < SV_TR * SV_KC; e += 128) {
      const int rr = e / SV_KC, kk = e % SV_KC;
      const bool ok = r0 + rr < R && k0 + kk < kend;
      cp_async4(smem_addr(&Es[bf][rr][kk]), ok ? E + (long long)(r0 + rr) * n + k0 + kk : E, ok);
    }
    for (int e = threadIdx.x; e < SV_KC * SV_TC / 4; e += 128) {
      const int kk = e / (SV_TC / 4), cc = (e % (SV_TC / 4)) * 4;
      const bool ok = k0 + kk < kend && c0 + cc < lda;   // lda is a multiple of 128: whole float4 in range
      const long long off = ok ? (long long)(k0 + kk) * lda + c0 + cc : 0;
      cp_async16(smem_addr(&Hs[bf][kk][cc]), Ahi + off, ok);
      cp_async16(smem_addr(&Ls[bf][kk][cc]), Alo + off, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  float sum[4][4], comp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { sum[i][j] = 0.f; comp[i][j] = 0.f; }
  if (kbeg < kend) load(0, kbeg);
  int bf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += SV_KC, bf ^= 1) {
    if (k0 + SV_KC < kend) {
      load(bf ^ 1, k0 + SV_KC);   // that buffer was released by the barrier that ended the last chunk
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (!live) {
      // all four rows of this thread lie past R (the last row tile is partly empty when
      // R is not a multiple of SV_TR): whole warps skip the products
    } else if constexpr (CHAIN == 2) {
#pragma unroll 2
      for (int kk = 0; kk < SV_KC; kk += 2) {   // SV_KC is even; rows past kend were copied as zeros
        const float4 h4a = *reinterpret_cast<const float4*>(&Hs[bf][kk][tx * 4]);
        const float4 h4b = *reinterpret_cast<const float4*>(&Hs[bf][kk + 1][tx * 4]);
        const float4 l4a = *reinterpret_cast<const float4*>(&Ls[bf][kk][tx * 4]);
        const float4 l4b = *reinterpret_cast<const float4*>(&Ls[bf][kk + 1][tx * 4]);
        float ea[4], eb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { ea[i] = Es[bf][ty * 4 + i][kk]; eb[i] = Es[bf][ty * 4 + i][kk + 1]; }
        const float ha[4] = {h4a.x, h4a.y, h4a.z, h4a.w}, hb[4] = {h4b.x, h4b.y, h4b.z, h4b.w};
        const float la[4] = {l4a.x, l4a.y, l4a.z, l4a.w}, lb[4] = {l4b.x, l4b.y, l4b.z, l4b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // p = e_a hi_a + e_b hi_b (one rounding); (t, es) = TwoSum(sum, p); es and the lo products to comp
            const float p = fmaf(eb[i], hb[j], __fmul_rn(ea[i], ha[j]));
            const float t = __fadd_rn(sum[i][j], p);
            const float z = __fsub_rn(t, sum[i][j]);
            const float es = __fadd_rn(__fsub_rn(sum[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));
            sum[i][j] = t;
            comp[i][j] = fmaf(eb[i], lb[j], fmaf(ea[i], la[j], comp[i][j] + es));
          }
      }
    } else if constexpr (CHAIN == 4) {
#pragma unroll 1
      for (int kk = 0; kk < SV_KC; kk += 4) {   // SV_KC is a multiple of 4; rows past kend were copied as zeros
        float hv[4][4], lv[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 h4 = *reinterpret_cast<const float4*>(&Hs[bf][kk + q][tx * 4]);
          const float4 l4 = *reinterpret_cast<const float4*>(&Ls[bf][kk + q][tx * 4]);
          hv[q][0] = h4.x; hv[q][1] = h4.y; hv[q][2] = h4.z; hv[q][3] = h4.w;
          lv[q][0] = l4.x; lv[q][1] = l4.y; lv[q][2] = l4.z; lv[q][3] = l4.w;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float ev[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ev[q] = Es[bf][ty * 4 + i][kk + q];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // p = the four hi products summed in FP32; (t, es) = TwoSum(sum, p); es and the
            // lo products to comp
            const float p = fmaf(ev[3], hv[3][j], fmaf(ev[2], hv[2][j], fmaf(ev[1], hv[1][j], __fmul_rn(ev[0], hv[0][j]))));
            const float t = __fadd_rn(sum[i][j], p);
            const float z = __fsub_rn(t, sum[i][j]);
            const float es = __fadd_rn(__fsub_rn(sum[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));
            sum[i][j] = t;
            comp[i][j] = fmaf(ev[3], lv[3][j], fmaf(ev[2], lv[2][j], fmaf(ev[1], lv[1][j], fmaf(ev[0], lv[0][j], comp[i][j] + es))));
          }
        }
      }
    } else {
      // plain form: per chunk the hi and lo products accumulate in FP32 (apart, so the lo
      // part is not absorbed); chunk sums join the running sum with Kahan compensation
      float ph[4][4], pl[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { ph[i][j] = 0.f; pl[i][j] = 0.f; }
#pragma unroll 8
      for (int kk = 0; kk < SV_KC; ++kk) {
        const float4 h4 = *reinterpret_cast<const float4*>(&Hs[bf][kk][tx * 4]);
        const float4 l4 = *reinterpret_cast<const float4*>(&Ls[bf][kk][tx * 4]);
        const float ev[4] = {Es[bf][ty * 4][kk], Es[bf][ty * 4 + 1][kk], Es[bf][ty * 4 + 2][kk], Es[bf][ty * 4 + 3][kk]};
        const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            ph[i][j] = fmaf(ev[i], hv[j], ph[i][j]);
            pl[i][j] = fmaf(ev[i], lv[j], pl[i][j]);
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {   // Kahan: sum += (hi part + lo part); comp holds the negated error
          const float yv = (ph[i][j] + pl[i][j]) + comp[i][j];
          const float t = sum[i][j] + yv;
          comp[i][j] = yv - (t - sum[i][j]);
          sum[i][j] = t;
        }
    }
    __syncthreads();
  }
  float2* dst = reinterpret_cast<float2*>(part) + (long long)blockIdx.z * R * n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= R) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < n) dst[(long long)r * n + c] = make_float2(sum[i][j], comp[i][j]);
    }
  }
}

// Bout[r][c] = the KSPLIT partial (sum, compensation) pairs added as an unevaluated
// float pair (TwoSum of the sums, the compensations and the TwoSum errors gathered in
// a second float: FP64 arithmetic is slow on this part), rounded once.
__global__ void solve_reduce(const float* __restrict__ part, int R, int n, float* __restrict__ Bout, int ldb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * n) return;
  const long long stride = (long long)R * n;
  const float2* __restrict__ pp = reinterpret_cast<const float2*>(part);
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int k = 0; k < SV_KSPLIT; ++k) {
    const float2 v = pp[k * stride + e];
    const float t = __fadd_rn(hi, v.x);
    const float z = __fsub_rn(t, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(v.x, z)) + v.y;
    hi = t;
  }
  const int r = (int)(e / n), c = (int)(e % n);
  Bout[(long long)r * ldb + c] = hi + lo;
}

// y = A x, one warp per row.  Each lane keeps a Kahan-compensated FP32 sum of
// its strided products (FP64 arithmetic is slow on this part); the 32 lane sums
// are reduced in FP64.
__global__ void gemv_f32(const float* __restrict__ A, const float* __restrict__ x, float* __restrict__ y, int rows, int cols) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  float sum = 0.f, comp = 0.f;
  for (int c = lane; c < cols; c += 32) {
    const float a = A[(long long)row * cols + c], xv = x[c];
    const float p = __fmul_rn(a, xv);   // not fused into the sums below
    const float pe = fmaf(a, xv, -p);   // exact rounding error of the product
    const float yv = __fsub_rn(p, comp) + pe;
    const float t = sum + yv;
    comp = (t - sum) - yv;
    sum = t;
  }
  double acc = (double)sum - (double)comp;
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = (float)acc;
}

}  // namespace

int chol_inverse_f64(ce_ctx* ctx, double* A, int n, cudaStream_t s, double** inv_out) {
  CE_CUDA_TRY(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), s));
  // 1. Cholesky, lower, in place.
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = n - kb < NB ? n - kb : NB;
    potrf_diag<<<1, 256, 0, s>>>(A, n, kb, nb, ctx->dev_status);
    const int rest = n - kb - nb;
    if (rest > 0) {
      trsm_panel<<<(rest + 127) / 128, 128, 0, s>>>(A, n, kb, nb);
      dim3 g((rest + 63) / 64, (rest + 63) / 64);
      const double* P = A + (long long)(kb + nb) * n + kb;
      gemm64_sub<false, true, true><<<g, 256, 0, s>>>(P, n, P, n, A + (long long)(kb + nb) * n + kb + nb, n, rest, rest, nb);
    }
  }
  CE_CUDA_TRY(cudaGetLastError());
  int st = 0;
  CE_CUDA_TRY(cudaMemcpyAsync(&st, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  double* diag = (double*)dalloc(ctx, sizeof(double) * n);
  double* X = (double*)dalloc(ctx, sizeof(double) * (size_t)n * n);
  if (!diag || !X) { dfree(ctx, diag); dfree(ctx, X); return fail(ctx, CE_ERR_OOM, "inverse workspace"); }
  diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(A, n, diag);
  std::vector<double> hd(n);
  CE_CUDA_TRY(cudaMemcpyAsync(hd.data(), diag, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  if (st != 0) { dfree(ctx, diag); dfree(ctx, X); return fail(ctx, CE_ERR_NOT_SPD, "prediction matrix is not positive definite"); }
  double ld = 0;
  for (int i = 0; i < n; ++i) ld += 2.0 * std::log(hd[i]);
  if (!inv_out) ctx->logdet = ld;
  // 2. X = L^-1 (forward, right-looking over block rows), then X = L^-T X.
  identity_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(X, n);
  const unsigned cgrid = (n + 127) / 128;
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = n - kb < NB ? n - kb : NB;
    trsv_block<true><<<cgrid, 128, 0, s>>>(A, n, kb, nb, X, n, n);
    const int rest = n - kb - nb;
    if (rest > 0) {
      dim3 g((n + 63) / 64, (rest + 63) / 64);
      gemm64_sub<false, false, false><<<g, 256, 0, s>>>(A + (long long)(kb + nb) * n + kb, n, X + (long long)kb * n, n,
                                                        X + (long long)(kb + nb) * n, n, rest, n, nb);
    }
  }
  const int last = ((n - 1) / NB) * NB;
  for (int kb = last; kb >= 0; kb -= NB) {
    const int nb = n - kb < NB ? n - kb : NB;
    trsv_block<false><<<cgrid, 128, 0, s>>>(A, n, kb, nb, X, n, n);
    if (kb > 0) {
      // rows [0, kb) -= (L[kb..kb+nb, 0..kb])^T X[kb..kb+nb, :]
      dim3 g((n + 63) / 64, (kb + 63) / 64);
      gemm64_sub<true, false, false><<<g, 256, 0, s>>>(A + (long long)kb * n, n, X + (long long)kb * n, n, X, n, kb, n, nb);
    }
  }
  if (inv_out) {   // caller keeps the FP64 inverse
    CE_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(ctx, diag);
    *inv_out = X;
    return CE_OK;
  }
  // 3. FP32 pair.
  const int ldp = ctx->nobs_pad;
  dfree(ctx, ctx->Ainv_hi);
  dfree(ctx, ctx->Ainv_lo);
  dfree(ctx, ctx->ainv_blk);   // the tensor-core copy of the old inverse
  ctx->ainv_blk = nullptr;
  ctx->Ainv_hi = (float*)dalloc(ctx, sizeof(float) * (size_t)ldp * ldp);
  ctx->Ainv_lo = (float*)dalloc(ctx, sizeof(float) * (size_t)ldp * ldp);
  if (!ctx->Ainv_hi || !ctx->Ainv_lo) { dfree(ctx, diag); dfree(ctx, X); return fail(ctx, CE_ERR_OOM, "inverse"); }
  CE_CUDA_TRY(cudaMemsetAsync(ctx->Ainv_hi, 0, sizeof(float) * (size_t)ldp * ldp, s));
  CE_CUDA_TRY(cudaMemsetAsync(ctx->Ainv_lo, 0, sizeof(float) * (size_t)ldp * ldp, s));
  split_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(X, n, ctx->Ainv_hi, ctx->Ainv_lo, ldp);
  CE_CUDA_TRY(cudaGetLastError());
  CE_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, diag);
  dfree(ctx, X);
  return CE_OK;
}

void gemm64_nn_sub(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N, int K,
                   cudaStream_t s) {
  dim3 g((N + 63) / 64, (M + 63) / 64);
  gemm64_sub<false, false, false><<<g, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K);
}

void launch_solve(ce_ctx* ctx, const float* E, int R, float* B, int ldb, cudaStream_t s) {
  const int n = ctx->nobs;
  dim3 g((n + SV_TC - 1) / SV_TC, (R + SV_TR - 1) / SV_TR, SV_KSPLIT);
  // the FP32 form keeps pairs (the tightest error); the tensor forms, whose correction
  // error dominates, sum four hi products per compensated step (a quarter faster)
  if (ctx->prec == CE_PREC_FP32 || ctx->prec == CE_PREC_FP64)
    solve_gemm_f32<2><<<g, 128, 0, s>>>(E, R, n, ctx->Ainv_hi, ctx->Ainv_lo, ctx->nobs_pad, ctx->Bpart);
  else
    solve_gemm_f32<4><<<g, 128, 0, s>>>(E, R, n, ctx->Ainv_hi, ctx->Ainv_lo, ctx->nobs_pad, ctx->Bpart);
  const long long tot = (long long)R * n;
  solve_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->Bpart, R, n, B, ldb);
}

void launch_gemm_hilo(const float* E, int R, int n, const float* hi, const float* lo, int lda, float* part, float* out,
                      int ldo, cudaStream_t s, bool compensated) {
  dim3 g((n + SV_TC - 1) / SV_TC, (R + SV_TR - 1) / SV_TR, SV_KSPLIT);
  if (compensated) solve_gemm_f32<2><<<g, 128, 0, s>>>(E, R, n, hi, lo, lda, part);
  else solve_gemm_f32<0><<<g, 128, 0, s>>>(E, R, n, hi, lo, lda, part);
  const long long tot = (long long)R * n;
  solve_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, R, n, out, ldo);
}

void launch_gemv_f32(const float* Amat, const float* x, float* y, int rows, int cols, cudaStream_t s) {
  gemv_f32<<<(rows + 7) / 8, 256, 0, s>>>(Amat, x, y, rows, cols);
}

}  // namespace ce
