// Gaussian log-likelihood of the data under the model of Eq. (condmvn):
// z ~ N(0, A) with A = K_oo + tau^2 I, so
//   l = -z^T A^-1 z / 2 - log det A / 2 - (n / 2) log(2 pi).
// The context holds A^-1 as an FP32 pair (hi + lo, internal site order) and
// log det A from the FP64 Cholesky factor of its set-up; the quadratic form is
// summed here in FP64, one warp per row of A^-1.
#include <cmath>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

// out += sum_q z[q] sum_j (hi[q][j] + lo[q][j]) z[j]; the pair is symmetric, rows of stride ld.
__global__ void __launch_bounds__(256) quad_form_kernel(const float* __restrict__ hi, const float* __restrict__ lo, int ld,
                                                        const float* __restrict__ z, int n, double* __restrict__ out) {
  const int row = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* __restrict__ h = hi + (size_t)row * ld;
  const float* __restrict__ l = lo + (size_t)row * ld;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma((double)h[j] + (double)l[j], (double)z[j], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomicAdd(out, s * (double)z[row]);
}

}  // namespace
}  // namespace ce

using namespace ce;

extern "C" int ce_loglik(ce_ctx* ctx, const float* z_dev, double* out, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!z_dev || !out) return fail(ctx, CE_ERR_ARG, "null pointer");
  if (ctx->mode != CE_LOCAL) {
    return fail(ctx, CE_ERR_STATE, "the data log-likelihood needs the local-Kriging set-up (ce_krige_weights, CE_LOCAL)");
  }
  if (ctx->trend_p > 0) return fail(ctx, CE_ERR_STATE, "the log-likelihood is of the zero-mean model (ce_set_trend -1 first)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = ctx->nobs;
  // z in the internal order of A^-1, then the FP64 sum, in one small buffer of the call
  void* buf = dalloc(ctx, sizeof(double) + sizeof(float) * (size_t)n);
  if (!buf) return fail(ctx, CE_ERR_OOM, "log-likelihood buffer");
  double* acc = static_cast<double*>(buf);
  float* zq = reinterpret_cast<float*>(acc + 1);
  int st = CE_OK;
  double q = 0.0;
  do {
    if (cudaMemsetAsync(acc, 0, sizeof(double), s) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); break; }
    launch_permute_rows(z_dev, zq, ctx->perm, 1, n, n, n, false, s);
    const unsigned blocks = (unsigned)(((long long)n * 32 + 255) / 256);
    quad_form_kernel<<<blocks, 256, 0, s>>>(ctx->Ainv_hi, ctx->Ainv_lo, ctx->nobs_pad, zq, n, acc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&q, acc, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "log-likelihood", __FILE__, __LINE__);
  } while (false);
  dfree(ctx, buf);
  if (st) return st;
  *out = -0.5 * q - 0.5 * ctx->logdet - 0.5 * (double)n * std::log(2.0 * M_PI);
  return CE_OK;
}
