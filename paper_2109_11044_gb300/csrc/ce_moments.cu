// Ensemble moments of conditional draws at every grid node: the per-node sum and
// sum of squares over realizations (FP64), accumulated over calls, and the mean
// and standard-deviation maps they give (the ensemble mean estimate and its
// standard error, as the paper's application reports them, Section 4).  Sums
// from several calls or ranks add.
#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

// sum[g] (+)= sum_r v[r][g], sumsq[g] (+)= sum_r v[r][g]^2; one thread per node.
// Within a call the sums run in FP32 with Kahan compensation (and the exact
// rounding error of every square kept aside), which FP64 would make several
// times slower on this part; the per-node totals join the FP64 buffers once.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

__global__ void moments_kernel(const float* __restrict__ v, int R, long long M, double* __restrict__ sum,
                               double* __restrict__ sumsq, int accumulate) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M) return;
  float s = 0.f, cs = 0.f, q = 0.f, cq = 0.f, qe = 0.f;
  int r = 0;
  for (; r + 8 <= R; r += 8) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = __ldcs(v + (long long)(r + u) * M + g);   // loads in flight together
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float p = __fmul_rn(x[u], x[u]);
      qe += fmaf(x[u], x[u], -p);   // exact rounding error of the square
      kahan_add(s, cs, x[u]);
      kahan_add(q, cq, p);
    }
  }
  for (; r < R; ++r) {
    const float x = __ldcs(v + (long long)r * M + g);
    const float p = __fmul_rn(x, x);
    qe += fmaf(x, x, -p);
    kahan_add(s, cs, x);
    kahan_add(q, cq, p);
  }
  const double ss = (double)s - (double)cs, qq = ((double)q - (double)cq) + (double)qe;
  sum[g] = accumulate ? sum[g] + ss : ss;
  sumsq[g] = accumulate ? sumsq[g] + qq : qq;
}

// mean = sum / N, sd = sqrt((sumsq - N mean^2) / (N - 1)) (0 for N = 1).
__global__ void stats_kernel(const double* __restrict__ sum, const double* __restrict__ sumsq, long long M, double count,
                             float* __restrict__ mean, float* __restrict__ sd) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= M) return;
  const double mu = sum[g] / count;
  if (mean) mean[g] = (float)mu;
  if (sd) sd[g] = count > 1.0 ? (float)sqrt(fmax(sumsq[g] - count * mu * mu, 0.0) / (count - 1.0)) : 0.f;
}

}  // namespace
}  // namespace ce

using namespace ce;

extern "C" int ce_ensemble_moments(ce_ctx* ctx, const float* v_dev, int R, double* sum_dev, double* sumsq_dev,
                                   int accumulate, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!v_dev || !sum_dev || !sumsq_dev) return fail(ctx, CE_ERR_ARG, "null buffer");
  if (R < 1) return fail(ctx, CE_ERR_ARG, "R must be at least 1");
  const long long M = (long long)ctx->m * ctx->m;
  moments_kernel<<<(unsigned)((M + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      v_dev, R, M, sum_dev, sumsq_dev, accumulate ? 1 : 0);
  ctx->launches += 1;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}

extern "C" int ce_ensemble_stats(ce_ctx* ctx, const double* sum_dev, const double* sumsq_dev, double count,
                                 float* mean_dev, float* sd_dev, void* stream) {
  if (!ctx) return fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (!sum_dev || !sumsq_dev) return fail(ctx, CE_ERR_ARG, "null buffer");
  if (!(count >= 1.0)) return fail(ctx, CE_ERR_ARG, "count must be at least 1");
  const long long M = (long long)ctx->m * ctx->m;
  stats_kernel<<<(unsigned)((M + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(sum_dev, sumsq_dev, M, count,
                                                                                               mean_dev, sd_dev);
  ctx->launches += 1;
  CE_CUDA_TRY(cudaGetLastError());
  return CE_OK;
}
