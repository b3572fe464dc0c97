// Special-function and FP32 FMA throughput of this GPU, for the rooflines of the
// Kriging correction and of the FP32 products (measurement support; the paper has
// no counterpart).
//
// Each evaluation of the closed-form Matern covariance in the correction takes
// one square root and one base-2 exponential on the special-function units, plus
// a few FP32 operations.  Three chain kernels time ex2 alone, sqrt alone, and the
// pair as the correction issues it (ex2(-sqrt(d2)) with d2 formed by an FMA), each
// over 8 independent chains per thread on every SM; a fourth times chains of FP32
// fused multiply-adds.
#include <cuda_runtime.h>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int kChains = 8, kIters = 2048;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// op 0: v <- -ex2(v) / 2 (stays in [-1/2, -1/4)); op 1: v <- sqrt(v) + 1/4 (stays
// positive); op 2: v <- ex2(-sqrt(d2)) with d2 = v^2 + 1/4; op 3: v <- 0.999 v + 1e-4
// (four FMAs per chain and step).  out: one float per thread.
template <int OP>
__global__ void __launch_bounds__(256) unit_chain_kernel(float* __restrict__ out, float seed) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = seed + 1e-3f * (float)(threadIdx.x + j);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      if (OP == 0) {
        v[j] = -0.5f * ex2_approx(v[j]);
      } else if (OP == 1) {
        v[j] = sqrt_approx(v[j]) + 0.25f;
      } else if (OP == 3) {
#pragma unroll
        for (int t = 0; t < 4; ++t) v[j] = fmaf(v[j], 0.999f, 1e-4f);
      } else {
        const float d2 = fmaf(v[j], v[j], 0.25f);
        v[j] = ex2_approx(-sqrt_approx(d2));
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
int time_chain(float* out, int blocks, cudaStream_t s, double* ops_per_s) {
  cudaEvent_t a, b;
  CE_CUDA_TRY(cudaEventCreate(&a));
  CE_CUDA_TRY(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
    CE_CUDA_TRY(cudaEventRecord(a, s));
    unit_chain_kernel<OP><<<blocks, 256, 0, s>>>(out, 0.5f);
    CE_CUDA_TRY(cudaEventRecord(b, s));
    CE_CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    CE_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ops_per_s = (double)blocks * 256 * kIters * kChains * (OP == 3 ? 4 : 1) / (best * 1e-3);
  return CE_OK;
}

}  // namespace
}  // namespace ce

using namespace ce;

extern "C" int ce_unit_rates(double* ex2_per_s, double* sqrt_per_s, double* matern_evals_per_s, double* fma_per_s,
                             void* stream) {
  if (!ex2_per_s || !sqrt_per_s || !matern_evals_per_s || !fma_per_s) return fail(nullptr, CE_ERR_ARG, "null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  CE_CUDA_TRY(cudaGetDevice(&dev));
  CE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8;
  float* out = nullptr;
  CE_CUDA_TRY(cudaMalloc(&out, sizeof(float) * (size_t)blocks * 256));
  int st = time_chain<0>(out, blocks, s, ex2_per_s);
  if (!st) st = time_chain<1>(out, blocks, s, sqrt_per_s);
  if (!st) st = time_chain<2>(out, blocks, s, matern_evals_per_s);
  if (!st) st = time_chain<3>(out, blocks, s, fma_per_s);
  cudaFree(out);
  return st;
}
