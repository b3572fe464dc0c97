// Allocation-free entry point for the unconditional ensemble.
//
// Some callers cannot allocate device memory when they call in: a host
// application that hands its whole GPU memory budget to its own pool before
// the work starts, or a latency-critical loop in which cudaMalloc and cudaFree
// would synchronise the device and stall the other streams.  For them,
// ce_unconditional_static runs the same row and column FFT passes as
// ce_unconditional, with the per-pair intermediate held in a fixed buffer that
// is part of this library's device image instead of a buffer allocated on
// first use.
//
// The buffer is a file-scope device array of CE_STATIC_SCRATCH_BYTES.  Every
// GPU that loads the library holds it until the process exits.  All calls on a
// device share it and it keeps whatever the last call left there; nothing in
// it needs clearing, because the row pass writes every element that the
// column pass then reads.  Two calls whose work overlaps on the GPU (for
// example on two streams) race on the buffer: order them on one stream or
// synchronise between them.
#include <cuda_runtime.h>

#include <mutex>

#include "ce_common.cuh"
#include "ce_internal.h"

namespace {

constexpr size_t kScratchBytes = CE_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char ce_static_scratch[kScratchBytes];

// Device address of ce_static_scratch, looked up once per device with that
// device current.  In host code the array's name is only a host-side handle.
std::mutex g_lock;
void* g_scratch[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = -1;
  CE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return ce::fail(nullptr, CE_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, ce_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return ce::cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(ce_static_scratch)",
                           __FILE__, __LINE__);
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return CE_OK;
}

}  // namespace

namespace ce {
// Looks up the scratch array's address for the current device ahead of the
// first call (ce_setup does this): with lazy module loading the lookup is what
// loads this file's module and places the array, so doing it here keeps that
// allocation out of ce_unconditional_static itself.
int static_scratch_resolve() {
  void* p = nullptr;
  return scratch_address(&p);
}
}  // namespace ce

extern "C" int ce_unconditional_static(ce_ctx* ctx, int R, uint64_t seed, uint64_t r_offset, float* y_dev, void* stream) {
  if (!ctx) return ce::fail(nullptr, CE_ERR_ARG, "null context");
  ctx->err.clear();
  if (R < 1 || R > 4096) return ce::fail(ctx, CE_ERR_ARG, "R must be in [1, 4096]");
  if (r_offset % 2) return ce::fail(ctx, CE_ERR_ARG, "r_offset must be even");
  if (!y_dev) return ce::fail(ctx, CE_ERR_ARG, "null output");
  if (!ctx->sqrt_lam) return ce::fail(ctx, CE_ERR_STATE, "the context has no embedding");
  const size_t per_pair = sizeof(float2) * (size_t)ctx->P * ctx->m;
  if (per_pair > kScratchBytes)
    return ce::fail(ctx, CE_ERR_ARG,
                    "ce_unconditional_static: one realization pair needs " + std::to_string(per_pair) +
                        " bytes of scratch (P x m complex floats) but the fixed buffer holds " +
                        std::to_string(kScratchBytes) + "; use ce_unconditional for this grid");
  void* scratch = nullptr;
  const int st = scratch_address(&scratch);
  if (st != CE_OK) return ce::fail(ctx, st, ce_last_error(nullptr));
  return ce::fft_unconditional_into(ctx, R, seed, r_offset, y_dev, reinterpret_cast<cudaStream_t>(stream), scratch,
                                    kScratchBytes);
}
