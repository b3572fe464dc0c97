// Tensor-core form of the Kriging correction (placeholder until the tcgen05 kernel lands).
#include "ce_common.cuh"
#include "ce_internal.h"

namespace ce {
int launch_correct_tc(ce_ctx* ctx, const float*, int, float*, cudaStream_t) {
  return fail(ctx, CE_ERR_ARG, "tensor-core correction not available in this build");
}
}  // namespace ce
