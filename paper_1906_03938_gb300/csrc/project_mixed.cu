// Mixed-precision fused assembly + projection (FP32 evaluation, BF16x3 tcgen05 contraction).
#include "internal.h"

namespace bem {

bem_status project_mixed(bem_ctx* ctx, const double*, int64_t, int, double*, double*,
                         cudaStream_t) {
  return fail(ctx, BEM_EINVAL, "bem_project: mixed precision path not available in this build");
}

}  // namespace bem
