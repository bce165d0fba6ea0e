// Mixed-precision form: BF16 shadow copy of the tensor, tcgen05 bulk sweeps,
// FP32 finishing sweeps. (Filled in by the tensor-core path.)
#include "internal.h"

namespace tals {

tals_status mixed_alloc(tals_ctx* c) {
  (void)c;
  return fail(TALS_ENOTSUP, "mixed BF16 precision is not available in this build");
}

void mixed_free(tals_ctx* c) { (void)c; }

tals_status run_mode_mixed(tals_ctx* c, ModeJob& j, bool set_norm_a) {
  (void)c; (void)j; (void)set_norm_a;
  return fail(TALS_ENOTSUP, "mixed BF16 precision is not available in this build");
}

}  // namespace tals
