// Split-bf16 tcgen05 DST (mixed path).  Not enabled yet: dst_tc_supported() is false, so the
// mixed path runs its DST on the float32 SIMT kernel.
#include "internal.h"

namespace lag {

bool dst_tc_supported(int) { return false; }
size_t dst_tc_bytes(int) { return 0; }
void dst_build_tc(DstPlan &, DevBuf &, size_t, cudaStream_t) {}
void dst_apply_tc_d2f(const DstPlan &, const double *, float *, int, int, const KrylovScalars *, cudaStream_t) {
  throw Error(LAG_EINVAL, "tensor-core DST not available");
}
void dst_apply_tc_f2d(const DstPlan &, const float *, double *, int, int, const KrylovScalars *, cudaStream_t) {
  throw Error(LAG_EINVAL, "tensor-core DST not available");
}

}  // namespace lag
