// Kernels of the fused net pipeline and of its persistent schedule in one precision:
// FP32 with the compensated refinement.
#include "qk_fused.cuh"

namespace qk {
QK_FUSED_INSTANTIATE(float, true, false)
}  // namespace qk
