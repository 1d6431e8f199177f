// Kernels of the fused net pipeline and of its persistent schedule in one precision:
// FP32 without refinement.
#include "qk_fused.cuh"

namespace qk {
QK_FUSED_INSTANTIATE(float, false, false)
}  // namespace qk
