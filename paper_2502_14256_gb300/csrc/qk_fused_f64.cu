// Kernels of the fused net pipeline and of its persistent schedule in one precision:
// FP64.
#include "qk_fused.cuh"

namespace qk {
QK_FUSED_INSTANTIATE(double, false, false)
}  // namespace qk
