// Kernels of the fused net pipeline and of its persistent schedule in one precision:
// FP32 with the float-float first column (QK_F32W).
#include "qk_fused.cuh"

namespace qk {
QK_FUSED_INSTANTIATE(float, true, true)
}  // namespace qk
