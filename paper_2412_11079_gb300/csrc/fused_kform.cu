// Instantiations of the fused pass for the kernel form diag(U) K diag(V) with a
// read-only K (FP32/BF16/FP16).
#include "fused_kernel.cuh"

namespace uot {
const FusedEntry kKformTable[kFusedConfigs] = UOT_FUSED_TABLE(true);
}  // namespace uot
