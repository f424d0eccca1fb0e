// Instantiations of the fused pass for plans stored in place (FP32/BF16/FP16).
#include "fused_kernel.cuh"

namespace uot {
const FusedEntry kInplaceTable[kFusedConfigs] = UOT_FUSED_TABLE(false);
}  // namespace uot
