// tcgen05 implicit-GEMM 3x3 convolution (placeholder until the kernel lands).
#include "net_internal.h"

namespace ppe {
bool conv3x3_tc_supported(const ConvArgs &) { return false; }
ppe_status conv3x3_tc(const ConvArgs &, cudaStream_t) { return PPE_ERR_ARG; }
}  // namespace ppe
