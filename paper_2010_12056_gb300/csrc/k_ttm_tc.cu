// Tensor-core first-level TTM (tcgen05 + TMA).  Placeholder until the kernel lands:
// reports "unsupported" so the driver uses the FP32 SIMT path.
#include "cpals_internal.h"

namespace cpk {
bool ttm_tc_supported(int64_t, int, int64_t, int) { return false; }
cudaError_t ttm_tc(const float*, const TcOperand&, float*, int64_t, int, int64_t, int, int, int,
                   unsigned*, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace cpk
