// Tensor-core path (filled in below).
#include "common.cuh"

namespace pm {
pm_status launch_batched_tensor(int64_t, const uint32_t*, const int64_t*, const uint32_t*,
                                const int64_t*, uint32_t*, const int64_t*, uint32_t, int64_t,
                                cudaStream_t, DeviceWorkspace*) {
    return PM_ERR_UNSUPPORTED;
}
}  // namespace pm
