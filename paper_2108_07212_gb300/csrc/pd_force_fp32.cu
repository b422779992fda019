// pd_force_fp32.cu -- FP32-split force kernel (placeholder until written).
#include "pd_device.cuh"

namespace pd {

cudaError_t launch_force_fp32(const DevPtrs &, const KParams &, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace pd
