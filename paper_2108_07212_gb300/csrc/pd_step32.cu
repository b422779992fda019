// pd_step32.cu -- FP32-split force kernels (multi-kernel and persistent paths).
#include <algorithm>

#include "pd_step.cuh"

namespace pd {

cudaError_t launch_force32(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase) {
    return launch_force_impl<true>(d, k, vin, update_v, s, phase);
}

cudaError_t launch_persistent32(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s) {
    return launch_persistent_impl<true>(d, k, vin, nsteps, block, s);
}

}  // namespace pd
