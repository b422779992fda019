// pd_step64.cu -- FP64 force kernels (multi-kernel and persistent paths),
// compiled without FMA contraction so every FP64 expression rounds as written.
#include <algorithm>

#include "pd_step.cuh"

namespace pd {

cudaError_t launch_force64(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase) {
    return launch_force_impl<false>(d, k, vin, update_v, s, phase);
}

cudaError_t launch_persistent64(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s) {
    return launch_persistent_impl<false>(d, k, vin, nsteps, block, s);
}

}  // namespace pd
