// pd_persist.cu -- the persistent step kernels of one precision and one thread
// count per node, for blocks of 128 and 256 threads.  Compiled once per pair,
// with PD_PERSIST_FP32 (1: FP32 split, 0: FP64) and PD_PERSIST_LANES defined,
// and with the compile flags of that precision's other kernels.
#include <algorithm>

#include "pd_step.cuh"

#if !defined(PD_PERSIST_FP32) || !defined(PD_PERSIST_LANES)
#error "PD_PERSIST_FP32 and PD_PERSIST_LANES must be defined"
#endif

namespace pd {

template <bool FP32, int LANES>
cudaError_t launch_persistent_lanes(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block,
                                    cudaStream_t s) {
    if (block == 256) return launch_persistent_cfg<FP32, LANES, 256>(d, k, vin, nsteps, s);
    return launch_persistent_cfg<FP32, LANES, 128>(d, k, vin, nsteps, s);
}

template cudaError_t launch_persistent_lanes<PD_PERSIST_FP32 != 0, PD_PERSIST_LANES>(const DevPtrs &, const KParams &,
                                                                                     int, int, int, cudaStream_t);

}  // namespace pd
