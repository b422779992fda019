// pd_step.cuh -- force kernels of the multi-kernel path and the persistent
// step kernel, instantiated per precision by pd_step64.cu (no FMA
// contraction) and pd_step32.cu.
#pragma once

#include <type_traits>

#include "pd_device.cuh"

namespace pd {

// Forces and update of nodes [node0, node0 + BLOCK / LANES): LANES threads per
// node compute the lane-summed bond / self-contact / contact parts, which meet
// in shared memory; then one thread per node adds the wall forces and
// integrates (FP64, converged warps).  Every thread of the block must call it.
template <bool FP32, bool PERSIST, int LANES, int BLOCK>
__device__ __forceinline__ void force_block(const DevPtrs &d, const KParams &k, int node0, int vin, int update_v) {
    constexpr int NB = BLOCK / LANES;
    using Sums = typename std::conditional<FP32, Sums32, Sums64>::type;
    __shared__ Sums sm[NB];
    const int local = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    const int i = node0 + local;
    Sums f;
    if constexpr (FP32) force_node32<PERSIST, LANES>(d, k, i, lane, i < k.N, vin, f);
    else force_node64<PERSIST, LANES>(d, k, i, lane, i < k.N, vin, f);
    if (lane == 0) sm[local] = f;
    __syncthreads();
    if ((int)threadIdx.x < NB && node0 + (int)threadIdx.x < k.N) {
        if constexpr (FP32) node_epilogue32<PERSIST>(d, k, node0 + threadIdx.x, vin, update_v, sm[threadIdx.x]);
        else node_epilogue64<PERSIST>(d, k, node0 + threadIdx.x, vin, update_v, sm[threadIdx.x]);
    }
    __syncthreads();
}

// The force phase reads the candidate lists of this step: it clears the
// rebuild flag for the next one.
__device__ __forceinline__ void clear_rebuild(const DevPtrs &d) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *d.rebuild = 0;
}

// Multi-kernel path: one block per BLOCK / LANES nodes.
template <bool FP32, int LANES>
__global__ void __launch_bounds__(kBlock, FP32 ? (LANES == 1 ? 8 : 5) : 4) k_force(DevPtrs d, KParams k, int vin, int update_v) {
    clear_rebuild(d);
    force_block<FP32, false, LANES, kBlock>(d, k, blockIdx.x * (kBlock / LANES), vin, update_v);
}

// Split variant: the lane sums of node i go to global memory (structure of
// arrays, six components) and a second pass adds walls and integrates.
template <bool FP32, bool PERSIST, int LANES>
__device__ __forceinline__ void sums_node(const DevPtrs &d, const KParams &k, int i, int lane, int vin) {
    const bool active = i < k.N;
    const size_t N = (size_t)k.N;
    if constexpr (FP32) {
        Sums32 f;
        force_node32<PERSIST, LANES>(d, k, i, lane, active, vin, f);
        if (active && lane == 0) {
            float *o = static_cast<float *>(d.fsum);
            if (k.store) {
                o[i] = f.bx, o[N + i] = f.by, o[2 * N + i] = f.sx, o[3 * N + i] = f.sy, o[4 * N + i] = f.nx,
                o[5 * N + i] = f.ny;
            } else {
                // only the total is needed: (F_b + F_s) + F_n, as the epilogue would form it
                reinterpret_cast<float2 *>(o)[i] = make_float2((f.bx + f.sx) + f.nx, (f.by + f.sy) + f.ny);
            }
        }
    } else {
        Sums64 f;
        force_node64<PERSIST, LANES>(d, k, i, lane, active, vin, f);
        if (active && lane == 0) {
            double *o = static_cast<double *>(d.fsum);
            if (k.store) {
                o[i] = f.bx, o[N + i] = f.by, o[2 * N + i] = f.sx, o[3 * N + i] = f.sy, o[4 * N + i] = f.nx,
                o[5 * N + i] = f.ny;
            } else {
                reinterpret_cast<double2 *>(o)[i] =
                    make_double2(__dadd_rn(__dadd_rn(f.bx, f.sx), f.nx), __dadd_rn(__dadd_rn(f.by, f.sy), f.ny));
            }
        }
    }
}

template <bool FP32, bool PERSIST>
__device__ __forceinline__ void epilogue_node(const DevPtrs &d, const KParams &k, int i, int vin, int update_v) {
    const size_t N = (size_t)k.N;
    // per-part sums (k.store) or the total of the parts
    if constexpr (FP32) {
        const float *o = static_cast<const float *>(d.fsum);
        if (k.store) {
            const Sums32 f{ldm<PERSIST>(o + i), ldm<PERSIST>(o + N + i), ldm<PERSIST>(o + 2 * N + i),
                           ldm<PERSIST>(o + 3 * N + i), ldm<PERSIST>(o + 4 * N + i), ldm<PERSIST>(o + 5 * N + i)};
            node_epilogue32<PERSIST>(d, k, i, vin, update_v, f);
        } else {
            const float2 t = ldm<PERSIST>(reinterpret_cast<const float2 *>(o) + i);
            node_epilogue32<PERSIST>(d, k, i, vin, update_v, Sums32{t.x, t.y, 0.f, 0.f, 0.f, 0.f}, true);
        }
    } else {
        const double *o = static_cast<const double *>(d.fsum);
        if (k.store) {
            const Sums64 f{ldm<PERSIST>(o + i), ldm<PERSIST>(o + N + i), ldm<PERSIST>(o + 2 * N + i),
                           ldm<PERSIST>(o + 3 * N + i), ldm<PERSIST>(o + 4 * N + i), ldm<PERSIST>(o + 5 * N + i)};
            node_epilogue64<PERSIST>(d, k, i, vin, update_v, f);
        } else {
            const double2 t = ldm<PERSIST>(reinterpret_cast<const double2 *>(o) + i);
            node_epilogue64<PERSIST>(d, k, i, vin, update_v, Sums64{t.x, t.y, 0.0, 0.0, 0.0, 0.0}, true);
        }
    }
}

template <bool FP32, int LANES>
__global__ void __launch_bounds__(kBlock, FP32 ? 8 : 4) k_sums(DevPtrs d, KParams k, int vin) {
    clear_rebuild(d);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    sums_node<FP32, false, LANES>(d, k, tid / LANES, tid % LANES, vin);
}

template <bool FP32>
__global__ void __launch_bounds__(256, 6) k_epilogue(DevPtrs d, KParams k, int vin, int update_v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k.N) epilogue_node<FP32, false>(d, k, i, vin, update_v);
}

// phase (split force phase only): 0 both passes, 1 the lane sums, 2 the epilogue.
template <bool FP32>
cudaError_t launch_force_impl(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase) {
    const long long threads = (long long)k.lanes * k.N;
    const unsigned grid = (unsigned)((threads + kBlock - 1) / kBlock);
    if (k.split) {
        if (phase != 2) {
            if (k.lanes == 8) k_sums<FP32, 8><<<grid, kBlock, 0, s>>>(d, k, vin);
            else if (k.lanes == 4) k_sums<FP32, 4><<<grid, kBlock, 0, s>>>(d, k, vin);
            else if (k.lanes == 2) k_sums<FP32, 2><<<grid, kBlock, 0, s>>>(d, k, vin);
            else k_sums<FP32, 1><<<grid, kBlock, 0, s>>>(d, k, vin);
        }
        if (phase != 1) k_epilogue<FP32><<<(unsigned)((k.N + 255) / 256), 256, 0, s>>>(d, k, vin, update_v);
        return cudaGetLastError();
    }
    if (phase != 0) return cudaErrorInvalidValue;
    if (k.lanes == 8) k_force<FP32, 8><<<grid, kBlock, 0, s>>>(d, k, vin, update_v);
    else if (k.lanes == 4) k_force<FP32, 4><<<grid, kBlock, 0, s>>>(d, k, vin, update_v);
    else if (k.lanes == 2) k_force<FP32, 2><<<grid, kBlock, 0, s>>>(d, k, vin, update_v);
    else k_force<FP32, 1><<<grid, kBlock, 0, s>>>(d, k, vin, update_v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// persistent step kernel

// Grid barrier with a bounded wait: the last block to arrive resets the
// arrival count and advances the generation; the others sleep-poll the
// generation for at most max_spins rounds (kBarrierSpins unless a test
// shortens it), then set status[PD_STATUS_TIMEOUT] and report failure (the
// kernel then returns, so the device never hangs).  Co-residency of all blocks
// is guaranteed by the cooperative launch.
__device__ __forceinline__ bool grid_barrier(const DevPtrs &d, long long max_spins) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = d.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(d.bar, 1u);
        ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(d.bar, 0u);
            __threadfence();
            atomicAdd(d.bar + 1, 1u);
        } else {
            long long n = 0;
            while (*gen == g) {
                if (++n > max_spins || *(volatile int *)&d.status[PD_STATUS_TIMEOUT]) {
                    atomicExch(&d.status[PD_STATUS_TIMEOUT], 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <int BLOCK>
__device__ __forceinline__ int block_sum(int v, int *sm) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = (lane < BLOCK / 32) ? sm[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) sm[32] = t;
    }
    __syncthreads();
    return sm[32];
}

// Exclusive scan of one value per thread over the block; returns the total.
template <int BLOCK>
__device__ __forceinline__ int block_scan1(int &v, int *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    __syncthreads();
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = (lane < BLOCK / 32) ? sm[lane] : 0;
        int wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        sm[lane] = wi - w;
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    v = sm[warp] + incl - v;
    return sm[32];
}

// One time step of the persistent kernel, all phases:
//   A  displacement update, positions, rebuild test       (Algorithm 1)
//      (FP32 split: taken by the previous step's velocity update instead,
//      except in the first step of a launch that finds no valid prediction)
//   when some node moved kSkinTrigger * skin since the last rebuild:
//     R1 bucket counts
//     R2 per-block sums of the bucket counts
//     R3 exclusive scan of the counts -> cell starts (counts cleared)
//     R4 counting-sort scatter of the node indices
//     R5 candidate lists
//   E  forces, acceleration and velocity update
// s_cur_u / s_cur_pq hold this step's current displacement and positions
// (parity vin ^ 1).  Bucket counts are zero on entry and on exit.  False when a
// grid barrier gave up (the kernel then returns).
template <bool FP32, int LANES, int BLOCK>
__device__ __forceinline__ bool persistent_step(const DevPtrs &d, const KParams &k, int vin, int st, int nsteps,
                                                bool predicted, int *sm, long long &s_step) {
    const int nthreads = gridDim.x * BLOCK;
    const int gtid = blockIdx.x * BLOCK + threadIdx.x;
    const unsigned T = k.T;
    const unsigned slice = (T + gridDim.x - 1) / gridDim.x;
    const unsigned lo = min(T, blockIdx.x * slice), hi = min(T, lo + slice);
    // A (the step counter's load is issued first, so that its latency
    // overlaps the displacement update of block 0's nodes)
    const long long s = (blockIdx.x == 0 && threadIdx.x == 0) ? __ldcg(d.step) + 1 : 0;
    if (st == 0) prefetch_force_inputs(d, k, gtid, nthreads);
    if (!predicted) {
        bool need = false;
        for (int i = gtid; i < k.N; i += nthreads) need |= predict_node<true>(d, k, i, vin, 1);
        if (__any_sync(0xffffffffu, need) && (threadIdx.x & 31) == 0) *(volatile int *)d.rebuild = 1;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            *d.step = s;
            *d.t_now = (double)s * k.dt;
            s_step = s;
            if constexpr (FP32) {
                // the previous velocity update's rebuild test becomes this step's
                // flag (no block reads the flag before the barrier below)
                if (predicted && *(volatile int *)d.rebuild_next) *(volatile int *)d.rebuild = 1;
                *(volatile int *)d.rebuild_next = 0;
            }
        }
        __syncthreads();
        wall_cells(d, k, (double)s_step * k.dt);
    }
    if (!grid_barrier(d, k.bar_spins)) return false;
    if (__ldcg(d.rebuild)) {
        // R1
        for (int i = gtid; i < k.N; i += nthreads) bin_node<true>(d, k, i);
        if (!grid_barrier(d, k.bar_spins)) return false;
        // R2
        int part = 0;
        for (unsigned b = lo + threadIdx.x; b < hi; b += BLOCK) part += __ldcg(&d.count[b]);
        part = block_sum<BLOCK>(part, sm);
        if (threadIdx.x == 0) d.blocksums[blockIdx.x] = part;
        if (!grid_barrier(d, k.bar_spins)) return false;
        // R3
        int off = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += BLOCK) off += __ldcg(&d.blocksums[b]);
        off = block_sum<BLOCK>(off, sm);
        for (unsigned b0 = lo; b0 < hi; b0 += BLOCK) {
            const unsigned b = b0 + threadIdx.x;
            int c = (b < hi) ? __ldcg(&d.count[b]) : 0;
            if (b < hi) d.count[b] = 0;
            const int tot = block_scan1<BLOCK>(c, sm);
            if (b < hi) {
                d.start[b] = off + c;
                d.cursor[b] = off + c;
            }
            off += tot;
        }
        if (gtid == 0) d.start[T] = k.N;
        if (!grid_barrier(d, k.bar_spins)) return false;
        // R4
        for (int i = gtid; i < k.N; i += nthreads) scatter_node<true>(d, k, i);
        if (!grid_barrier(d, k.bar_spins)) return false;
        // R5 (every block has read the flag: clear it for the next step)
        if (gtid == 0) {
            *d.rebuild = 0;
            atomicAdd(&d.status[PD_STATUS_REBUILDS], 1);
        }
        for (int i = gtid; i < k.N; i += nthreads) build_list_node<true>(d, k, i);
        if (!grid_barrier(d, k.bar_spins)) return false;
    }
    // E
    if (k.split) {
        const long long total = (((long long)LANES * k.N + 31) / 32) * 32;
        for (long long t = gtid; t < total; t += nthreads) sums_node<FP32, true, LANES>(d, k, (int)(t / LANES), (int)(t % LANES), vin);
        if (!grid_barrier(d, k.bar_spins)) return false;
        for (int i = gtid; i < k.N; i += nthreads) epilogue_node<FP32, true>(d, k, i, vin, 1);
    } else {
        for (int node0 = blockIdx.x * (BLOCK / LANES); node0 < k.N; node0 += gridDim.x * (BLOCK / LANES))
            force_block<FP32, true, LANES, BLOCK>(d, k, node0, vin, 1);
    }
    // the end of the launch orders the last step before whatever follows
    return st + 1 >= nsteps || grid_barrier(d, k.bar_spins);
}

// nsteps time steps in one cooperative launch, phases separated by bounded
// grid barriers.  Every step reads its current displacement and positions
// through s_cur_u / s_cur_pq, the buffers of its parity (the FP32 split keeps
// two of each; the FP64 path one).
// (FP32 split, one thread per node: capped at 64 registers, eight blocks of 128
// per SM, as the lane-sum kernel of the graph path; the phases that need more
// spill a few hundred bytes, which costs less than the halved occupancy.  Two
// or more threads per node, and the FP64 path: capped at 128 registers, four
// blocks of 128.)
template <bool FP32, int LANES, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (FP32 && LANES == 1 ? 1024 : 512) / BLOCK)
    k_persistent(DevPtrs d, KParams k, int vin, int nsteps) {
    __shared__ int sm[33];
    __shared__ long long s_step;
    // wait test: the withheld block never arrives, so the others' barrier waits run out
    if ((int)blockIdx.x == k.withhold_block) return;
    // read by every thread before the first grid barrier; written only after it
    const bool pred0 = FP32 && *(volatile int *)d.pred_ok != 0;
    for (int st = 0; st < nsteps; ++st) {
        if (threadIdx.x == 0) {
            s_cur_u = d.ub[vin ^ 1];
            s_cur_pq = d.pqb[vin ^ 1];
        }
        __syncthreads();
        const bool predicted = FP32 && (st > 0 || pred0);
        if (!persistent_step<FP32, LANES, BLOCK>(d, k, vin, st, nsteps, predicted, sm, s_step)) return;
        vin ^= 1;
    }
    // the next launch may skip its first update phase (the end of this launch
    // orders every node's prediction before it)
    if (FP32 && blockIdx.x == 0 && threadIdx.x == 0) *(volatile int *)d.pred_ok = 1;
}

template <bool FP32, int LANES, int BLOCK>
cudaError_t launch_persistent_cfg(const DevPtrs &d, const KParams &k, int vin, int nsteps, cudaStream_t s) {
    auto kern = k_persistent<FP32, LANES, BLOCK>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, 0)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long need = ((long long)LANES * k.N + BLOCK - 1) / BLOCK;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * sms, need));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BLOCK);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, d, k, vin, nsteps);
}

// The persistent kernels of one precision and one thread count per node (both
// block sizes), each instantiated in a translation unit of its own
// (pd_persist.cu, compiled once per pair) so that they build in parallel.
template <bool FP32, int LANES>
cudaError_t launch_persistent_lanes(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block,
                                    cudaStream_t s);

template <bool FP32>
cudaError_t launch_persistent_impl(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s) {
    if (k.lanes == 8) return launch_persistent_lanes<FP32, 8>(d, k, vin, nsteps, block, s);
    if (k.lanes == 4) return launch_persistent_lanes<FP32, 4>(d, k, vin, nsteps, block, s);
    if (k.lanes == 2) return launch_persistent_lanes<FP32, 2>(d, k, vin, nsteps, block, s);
    return launch_persistent_lanes<FP32, 1>(d, k, vin, nsteps, block, s);
}

}  // namespace pd
