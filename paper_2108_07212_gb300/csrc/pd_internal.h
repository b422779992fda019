// pd_internal.h -- shared declarations of the GB300 PeriDEM library
// (host runtime <-> CUDA kernels).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pd {

// Upper bound on contact candidates (nodes within R_c) gathered per lane.
constexpr int kMaxCand = 16;
// Threads per block of the node-parallel multi-kernel path.
constexpr int kBlock = 128;
// Scan tile: threads x items per thread.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
// Bounded spin of the persistent kernel's grid barrier (~1 s with 64 ns sleeps).
constexpr long long kBarrierSpins = 16LL * 1000 * 1000;

// Per-aggregate parameters: every aggregate is an independent problem with its
// own wall box, contact radius and contact stiffness (R_c and K_n follow the
// aggregate's smallest lattice spacing).
struct AggParams {
    double Rc, Kn;
    double w0[4], wv[4];   // walls x_lo, x_hi, y_lo, y_hi at t = 0 and their normal velocities
    double ox, oy, cell;   // hash-grid origin and cell side (>= R_c)
    double sx, sy;         // FP32-split shift: coordinates of the box map to [L, 2L)
    float rc2_hi, rc2_lo;  // R_c^2 as a float-float pair
};

// Device pointers carved out of the caller's arena.
struct DevPtrs {
    // node state (N entries of (x, y))
    double2 *X, *u, *v[2], *a, *p, *F, *parts;
    double *V;
    int *grain;
    // bonds: CSR, reference lengths |xi|, broken bits (wpn words per node)
    int *row_ptr, *col;
    double *xi;
    uint32_t *bits;
    // per-grain constants and aggregate of each grain
    double *g_cw, *g_s0, *g_eps;
    int *g_agg;
    AggParams *agg;
    // contact hash grid (T buckets)
    int *key, *count, *start, *cursor, *sorted, *blocksums;
    // globals
    long long *step;
    double *t_now;      // time of the force evaluation that follows the predict phase
    int *status;        // PD_STATUS_COUNT counters
    unsigned *bar;      // grid barrier: [0] arrivals, [1] generation
    double *diag_part;  // per-block diagnostic partial sums
    double *diag_out;   // PD_DIAG_COUNT
    // FP32-split path
    int2 *lat;          // lattice indices (i, j) of every node in its grain frame
    float4 *gq;         // per grain: (h, h^2 hi, h^2 lo, V = h^2 as float)
    float2 *ph, *pl;    // shifted position (p + shift) as a float-float pair
    // autotuner backup of the state
    double2 *bu, *bv, *ba;
    uint32_t *bbits;
};

// By-value kernel parameters (baked into captured graphs).
struct KParams {
    int N, G, wpn, n_diag_blocks, n_agg;
    unsigned T;         // hash buckets (power of two)
    double rho, rd, mu, gx, gy, dt, half_dt, half_dt2;
    float guard;        // FP32-split: |(|s| - s0)| < guard * s0 re-decides breaking in FP64
    int micro, store;
    int lanes;          // threads per node in the force kernels (1, 4 or 8)
    int fp32;           // precision of the force phase
};

// Record an error for pd_last_error() and return `code`.
int set_error(int code, const char *msg);

// Launch wrappers (stream-ordered, capture-safe).
cudaError_t launch_predict(const DevPtrs &d, const KParams &k, int vin, int advance, cudaStream_t s);
cudaError_t launch_bin(const DevPtrs &d, const KParams &k, cudaStream_t s);
cudaError_t launch_force(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s);
cudaError_t launch_force64(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s);
cudaError_t launch_force32(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s);
cudaError_t launch_positions(const DevPtrs &d, const KParams &k, cudaStream_t s);
cudaError_t launch_diagnostics(const DevPtrs &d, const KParams &k, int vcur, cudaStream_t s);

// Persistent cooperative step kernel: nsteps full time steps in one launch
// (phases separated by bounded grid barriers).  block = threads per block
// (128 or 256); the grid is the largest co-resident one (occupancy API).
cudaError_t launch_persistent(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);
cudaError_t launch_persistent64(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);
cudaError_t launch_persistent32(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);

}  // namespace pd
