// pd_internal.h -- shared declarations of the GB300 PeriDEM library
// (host runtime <-> CUDA kernels).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pd {

// Upper bound on contact candidates (nodes within R_c) gathered per node.
constexpr int kMaxCand = 32;
// Threads per block of the node-parallel kernels.
constexpr int kBlock = 128;
// Scan tile: threads x items per thread.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

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
    // per-grain constants
    double *g_cw, *g_s0, *g_eps;
    // contact hash grid (T buckets)
    int *key, *count, *start, *cursor, *sorted, *blocksums;
    // globals
    long long *step;
    double *walls_now;  // 4 wall positions used by the current force evaluation
    int *status;        // PD_STATUS_COUNT counters
    double *diag_part;  // per-block diagnostic partial sums
    double *diag_out;   // PD_DIAG_COUNT
    // FP32-split path
    int2 *lat;          // lattice indices (i, j) of every node in its grain frame
    float4 *gq;         // per grain: (h, h^2 hi, h^2 lo, V = h^2 as float)
    float2 *ph, *pl;    // shifted position (p + shift) as a float-float pair
};

// By-value kernel parameters (baked into captured graphs).
struct KParams {
    int N, G, wpn, n_diag_blocks;
    unsigned T;         // hash buckets (power of two)
    double rho, Kn, Rc, rd, mu, gx, gy, dt, half_dt, half_dt2;
    double w0[4], wv[4];
    double cell, ox, oy;
    double sx, sy;      // FP32-split position shift: coordinates map to [box, 2 box)
    float rc2_hi, rc2_lo;  // R_c^2 as a float-float pair
    float guard;        // FP32-split: |(|s| - s0)| < guard * s0 re-decides breaking in FP64
    int micro, store;
};

// Record an error for pd_last_error() and return `code`.
int set_error(int code, const char *msg);

// Launch wrappers (stream-ordered, capture-safe).
cudaError_t launch_predict(const DevPtrs &d, const KParams &k, int vin, int advance, cudaStream_t s);
cudaError_t launch_bin(const DevPtrs &d, const KParams &k, cudaStream_t s);
cudaError_t launch_force_fp64(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s);
cudaError_t launch_force_fp32(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s);
cudaError_t launch_positions(const DevPtrs &d, const KParams &k, cudaStream_t s);
cudaError_t launch_diagnostics(const DevPtrs &d, const KParams &k, int vcur, cudaStream_t s);

}  // namespace pd
