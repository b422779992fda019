// pd_internal.h -- shared declarations of the GB300 PeriDEM library
// (host runtime <-> CUDA kernels).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pd {

// Contact candidate list (Verlet list with a skin): every node keeps the nodes
// y of its aggregate with |p(y) - p(x)| < R_c + skin at the last rebuild, at
// most kMaxList of them, in ascending index.  A rebuild runs when some node
// has moved more than kSkinTrigger * skin since the last one, so every pair
// closer than R_c is always in the list (the force phase tests R_c exactly).
constexpr int kMaxList = 24;
constexpr double kSkinRatio = 0.10;     // skin = kSkinRatio * R_c
constexpr double kSkinTrigger = 0.45;   // < 1/2: margin for the float displacement test
// Rows q < kPrefetchListRows of the candidate lists are prefetched into L2 with
// the other read-only arrays of the force phase (most lists are shorter).
constexpr int kPrefetchListRows = 4;
// The force phase's read-only arrays are prefetched into L2 at the start of a
// step only when they take less than this (a fifth of the 129 MB L2).
constexpr size_t kPrefetchMaxBytes = 24u << 20;
// FP32-split bond columns: node index in the low kColBits bits, the bond's
// lattice offset di^2 + dj^2 (< 16 for horizons up to 4 h) in the top bits.
constexpr int kColBits = 28;
constexpr uint32_t kColMask = (1u << kColBits) - 1u;
// FP32-split bond stencil (horizon 3 h: the 24 offsets (di, dj) of the 5 x 5
// lattice block without its centre, numbered o = 0..23 in (dj, di) order).
// Nodes of a grain are numbered row by row (j, then i), so for a node whose
// neighbour rows are contiguous runs near it the neighbour at offset o is node
// x + di + D[dj], and the CSR order of its bonds is the order of o.  Per node:
//   x: bit o = bond at offset o exists (reference list), bit 31 = irregular
//      (a row with a gap near the node: its bonds are read from the CSR columns)
//   y: D[-2] | D[-1] << 16, z: D[1] | D[2] << 16 (16-bit two's complement)
//   w: first bond of the node's CSR row
constexpr uint32_t kStnIrregular = 0x80000000u;
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
    double pe5;            // pi eps_c^5: K_n = 18 k / pe5 for a pair's bulk modulus k (materials)
    double w0[4], wv[4];   // walls x_lo, x_hi, y_lo, y_hi at t = 0 and their normal velocities
    double ox, oy, cell;   // hash-grid origin and cell side (>= R_c)
    double inv_cell;       // 1 / cell
    double sx, sy;         // FP32-split shift: coordinates of the box map to [L, 2L)
    float rc2_hi, rc2_lo;  // R_c^2 as a float-float pair
    float rcf, knf;        // R_c and K_n as floats
    float oxs, oys, inv_cell_f;  // FP32 split: grid origin in shifted coordinates, 1 / cell
    float rs2;             // (R_c + skin)^2 as a float: radius of the candidate lists
    float dmax2;           // (kSkinTrigger skin)^2: displacement since the last rebuild that triggers the next
};

// Device pointers carved out of the caller's arena.
struct DevPtrs {
    // node state (N entries of (x, y)).  u and pq are the current step's
    // displacement and positions: a launch gets the buffers of its parity (the
    // host sets them per launch, the persistent kernel per step).  The FP32-split
    // path keeps two buffers of each, ub / pqb: the step with velocity parity vin
    // reads u^(n-1) from ub[vin] and holds u^n in ub[vin ^ 1], and its persistent
    // form writes the next step's u and pq into ub[vin] / pqb[vin] while the
    // others still read the current ones.  The FP64 path has one (ub[0] = ub[1]).
    double2 *X, *u, *v[2], *a, *p, *F, *parts;
    double2 *ub[2];
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
    // materials: per grain density, bulk modulus (FP64) and its own-material
    // contact stiffness 18 k / (pi eps_c^5) as a float (FP32-split contact laws)
    double *g_rho, *g_k;
    float *g_kf;
    // contact hash grid (T buckets)
    int *key, *count, *start, *cursor, *sorted, *blocksums;
    int2 *cell;         // hash-grid cell (x, y) of every node at the last rebuild
    // contact candidate lists (rebuilt when a node has moved kSkinTrigger * skin)
    int *nbr_cnt;       // list length of every node
    int *nbr;           // list entry q of node i at nbr[q N + i] (kMaxList slots), ascending node index
    float4 *sref;       // at the last rebuild: FP32 split pq, FP64 path (float u, 0, 0)
    int *rebuild;       // nonzero: rebuild the lists before the next force phase (cleared by the force phase)
    unsigned *pred_done;  // blocks of the displacement update that have finished (last-block election)
    int *rebuild_next;  // FP32-split persistent kernel: the next step's rebuild flag, raised in the velocity update
    int *pred_ok;       // nonzero: ub / pqb of the other parity hold the next step's u and pq (persistent kernel)
    uint4 *srec;        // position of sorted[t] in bucket order: FP32 split pq, FP64 p (16 bytes)
    void *fsum;         // split force phase: per-node lane sums, six components of N floats (FP32) or doubles
    // globals
    long long *step;
    double *t_now;      // time of the force evaluation that follows the predict phase
    int *status;        // PD_STATUS_COUNT counters
    unsigned *bar;      // grid barrier: [0] arrivals, [1] generation
    double *diag_part;  // per-block diagnostic partial sums
    double *diag_out;   // PD_DIAG_COUNT
    double *obs_gdam;   // particle damage of every grain (G)
    double *obs_wall;   // per aggregate: sums of the wall terms (16 n_agg)
    // FP32-split path
    int2 *lat;          // lattice indices (i, j) of every node in its grain frame
    float4 *gq;         // per grain: (h, h^2 hi, h^2 lo, V = h^2 as float)
    float4 *pq;         // shifted position (p + shift) as a float-float pair: (hi x, hi y, lo x, lo y)
    float4 *pqb[2];     // its two buffers (see ub)
    double2 *xs;        // X + the aggregate's shift (FP64)
    uint32_t *colx;     // bond columns with the lattice offset n = di^2 + dj^2 in the top 4 bits
    uint4 *stn;         // lattice stencil of every node's bonds (see kStnIrregular), when KParams::stencil
    float4 *gc;         // per grain: (c_w, s0, eps, rho) as floats
    double *g_invm;     // per grain: 1 / (rho V)
    float *g_invmf;     // the same as floats (FP32-split contexts)
    int4 *wall_cell;    // per aggregate: hash-grid cells of its walls x_lo, x_hi, y_lo, y_hi at the current time
    // autotuner backup of the state
    double2 *bu, *bv, *ba;
    float2 *af;         // FP32-split contexts: the acceleration, a = F / m + g rounded to float (d.a unused)
    uint32_t *bbits;
    // learned modal surrogate (FP32-split path)
    int *g_start;       // first node of every grain (G + 1)
    int *g_tmpl;        // template of every grain (-1: none)
    int *g_slot;        // row of the grain in its template's network batch
    int *tmpl_node;     // first basis row of every template (n_tmpl + 1)
    int *tmpl_slot;     // first network row of every template (n_tmpl + 1)
    float *basis;       // per template: mode-major [n_modes][2 n_t] (row r = 2 l + c of template node l), lattice frame
    uint16_t *bnm_hi, *bnm_lo;  // BF16 split of the basis, node-major [2 n_t][n_modes] (tensor-core expansion)
    uint16_t *bmm_hi, *bmm_lo;  // BF16 split of the basis, mode-major [n_modes][2 n_t] (tensor-core projection)
    int *slot_grain;    // grain of every network row (inverse of tmpl_slot + g_slot)
    int *tmpl_rows;     // first padded basis row of every template (n_tmpl + 1; 2 n_t rounded up to kSurExpandRows)
    int4 *proj_work;    // projection tiles: (template, first row, first basis row, chunk)
    int4 *exp_work;     // expansion tiles: (template, first row, first basis row, 0)
    float2 *sur_w;      // co-rotated local deformation / h of every node of an active grain, lattice frame
    float2 *sur_f;      // surrogate bond force / (E h) of every node of an active grain, lattice frame
    float *sur_xpart;   // projection partial sums [chunk][network row][mode]
    struct MlpRef *mlp_refs;  // per template: the network's device parameters
    int4 *mlp_work;     // inference tiles: (template, first row, end row, 0)
    int *mlp_err;       // set when a network tile's tensor-core wait gave up
    double *g_theta;    // grain orientation at meshing
    float4 *sur_fc;     // per grain: h as a float-float pair (hi, lo), centroid of its lattice indices (i, j)
    int *sur_active;    // 1 while the grain is advanced by the surrogate
    float2 *sur_rot;    // cos, sin of (theta + phi): lattice frame -> world
    float *sur_x;       // network input rows (modal coefficients / h)
    float *sur_y;       // network output rows (modal bond force / (E h))
    float2 *sur_fb;     // full bond force of surrogate nodes on judge steps
    float *sur_err;     // judged relative error of the surrogate nodal bond force
    float *sur_merr;    // judged relative error of the surrogate modal bond force
    float *sur_maxs;    // judged max |s| / s0 over the grain's bonds
    float *sur_qs, *sur_fs;  // per-grain samples (modal coefficients, modal bond force)
    float *sur_lambda;  // per template and mode: linearised modal stiffness (dimensionless)
};

// By-value kernel parameters (baked into captured graphs).
struct KParams {
    int N, G, wpn, n_diag_blocks, n_agg;
    unsigned T;         // hash buckets (power of two)
    double rho, rd, mu, gx, gy, dt, half_dt, half_dt2;
    float rhof, rdf, muf, dtf;   // the same as floats (FP32-split contact laws)
    float gxf, gyf;              // gravity as floats (FP32-split acceleration)
    float guard;        // FP32-split: |(|s| - s0)| < guard * s0 re-decides breaking in FP64
    float dmax2;        // smallest (kSkinTrigger skin)^2 of the aggregates: rebuild trigger
    int mat;            // 1: per-grain materials (K_n per pair, densities per grain)
    int micro, store;
    int lanes;          // threads per node in the force kernels (1, 4 or 8)
    int split;          // 1: lane sums through global memory and a separate epilogue pass
    int fp32;           // precision of the force phase
    int pf_bonds;       // > 0: prefetch the force phase's read-only arrays (this many bonds) into L2
    int stencil;        // FP32 split: bonds from the lattice stencil (DevPtrs::stn) instead of the columns
    // surrogate
    int sur;            // surrogate on
    int n_modes;        // modes of the basis (32)
    int judge_every;    // full bond kernel every judge_every steps
    float E;            // Young's modulus (force scale of the network output)
    float gate;         // fall back when max |s| > gate * s0
    float err_tol;      // fall back when the judged relative error exceeds this
    int n_proj_work, n_exp_work;  // tensor-core tiles of the projection / expansion
    int n_rows;                   // network rows (templated grains)
    // bounded waits of the persistent kernel: polls of a grid barrier before it
    // gives up, and a block that withholds its arrival (-1: none; a wait test)
    long long bar_spins;
    int withhold_block;
};


// Surrogate phases (pd_surrogate.cu): co-rotated modal coefficients of the
// active grains before the force phase, and the judge after it.
// Tile sizes of the tensor-core projection (rows of 2 n_t per chunk) and expansion.
constexpr int kSurChunk = 128;
constexpr int kSurExpandRows = 128;
constexpr int kSurTile = 128;      // network rows (grains) per tile
cudaError_t sur_init_attributes();   // shared-memory limits of the tensor-core kernels (not capturable)
cudaError_t launch_sur_frame(const DevPtrs &d, const KParams &k, int all_templated, cudaStream_t s);
// CUDA-core projection of a per-node vector field onto the basis, for every
// templated grain: world-frame bond forces (rotated into the lattice frame and
// scaled by 1/(E h)) when F is given, else the local deformation sur_w.
cudaError_t launch_sur_project_cc(const DevPtrs &d, const KParams &k, const double2 *F, float *out, cudaStream_t s);
// The chain after the frame kernel; with pdl, each is launched with
// programmatic stream serialisation (it may begin while its predecessor on the
// stream finishes, staging its basis or weight operands meanwhile).
cudaError_t launch_sur_project_tc(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl = false);
cudaError_t launch_sur_reduce(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl = false);
cudaError_t launch_sur_expand_tc(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl = false);
cudaError_t launch_sur_judge(const DevPtrs &d, const KParams &k, cudaStream_t s);

// Device pointers of one network's inference parameters (BF16 weights, FP32
// parameter vector with the biases).
struct MlpRef {
    const void *W1, *W2, *W3;
    const float *p;
    const float *lin;   // nullable: y = net(x) - lin (.) x (the surrogate's linear modal part, 32 values)
};
}  // namespace pd
struct pd_mlp;
namespace pd {
// Forward pass of a surrogate network on a given stream (captured into the step graph).
int mlp_forward_stream(pd_mlp *m, const float *x, float *y, int batch, cudaStream_t s);
int mlp_ref(pd_mlp *m, MlpRef *out);
// Several networks in one launch: work item (network, first row, end row), rows of x / y.
cudaError_t launch_mlp_grouped(const MlpRef *refs, const int4 *work, int n_work, const float *x, float *y, int *err,
                               cudaStream_t s, bool pdl = false);
cudaError_t mlp_init_attributes();

// Launch of kernel `kern` on stream s, with programmatic stream serialisation
// when pdl is set (the kernel then has to call grid_dep_wait() before it reads
// what the previous kernel of the stream writes).
template <class... KArgs, class... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Record an error for pd_last_error() and return `code`.
int set_error(int code, const char *msg);

// Launch wrappers (stream-ordered, capture-safe).
// Displacement update and positions; with use_cond, the last block sets the
// graph conditional `cond` to the rebuild flag.
cudaError_t launch_predict(const DevPtrs &d, const KParams &k, int vin, int advance, cudaStream_t s,
                           cudaGraphConditionalHandle cond, int use_cond);
// Rebuild of the contact candidate lists (kernels return at once when the
// rebuild flag is clear).
cudaError_t launch_rebuild(const DevPtrs &d, const KParams &k, cudaStream_t s);
// Force phase; with the split variant, phase 1 launches only the lane sums
// and phase 2 only the epilogue (0: both; the fused variant takes only 0).
cudaError_t launch_force(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase = 0);
cudaError_t launch_force64(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase = 0);
cudaError_t launch_force32(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase = 0);
cudaError_t launch_positions(const DevPtrs &d, const KParams &k, cudaStream_t s);
// Element-wise conversions of n float2 / double2 pairs (the FP32-split acceleration field).
cudaError_t launch_widen(const float2 *src, double2 *dst, size_t n, cudaStream_t s);
cudaError_t launch_narrow(const double2 *src, float2 *dst, size_t n, cudaStream_t s);
cudaError_t launch_diagnostics(const DevPtrs &d, const KParams &k, int vcur, cudaStream_t s);
// Particle damage of every grain (gdam[G]) and per-aggregate sums of the wall
// terms (wsum[16 n_agg]) at the current state.
cudaError_t launch_observables(const DevPtrs &d, const KParams &k, int vcur, double *gdam, double *wsum,
                               cudaStream_t s);

// Persistent cooperative step kernel: nsteps full time steps in one launch
// (phases separated by bounded grid barriers).  block = threads per block
// (128 or 256); the grid is the largest co-resident one (occupancy API).
cudaError_t launch_persistent(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);
cudaError_t launch_persistent64(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);
cudaError_t launch_persistent32(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s);

}  // namespace pd
