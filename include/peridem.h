/*
 * peridem.h -- C ABI of the GB300 PeriDEM library (libperidem.so).
 *
 * The library advances the PeriDEM equations of motion (eq:full) of an
 * aggregate of deformable, breakable 2D grains with velocity Verlet
 * (Algorithm 1).  Everything in the time loop runs in hand-written CUDA
 * kernels for sm_103a: intra-grain bond forces with irreversible breaking
 * (eq:peri, eq:pmb, Sec. 3.1), node-to-node contact with repulsion, normal
 * damping and regularised stick/slip friction (Secs. 4.1-4.3), self-contact
 * between unbonded nodes of one grain (Sec. 4.4), analytic wall contact with
 * corner inclusion-exclusion (Sec. 4.5), and the Verlet update.
 *
 * Conventions
 *  - Units are SI.  Vectors are interleaved (x, y) pairs of doubles.
 *  - Every entry point returns 0 (PD_OK) or a negative PD_E* code; the text of
 *    the last error of the calling thread is returned by pd_last_error().
 *    No C++ exception crosses this boundary.
 *  - Ownership: the caller owns every buffer it passes.  Device memory for the
 *    simulation state is ONE caller-allocated arena (pd_arena_bytes /
 *    pd_bind_arena) that must stay alive until pd_destroy; the library never
 *    frees caller memory.  The context itself owns only host metadata, CUDA
 *    graphs and its host copies of the mesh.
 *  - Streams: all device work is enqueued on the stream given to pd_create,
 *    in stream order; calls return without waiting unless stated otherwise.
 *  - Device-side error conditions (non-finite acceleration, candidate list
 *    overflow, a node past a wall) are latched in a device status word and
 *    reported by pd_status().
 */
#ifndef PERIDEM_H
#define PERIDEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define PD_OK 0
#define PD_EINVAL -1     /* invalid argument (null pointer, size, value)       */
#define PD_ESTATE -2     /* call out of order (e.g. pd_step before bind)        */
#define PD_ECUDA -3      /* a CUDA runtime call failed                          */
#define PD_ENUMERIC -4   /* non-finite acceleration detected on the device      */
#define PD_EOVERFLOW -5  /* a node had more contact candidates than supported   */
#define PD_ENOMEM -6     /* host allocation failed or arena too small           */
#define PD_ETIMEOUT -7   /* a bounded device wait gave up                       */

/* ---- precision modes ------------------------------------------------------- */
#define PD_FP64 0        /* plain FP64 everywhere                               */
#define PD_FP32_SPLIT 1  /* FP32 bond/contact arithmetic, FP64 integration      */

/* ---- micromodulus (Table 1) ------------------------------------------------ */
#define PD_MICRO_CONSTANT 0
#define PD_MICRO_CONIC 1

/*
 * Run parameters.  Material (E, nu, k_bulk, rho, Gc) is shared by all grains.
 * Each grain has its own lattice spacing h (grain_geom), hence its own horizon
 * eps = horizon_ratio * h and its own c_w, s0 (Table 1).  The contact radius is
 * R_c = rc_ratio * h_min and the contact stiffness K_n = 18 k / (pi eps_c^5)
 * with eps_c = horizon_ratio * h_min (Sec. 4.1), h_min the smallest spacing.
 * Walls form the rectangle [wall_lo, wall_hi] at t = 0; wall_vel_* are the
 * normal velocities of the four walls (x_lo, y_lo in wall_vel_lo; x_hi, y_hi
 * in wall_vel_hi), so a wall is at w0 + v t (Sec. 6.4 moving top wall).
 */
typedef struct pd_params {
    double E;               /* Young's modulus [Pa]                             */
    double nu;              /* Poisson ratio used in c_w (1/3 for 2D bonds)     */
    double k_bulk;          /* bulk modulus in K_n [Pa]                         */
    double rho;             /* density [kg/m^3]                                 */
    double Gc;              /* critical energy release rate [J/m^2]             */
    double horizon_ratio;   /* eps / h                                          */
    double rc_ratio;        /* R_c / h_min                                      */
    double damping_ratio;   /* r_d in beta_d = 2 r_d sqrt(K_n rho / V_y)         */
    double friction;        /* mu                                               */
    double gravity[2];      /* body acceleration b / rho [m/s^2]                */
    double dt;              /* time step [s]                                    */
    double wall_lo[2];      /* x_min, y_min at t = 0                            */
    double wall_hi[2];      /* x_max, y_max at t = 0                            */
    double wall_vel_lo[2];  /* velocity of the x_min wall (along x), y_min (y)  */
    double wall_vel_hi[2];  /* velocity of the x_max wall (along x), y_max (y)  */
    int32_t micromodulus;   /* PD_MICRO_*                                       */
    int32_t precision;      /* PD_FP64 or PD_FP32_SPLIT                         */
    int32_t store_parts;    /* nonzero: keep the four force parts of the last   */
                            /* evaluation (bond|self|neighbour|wall), for tests */
    int32_t lanes;          /* threads per node in the force kernels: 1, 2, 4,  */
                            /* 8, or 0 for the default (4); 1 sums every force  */
                            /* in the textbook order of eq:full                 */
} pd_params;

/* ---- state fields (pd_get_state / pd_set_state) ---------------------------- */
#define PD_FIELD_X 0            /* double[2N] reference positions (get)              */
#define PD_FIELD_DISP 1         /* double[2N] displacement u (get/set)               */
#define PD_FIELD_VEL 2          /* double[2N] velocity (get/set)                     */
#define PD_FIELD_ACC 3          /* double[2N] acceleration of the last step (get/set)*/
                                /* (FP32-split contexts keep it in FP32: a set      */
                                /* rounds to float, a get returns the floats)       */
#define PD_FIELD_POS 4          /* double[2N] current position X + u (get)           */
#define PD_FIELD_FORCE 5        /* double[2N] total nodal force, last evaluation     */
#define PD_FIELD_FORCE_PARTS 6  /* double[8N] bond|self|neighbour|wall (store_parts) */
#define PD_FIELD_BROKEN 7       /* uint8[n_bonds] 1 = broken, CSR order (get/set)    */
#define PD_FIELD_DAMAGE 8       /* double[N] broken / reference bonds (get)          */
#define PD_FIELD_GRAIN 9        /* int32[N] grain id of each node (get)              */
#define PD_FIELD_VOLUME 10      /* double[N] nodal volume h^2 (get)                  */
#define PD_FIELD_ROW_PTR 11     /* int32[N+1] CSR row pointer of the bond lists      */
#define PD_FIELD_COL 12         /* int32[n_bonds] CSR columns (ascending per row)    */
#define PD_FIELD_LATTICE 13     /* int32[2N] lattice indices (i, j) in grain frame   */
#define PD_FIELD_STEP 14        /* int64[1] number of completed time steps (get/set) */
#define PD_FIELD_GRAIN_TEMPLATE 15 /* int32[G] bond-network template of every grain (get) */

/* ---- status word slots (pd_status) ------------------------------------------ */
#define PD_STATUS_PENETRATION 0 /* node found past a wall (treated as touching)     */
#define PD_STATUS_COINCIDENT 1  /* two nodes at the same position (pair skipped)    */
#define PD_STATUS_NONFINITE 2   /* non-finite acceleration                          */
#define PD_STATUS_OVERFLOW 3    /* contact candidates beyond the per-node capacity  */
#define PD_STATUS_TIMEOUT 4     /* a grid barrier of the persistent kernel gave up  */
#define PD_STATUS_REBUILDS 5    /* rebuilds of the contact candidate lists (not an error) */
#define PD_STATUS_COUNT 8

/* ---- diagnostics (pd_diagnostics) ------------------------------------------- */
#define PD_DIAG_KE 0            /* kinetic energy sum 1/2 rho V |v|^2                */
#define PD_DIAG_EBOND 1         /* bond energy sum over bonds 1/2 c w s^2 |xi| V V   */
#define PD_DIAG_PX 2            /* linear momentum x                                 */
#define PD_DIAG_PY 3            /* linear momentum y                                 */
#define PD_DIAG_LZ 4            /* angular momentum about the origin                 */
#define PD_DIAG_NBROKEN 5       /* number of broken directed bonds                   */
#define PD_DIAG_ECONTACT 6      /* contact potential: 1/2 K_n V_x V_y (R_c - d)^2 over  */
                                /* pairs of grains within R_c (eq:law-repulsive) plus  */
                                /* the self-contact springs of unbonded nodes of one   */
                                /* grain (Sec. 4.4: stiffness c_w / R_c about R_c, or  */
                                /* c_w / |xi| about |xi| when |xi| < R_c)               */
#define PD_DIAG_EWALL 7         /* single-wall potential: sum over nodes and walls of  */
                                /* K_n V_x int_d^{R_c} |S_l| (R_c - |c_l - p|) ds       */
                                /* (Sec. 4.5); corner regions carry none               */
#define PD_DIAG_COUNT 8

typedef struct pd_ctx pd_ctx;

/* Text of the last error raised on the calling thread ("" if none). */
const char *pd_last_error(void);

/*
 * Create a context.  `params` is copied.  `cuda_stream` is a cudaStream_t (may
 * be NULL for the legacy default stream) on which all later device work of
 * this context is enqueued; no device work happens before pd_bind_arena, so a
 * context can mesh and build bonds on a machine without a GPU.
 * Errors: PD_EINVAL (null out/params, non-positive dt/rho/E/horizon_ratio).
 */
int pd_create(pd_ctx **out, const pd_params *params, void *cuda_stream);

/* Destroy a context (waits for its stream).  Safe on NULL. */
int pd_destroy(pd_ctx *ctx);

/*
 * Mesh the grains (host).  Grain shapes are polygon loops in units of the
 * grain radius R: shape s owns loops shape_loop_start[s] .. shape_loop_start[s+1]-1,
 * loop l owns vertices loop_vtx_start[l] .. loop_vtx_start[l+1]-1 of vtx_xy
 * (interleaved x, y).  The first loop of a shape is its outer boundary
 * (counter-clockwise), further loops are holes (clockwise).
 * grain_geom holds n_grains rows of 7 doubles (cx, cy, R, theta, vx, vy, h).
 * Each grain is discretised on the lattice (i h, j h) of its own frame: the
 * points strictly inside the grain and at least 1e-6 h from its boundary, in
 * order of j then i, rotated by theta and moved to (cx, cy); every node has
 * volume h^2 (Sec. 5: nodes inside the grain, mesh size = node spacing) and
 * initial velocity (vx, vy).  Nodes are numbered grain by grain.
 * Writes the node count to *n_nodes_out.  Errors: PD_EINVAL, PD_ESTATE
 * (called twice), PD_ENOMEM.
 */
int pd_mesh_grains(pd_ctx *ctx, int n_shapes, const int32_t *shape_loop_start,
                   const int32_t *loop_vtx_start, const double *vtx_xy, int n_grains,
                   const int32_t *grain_shape, const double *grain_geom, int64_t *n_nodes_out);

/*
 * Build the reference neighbour (bond) lists S^ref of Algorithm 1 (host):
 * node y of the same grain is a neighbour of x when their lattice offset has
 * di^2 + dj^2 < horizon_ratio^2 (strict |xi| < eps) and the segment x-y does
 * not cross the grain's extended boundary (every boundary loop moved out by
 * delta along the outward vertex bisectors) nor an outer-angle bisector ray
 * of a non-convex cusp (Sec. 4 "bonds in nonconvex domains").  Lists are CSR,
 * sorted by node, columns ascending.  Writes the directed bond count.
 * Errors: PD_ESTATE (before pd_mesh_grains), PD_ENOMEM, PD_EINVAL (more than
 * 2^29 nodes, the limit of the contact grid's 32-bit buckets).
 */
int pd_build_bonds(pd_ctx *ctx, int64_t *n_bonds_out);

/* Bytes of device memory the caller must provide to pd_bind_arena (after
 * pd_build_bonds).  Errors: PD_ESTATE. */
int pd_arena_bytes(pd_ctx *ctx, size_t *bytes);

/*
 * Bind a caller-owned device arena of at least pd_arena_bytes bytes (256-byte
 * aligned), upload the mesh, bonds and initial state on the context stream and
 * compute the initial acceleration a^0 = F(u^0, v^0) / (rho V) + b / rho
 * (Algorithm 1, first line).  Errors: PD_ESTATE, PD_EINVAL (null/misaligned
 * pointer, too small), PD_ECUDA.
 */
int pd_bind_arena(pd_ctx *ctx, void *device_arena, size_t bytes);

/*
 * Advance n_steps >= 0 velocity-Verlet steps (Algorithm 1) asynchronously on
 * the context stream; the step sequence runs as captured CUDA graphs.  The
 * contact neighbourhoods S^nbr (Algorithm 1, nodes within R_c) are taken from
 * per-node candidate lists of radius R_c + skin (skin = 0.1 R_c), rebuilt by
 * a hash-grid counting sort in a conditional graph node only in steps where
 * some node has moved more than 0.45 skin since the last rebuild; every pair
 * is still tested against R_c exactly, so the forces are those of a full
 * search.  status[PD_STATUS_REBUILDS] counts the rebuilds.
 * Errors: PD_ESTATE (not bound), PD_EINVAL (n_steps < 0), PD_ECUDA.
 */
int pd_step(pd_ctx *ctx, int n_steps);

/* Where the caller's buffer of pd_get_state / pd_set_state lives. */
#define PD_MEM_HOST 0        /* host memory: the call waits for the stream        */
#define PD_MEM_DEVICE 1      /* device memory: a copy enqueued on the stream      */
#define PD_MEM_HOST_ASYNC 2  /* page-locked host memory: a copy enqueued on the   */
                             /* stream; the call does not wait, and the caller   */
                             /* keeps the buffer valid (and, for a get, reads it) */
                             /* only after synchronising the stream              */

/*
 * Copy a state field (PD_FIELD_*) into dst (bytes must equal the field size).
 * dst_on_device: PD_MEM_HOST (the call waits for the stream and copies to host
 * memory), PD_MEM_DEVICE (device-to-device copy enqueued on the stream) or
 * PD_MEM_HOST_ASYNC (copy to page-locked host memory enqueued on the stream;
 * BROKEN and DAMAGE, converted on the host, always wait).  Mesh fields (X,
 * GRAIN, VOLUME, ROW_PTR, COL, LATTICE) can be read from host copies before
 * pd_bind_arena.  Errors: PD_EINVAL (unknown field, size mismatch), PD_ESTATE,
 * PD_ECUDA.
 */
int pd_get_state(pd_ctx *ctx, int field, void *dst, size_t bytes, int dst_on_device);

/* Overwrite a settable state field (DISP, VEL, ACC, BROKEN, STEP) from host
 * memory (src_on_device = PD_MEM_HOST: the call waits), device memory
 * (PD_MEM_DEVICE) or page-locked host memory without waiting
 * (PD_MEM_HOST_ASYNC; BROKEN and STEP, read on the host, always wait),
 * stream-ordered.  Errors as above. */
int pd_set_state(pd_ctx *ctx, int field, const void *src, size_t bytes, int src_on_device);

/* Recompute the forces and acceleration of the current state without moving
 * it (as for a^0): fills FORCE (and FORCE_PARTS) and sets ACC.  Bonds may
 * break.  Errors: PD_ESTATE, PD_ECUDA. */
int pd_eval_forces(pd_ctx *ctx);

/* Reductions of the current state into out[PD_DIAG_COUNT] (waits for the
 * stream).  The kinetic energy, momenta and the bond, contact and wall
 * potentials give the energy balance of Sec. 4.3 (with r_d = mu = 0 and no
 * breaking, KE + E_bond + E_contact + E_wall minus the work of the body force
 * is conserved away from wall corners).  The contact candidate lists are
 * rebuilt for the current state first (counted in
 * status[PD_STATUS_REBUILDS]).  Errors: PD_ESTATE, PD_ECUDA. */
int pd_diagnostics(pd_ctx *ctx, double *out);

/* Copy the device status word into out[PD_STATUS_COUNT] (waits) and return
 * PD_OK, or the first error code it implies (PD_ENUMERIC, PD_EOVERFLOW,
 * PD_ETIMEOUT: a bounded device wait -- a grid barrier of the persistent
 * kernel or a tensor-core wait of the surrogate -- gave up; the surrogate's
 * results of that step are invalid and it is off from then on). */
int pd_status(pd_ctx *ctx, int32_t *out);

/* Zero the status counters, the surrogate networks' error word and the grid
 * barrier of the persistent kernel, and make the next step rebuild the contact
 * candidate lists (waits for the stream).  After PD_ETIMEOUT the step that gave
 * up is partly done: restore DISP, VEL, ACC, BROKEN and STEP from a copy, then
 * clear the status, before stepping on.  Errors: PD_ESTATE, PD_ECUDA. */
int pd_clear_status(pd_ctx *ctx);

/* Test hook of the bounded waits of the persistent kernel (pd_set_path modes 1
 * and 3, surrogate off).  withhold_block >= 0: that block of every later
 * launch returns before its first grid-barrier arrival, so the other blocks'
 * waits run out after max_spins polls of about 64 ns each, set
 * status[PD_STATUS_TIMEOUT] and return; no device fault is involved.
 * withhold_block = -1 and max_spins = 0 restore the default (no block
 * withheld, about 1 s of polling).  Re-captures the step graphs.
 * Errors: PD_EINVAL (withhold_block < -1, max_spins < 0), PD_ESTATE, PD_ECUDA. */
int pd_set_wait_test(pd_ctx *ctx, int withhold_block, long long max_spins);

/* Scalar facts of the context (out has 15 slots): out[0] N, out[1] directed
 * bonds, out[2] grains, out[3] h_min, out[4] R_c, out[5] K_n (aggregate 0),
 * out[6] dt, out[7] completed steps, out[8] max bonds per node, out[9] contact
 * hash buckets, out[10] step path (0 graph of kernels, 1 persistent kernel),
 * out[11] threads per node, out[12] threads per block of the persistent
 * kernel, out[13] aggregates, out[14] bond-network templates (grains of one
 * shape meshed at the same h/R share one lattice and one bond network). */
int pd_info(pd_ctx *ctx, double *out);

/*
 * Batched ensembles: declare that the meshed grains form n_agg independent
 * aggregates (after pd_mesh_grains, before pd_bind_arena).  grain_agg[g] is
 * the aggregate of grain g; agg_walls holds 8 doubles per aggregate: the wall
 * box x_lo, x_hi, y_lo, y_hi at t = 0 and the normal velocities of those four
 * walls.  Each aggregate gets its own R_c and K_n from its smallest lattice
 * spacing (Sec. 4.1) and contact never crosses aggregates, so a batched run
 * advances every aggregate exactly as a run of that aggregate alone would,
 * with all aggregates in the same launches.  Without this call the context is
 * one aggregate bounded by the walls of pd_params.
 * Errors: PD_ESTATE, PD_EINVAL (ids out of range, empty box).
 */
int pd_set_aggregates(pd_ctx *ctx, int n_agg, const int32_t *grain_agg, const double *agg_walls);

/*
 * Materials (Sec. 4.1 and the material table of Sec. 5): grain g takes the
 * properties of material grain_material[g] (int32[G], 0 <= m < n_mat), read
 * from props (double[4 n_mat], caller-owned, copied): E (Pa), bulk modulus k
 * (Pa), density rho (kg/m^3) and fracture energy Gc (J/m^2).  Its bond
 * constants c_w and s0 (Table 1) follow from its E and Gc.  Contact between
 * grains of bulk moduli k1 and k2 uses K_n = 18 k / (pi eps_c^5) with the
 * harmonic mean k = 2 k1 k2 / (k1 + k2) (Sec. 4.1); a wall, a rigid body,
 * uses the grain's own k.  The damping coefficient beta_d takes the harmonic
 * mean of the two densities (so that a pair's damping ratio stays sqrt(2) r_d);
 * friction's regularisation dt / (rho V_x) and the nodal mass rho V take the
 * node's own density.  Without this call every grain has the material of
 * pd_params.  Call after pd_mesh_grains and before pd_bind_arena; the learned
 * surrogate runs with one material only.
 * Errors: PD_ESTATE (order, or a surrogate configured), PD_EINVAL (non-positive
 * or non-finite property, material index out of range).
 */
int pd_set_materials(pd_ctx *ctx, int n_mat, const double *props, const int32_t *grain_material);

/*
 * Autotuner: time candidate step paths on the current state -- a graph of
 * separate kernels or one persistent cooperative kernel per 16 steps, each with
 * the force phase fused or split, 1, 2, 4 or 8 threads per node,
 * pd_set_path modes 0-4 and 6 (threads per node fixed when pd_params.lanes is
 * nonzero), 128 or 256 threads per persistent block -- pick the fastest, and
 * re-capture the step graphs.  The
 * state is saved and restored around the trials, so the simulation does not
 * advance.  report (nullable, 4 doubles): path, threads per node, block, best
 * ms per step.  Different choices only reorder floating-point sums.
 * Errors: PD_ESTATE, PD_ECUDA.
 */
int pd_autotune(pd_ctx *ctx, double *report);

/* Select the step path explicitly (instead of pd_autotune): mode 0 = graph of
 * separate kernels, 1 = persistent cooperative kernel, 2 and 3 = the same with
 * the force phase split in two passes (lane sums through device memory, then
 * walls and update one thread per node); modes 4-7 = modes 0-3 with the
 * candidate-list rebuild kernels launched every step (returning at once when no
 * rebuild is due) instead of behind a conditional graph node (same results;
 * the persistent kernel ignores this bit; profilers that cannot trace kernels
 * of graphs with conditional nodes need it); lanes 1, 2, 4 or 8 threads per
 * node (1 = textbook summation order); block 128 or 256 threads (persistent
 * kernel).  The FP32-split persistent kernel forms the next step's displacement
 * and positions in its velocity update (device memory of the arena holds two
 * buffers of each); the next launch starts from them unless the state was
 * written (pd_set_state), evaluated (pd_eval_forces) or stepped on another path
 * in between.  The default path is mode 2 with 4 threads per node.  Re-captures
 * the step graphs.  Errors: PD_ESTATE, PD_EINVAL, PD_ECUDA. */
int pd_set_path(pd_ctx *ctx, int mode, int lanes, int block);

/* ---- kernel timing (instrumentation) ----------------------------------------- */
#define PD_TIMER_PREDICT 0      /* memset + displacement update / positions / bucket counts */
#define PD_TIMER_BIN 1          /* scan + scatter of the contact hash grid               */
#define PD_TIMER_FORCE 2        /* force + acceleration + velocity kernel                */
#define PD_TIMER_COUNT 4

/* Enable (1) or disable (0) per-kernel timing: while enabled, pd_step runs
 * one-step graphs that also record CUDA events around each kernel group.
 * Errors: PD_ESTATE (not bound), PD_ECUDA. */
int pd_set_timing(pd_ctx *ctx, int enable);

/* Durations in milliseconds of the kernel groups of the LAST step run with
 * timing enabled (waits for the stream): out[PD_TIMER_*]. */
int pd_kernel_times(pd_ctx *ctx, double *out);

/* ---- surrogate network: MLP on the tensor cores -------------------------------- */
#define PD_MLP_IN 32
#define PD_MLP_HIDDEN 128
#define PD_MLP_OUT 32
#define PD_MLP_NPARAMS 24864

/*
 * A small network for the learned per-grain modal surrogate (not in the paper):
 * y = W3 g(W2 g(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 32, g = GELU
 * (x Phi(x), erf form).  Weights and activations enter the tensor cores as BF16
 * (tcgen05.mma), accumulation is FP32; FP32 master parameters are trained with
 * Adam on mean squared error by the library's own forward and backward kernels.
 * Parameters are one flat FP32 array of PD_MLP_NPARAMS values: W1[128][32],
 * b1[128], W2[128][128], b2[128], W3[32][128], b3[32] (weights [out][in]).
 * Device memory: one caller-owned arena (pd_mlp_arena_bytes, 256-byte aligned).
 * Inputs x are FP32 [batch][32] row-major, outputs y FP32 [batch][32], targets t
 * FP32 [batch][32], all device pointers; 1 <= batch <= max_batch.
 * Errors: PD_EINVAL, PD_ESTATE (not bound), PD_ECUDA, PD_ETIMEOUT (a bounded
 * tensor-core wait gave up).
 */
typedef struct pd_mlp pd_mlp;
int pd_mlp_create(pd_mlp **out, int max_batch, void *cuda_stream);
int pd_mlp_destroy(pd_mlp *mlp);
int pd_mlp_arena_bytes(pd_mlp *mlp, size_t *bytes);
int pd_mlp_bind_arena(pd_mlp *mlp, void *device_arena, size_t bytes);
int pd_mlp_set_params(pd_mlp *mlp, const float *params_host);   /* also resets Adam */
int pd_mlp_get_params(pd_mlp *mlp, float *params_host);
/* y = net(x), stream-ordered, no wait. */
int pd_mlp_forward(pd_mlp *mlp, const float *x, float *y, int batch);
/* Loss mean((net(x) - t)^2) and its gradient w.r.t. the parameters (host
 * outputs, nullable; waits).  The parameters do not change. */
int pd_mlp_loss_grad(pd_mlp *mlp, const float *x, const float *t, int batch, float *loss_host, float *grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; the
 * loss before the step is written to *loss_host when non-null (waits). */
int pd_mlp_train_step(pd_mlp *mlp, const float *x, const float *t, int batch, float lr, float *loss_host);

/*
 * Learned per-grain modal surrogate (not in the paper; FP32-split path only).
 * Each template t (PD_FIELD_GRAIN_TEMPLATE) has a basis Phi_t of n_modes
 * vectors over its n_t nodes in the lattice frame of the template.  A grain is
 * followed in its co-rotated frame (centroid and best-fit rotation of the
 * current positions onto the reference ones); its deformation w gives modal
 * coefficients q = Phi^T w / h, a network (pd_mlp) maps q to the modal bond
 * force f = Phi^T F_bond / (E h), and the force kernel uses R Phi f E h in place
 * of the bond loop for active grains.  Both basis products run per template
 * as GEMMs over all of its active grains on the tensor cores (BF16 hi/lo
 * split operands, FP32 accumulation).  Every judge_every steps the full bond
 * kernel runs instead; a grain whose largest |s| exceeds gate * s0, or whose
 * surrogate bond force differs from the full one by more than err_tol
 * (relative, floored at the grain's weight), leaves the surrogate for good.
 * Bonds of a surrogate grain do not break between judge steps.
 */
/*
 * The modal basis of every template (host; after pd_build_bonds, before or
 * after pd_bind_arena; one material only): the n_modes softest non-rigid
 * eigenvectors of the template's linearised bond operator K / E, and their
 * eigenvalues, in the layout pd_surrogate_setup takes.  Linearising the bond
 * force of eq:pmb about the reference lattice, a bond of lattice offset d with
 * micromodulus c_w w (Table 1, the library's own constants) adds the
 * stiffness k = c_w w V^2 / (E h |d|) e e^T (e = d / |d|, V = h^2) to the
 * diagonal 2 x 2 blocks of its node and subtracts it from the block coupling
 * the two nodes, so that F / (E h) = -(K / E) u / h.  The three zero modes
 * (rigid motions) are skipped; vectors are orthonormal over the template's 2 n_t
 * unknowns (sign, and the basis of a repeated eigenvalue, are arbitrary).
 *   basis     float[*basis_len]: per template t, per node l of the template
 *             (meshing order), n_modes x-components then n_modes y-components;
 *             NULL: write the required length sum_t 2 n_t n_modes to *basis_len
 *   lambda    float[n_templates n_modes] eigenvalues, ascending per template
 *   rigid     double[3 n_templates] (nullable): the three lowest eigenvalues
 *             (zero up to round-off)
 * Method: Chebyshev-filtered subspace iteration on the sparse operator (dense
 * Jacobi below 400 unknowns).  Errors: PD_ESTATE (before pd_build_bonds),
 * PD_EINVAL (sizes, several materials), PD_ENUMERIC (no convergence).
 */
int pd_surrogate_basis(pd_ctx *ctx, int n_modes, float *basis, size_t *basis_len, float *lambda, double *rigid);

/* Before pd_bind_arena.  n_modes: 8, 16, 24 or 32.  basis: for t = 0, 1, ...
 * the template's nodes in meshing order, per node n_modes x-components then
 * n_modes y-components (copied; the library keeps its own layouts);
 * lambda: per template the n_modes eigenvalues of the dimensionless
 * linearised bond operator K / E (F / (E h) = -(K / E) w / h) for those modes.
 * The modal force is f = -lambda q + net(q): the network learns the nonlinear
 * correction (and is optional -- without one, no grain is active). */
int pd_surrogate_setup(pd_ctx *ctx, int n_modes, const float *basis, const float *lambda, int judge_every,
                       double gate, double err_tol);
/* Network of template t (its max_batch >= grains of the template); NULL
 * removes it and its grains leave the surrogate.  The network must stay alive
 * while the context may step.  A network takes the 32 modal coefficients of a
 * grain: PD_EINVAL unless pd_surrogate_setup was given n_modes = 32. */
int pd_surrogate_set_mlp(pd_ctx *ctx, int tmpl, pd_mlp *mlp);
/* on = 1: every grain of a template with a network becomes active; 0: off. */
int pd_surrogate_enable(pd_ctx *ctx, int on);
/* Training pairs at the current state (needs store_parts): per grain the modal
 * coefficients q and the modal FULL bond force f, host float[G][n_modes] each
 * (grains without a template: untouched).  Bonds may break, as in pd_eval_forces. */
int pd_surrogate_sample(pd_ctx *ctx, float *q_host, float *f_host);
/* Per grain (host, nullable): active flag, last judged relative error of the
 * nodal bond force (the fallback criterion), last judged relative error of the
 * modal bond force f (what the network predicts; floored likewise), last
 * judged max |s| / s0. */
int pd_surrogate_stats(pd_ctx *ctx, int32_t *active_host, float *err_host, float *merr_host, float *maxs_host);
/* The surrogate phases at the current state, as pd_eval_forces (which this
 * runs; with store_parts the bond part of PD_FIELD_FORCE_PARTS then holds the
 * surrogate force of active grains unless the step is a judge step): per grain
 * the network input q and the modal force f = -lambda q + net(q), host
 * float[G][n_modes] each (zero rows for grains without a template).  Needs the
 * surrogate enabled; waits. */
int pd_surrogate_inspect(pd_ctx *ctx, float *q_host, float *y_host);

/* ---- observables of the settling and compaction sections (Sec. 6) ---------- */
#define PD_OBS_PHI 0            /* volume fraction: particle volume / container area      */
#define PD_OBS_BULK_DAMAGE 1    /* bulk damage: mean particle damage of the aggregate     */
#define PD_OBS_FORCE_TOP 2      /* y force the aggregate exerts on its top wall (y_hi)    */
#define PD_OBS_FORCE_BOTTOM 3   /* y force the aggregate exerts on its bottom wall (y_lo) */
#define PD_OBS_COUNT 4

/*
 * Per aggregate a, out[PD_OBS_COUNT * a + PD_OBS_*] (host, n_agg x 4 doubles)
 * at the current state and time t = step dt.  Volume fraction phi(t) = sum of
 * the node volumes / ((x_hi - x_lo)(y_hi - y_lo)) with the walls at time t
 * (the compaction section's sum V_i / (l (h - v t))).  Particle damage is the
 * mean over a grain's nodes of the node damage (broken / reference bonds,
 * Sec. 3.1); bulk damage is the mean particle damage over the aggregate's
 * grains.  The force on a wall is minus the sum over nodes of that wall's
 * force on them (eq:wall-total): its own segment term less half of each
 * corner term it shares with a neighbouring wall.  Runs on the caller's stream
 * and waits.  Errors: PD_ESTATE, PD_EINVAL, PD_ECUDA.
 */
int pd_observables(pd_ctx *ctx, double *out_host);

/*
 * Check of the FP64 path's square root (no counterpart in the paper).  The
 * plain FP64 bond loop takes L = sqrt(|d|^2) from integer and FP32 arithmetic
 * instead of GB300's 2-lane FP64 pipe and relies on it being the correctly
 * rounded IEEE value, as the FP64 definition of the stretch (eq:pmb) is.  This
 * call compares it with the hardware's IEEE square root on n pseudo-random
 * positive doubles (splitmix64 of seed; magnitudes 2^-80 .. 2^20) on the given
 * stream, waits, and writes the number of differing results to *mismatches and
 * the first differing input to *first_mismatch (nullable; unchanged when there
 * is none).  Allocates 16 bytes of device memory for the count.
 * Errors: PD_EINVAL (n < 0, null mismatches), PD_ECUDA.
 */
int pd_check_sqrt(long long n, unsigned long long seed, void *cuda_stream, long long *mismatches,
                  double *first_mismatch);

/* ---- diagnostics without device allocation ---------------------------------- */
#define PD_NOALLOC_MAX_NODES 2097152

/*
 * The reductions of pd_diagnostics for callers that cannot allocate device
 * memory (their device memory comes from a fixed budget or another runtime,
 * or an allocation would synchronise the device inside their loop).  The
 * paper has no counterpart: this is a deployment variant of the diagnostics
 * kernel whose scratch (per-block partial sums, 64 KiB) is a fixed device
 * array inside the library, held by every GPU that loads the library until
 * the process exits.  The call allocates nothing.
 *   n_nodes   N, 0 <= N <= PD_NOALLOC_MAX_NODES (larger: PD_EINVAL)
 *   X, u, v   device double[2N] reference positions, displacements, velocities
 *   V         device double[N] nodal volumes;  grain device int32[N]
 *   row_ptr   device int32[N+1], col device int32[n_bonds] (bond lists as
 *             PD_FIELD_ROW_PTR / PD_FIELD_COL), broken device uint8[n_bonds]
 *   g_cw, g_eps  device double[G] per-grain c_w and horizon
 *   rho, micromodulus as in pd_params (one density for every node: with
 *             per-grain materials, pd_diagnostics weighs each node by its own)
 *   out       device double[PD_DIAG_COUNT] (same slots as pd_diagnostics;
 *             PD_DIAG_ECONTACT and PD_DIAG_EWALL, which need the context's
 *             contact lists and walls, are written as 0)
 *   cuda_stream  the stream the work is enqueued on (returns without waiting)
 * The first call on a device, with that device current, looks up the device
 * address of the scratch array; make that first call before any stream
 * capture.  All calls share the scratch: calls that overlap on the GPU (on
 * different streams, or concurrently from several threads) race.  Nothing
 * needs clearing between calls: each call overwrites every partial it reads.
 * Errors: PD_EINVAL (size, null pointer), PD_ECUDA.
 */
int pd_diagnostics_noalloc(int n_nodes, const double *X, const double *u, const double *v, const double *V,
                           const int32_t *grain, const int32_t *row_ptr, const int32_t *col,
                           const uint8_t *broken, const double *g_cw, const double *g_eps, double rho,
                           int micromodulus, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PERIDEM_H */
