// pd_host.cpp -- host runtime of the GB300 PeriDEM library: the C ABI of
// include/peridem.h, the lattice mesher, the reference bond builder of the
// paper's non-convex rule, arena layout, uploads and the captured step graphs.
#include "peridem.h"
#include "pd_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMeshClear = 1e-6;   // nodes closer than this * h to the boundary are dropped
constexpr double kExtend = 1e-7;      // extended-boundary offset delta, in units of h
constexpr int kChunk = 16;            // time steps per captured chunk graph

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define PD_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

struct Vec2 {
    double x, y;
};
inline Vec2 sub(Vec2 a, Vec2 b) { return {a.x - b.x, a.y - b.y}; }
inline double crs(Vec2 a, Vec2 b) { return a.x * b.y - a.y * b.x; }
inline double nrm(Vec2 a) { return std::sqrt(a.x * a.x + a.y * a.y); }
inline Vec2 unit(Vec2 a) {
    double l = nrm(a);
    return {a.x / l, a.y / l};
}

// A grain outline in its own frame, physical units.
struct Outline {
    std::vector<std::vector<Vec2>> loops;
};

// --- lattice mesher -------------------------------------------------------

// Winding number of the region bounded by all loops around q (outer loop
// counter-clockwise, holes clockwise): nonzero inside the material.
int winding(const Outline &o, Vec2 q) {
    int wn = 0;
    for (const auto &lp : o.loops) {
        size_t n = lp.size();
        for (size_t k = 0; k < n; ++k) {
            Vec2 a = lp[k], b = lp[(k + 1) % n];
            double side = crs(sub(b, a), sub(q, a));
            if (a.y <= q.y) {
                if (b.y > q.y && side > 0) ++wn;
            } else {
                if (b.y <= q.y && side < 0) --wn;
            }
        }
    }
    return wn;
}

double seg_dist(Vec2 q, Vec2 a, Vec2 b) {
    Vec2 e = sub(b, a);
    double l2 = e.x * e.x + e.y * e.y;
    double t = l2 > 0 ? ((q.x - a.x) * e.x + (q.y - a.y) * e.y) / l2 : 0.0;
    t = std::min(1.0, std::max(0.0, t));
    double dx = a.x + t * e.x - q.x, dy = a.y + t * e.y - q.y;
    return std::sqrt(dx * dx + dy * dy);
}

double boundary_dist(const Outline &o, Vec2 q) {
    double best = 1e300;
    for (const auto &lp : o.loops)
        for (size_t k = 0; k < lp.size(); ++k) best = std::min(best, seg_dist(q, lp[k], lp[(k + 1) % lp.size()]));
    return best;
}

// --- paper's non-convex horizon construction ------------------------------

struct Seg {
    Vec2 a, b;
};

// Closed segment intersection by orientation tests.
bool on_seg(Vec2 a, Vec2 b, Vec2 q) {
    return std::min(a.x, b.x) <= q.x && q.x <= std::max(a.x, b.x) && std::min(a.y, b.y) <= q.y &&
           q.y <= std::max(a.y, b.y);
}
bool segs_meet(Vec2 a, Vec2 b, Vec2 c, Vec2 d) {
    double d1 = crs(sub(d, c), sub(a, c)), d2 = crs(sub(d, c), sub(b, c));
    double d3 = crs(sub(b, a), sub(c, a)), d4 = crs(sub(b, a), sub(d, a));
    if (((d1 > 0 && d2 < 0) || (d1 < 0 && d2 > 0)) && ((d3 > 0 && d4 < 0) || (d3 < 0 && d4 > 0))) return true;
    if (d1 == 0 && on_seg(c, d, a)) return true;
    if (d2 == 0 && on_seg(c, d, b)) return true;
    if (d3 == 0 && on_seg(a, b, c)) return true;
    if (d4 == 0 && on_seg(a, b, d)) return true;
    return false;
}

// Barriers of one grain (Sec. 4): the extended boundary (every vertex p^i
// moved by delta along its outward normal n_i, the bisector of the outer angle)
// and, at each non-convex cusp, the bisector segment from p^i + delta n_i to
// q^i - delta n_i, where the ray p^i + t n_i meets the boundary again (or, with
// no hit, to t0 = |p^i| + sup |x|).  A bond is dropped when it meets any barrier.
std::vector<Seg> barriers(const Outline &o, double delta) {
    std::vector<Seg> out;
    double sup = 0;
    for (const auto &lp : o.loops)
        for (auto v : lp) sup = std::max(sup, nrm(v));
    for (const auto &lp : o.loops) {
        size_t n = lp.size();
        std::vector<Vec2> ext(n), nrmv(n);
        std::vector<char> cusp(n, 0);
        for (size_t i = 0; i < n; ++i) {
            Vec2 p = lp[i], pm = lp[(i + n - 1) % n], pp = lp[(i + 1) % n];
            Vec2 vm = unit(sub(p, pm)), vi = unit(sub(pp, p));
            double c = crs(vm, vi);
            Vec2 nn;
            if (c > 0) {
                nn = unit(Vec2{vm.x - vi.x, vm.y - vi.y});          // convex corner
            } else if (c < 0) {
                nn = unit(Vec2{vi.x - vm.x, vi.y - vm.y});          // non-convex cusp
                cusp[i] = 1;
            } else {
                nn = Vec2{vi.y, -vi.x};                               // straight: edge normal
            }
            nrmv[i] = nn;
            ext[i] = Vec2{p.x + delta * nn.x, p.y + delta * nn.y};
        }
        for (size_t i = 0; i < n; ++i) out.push_back(Seg{ext[i], ext[(i + 1) % n]});
        for (size_t i = 0; i < n; ++i) {
            if (!cusp[i]) continue;
            Vec2 p = lp[i], nn = nrmv[i];
            double tbest = 1e300;
            for (const auto &lq : o.loops) {
                size_t m = lq.size();
                for (size_t k = 0; k < m; ++k) {
                    Vec2 c = lq[k], d = lq[(k + 1) % m];
                    Vec2 s = sub(d, c);
                    double den = crs(nn, s);
                    if (den == 0) continue;
                    Vec2 w = sub(c, p);
                    double t = crs(w, s) / den, u = crs(w, nn) / den;
                    // tolerant end test: a ray through a vertex must not slip between
                    // the two edges that share it
                    if (t > delta && u >= -1e-9 && u <= 1.0 + 1e-9) tbest = std::min(tbest, t);
                }
            }
            // the bisector stops delta short of q^i, as it starts delta away from p^i:
            // a bond that merely touches the boundary at either end point stays
            double tend = (tbest == 1e300) ? nrm(p) + sup : tbest - delta;
            out.push_back(Seg{Vec2{p.x + delta * nn.x, p.y + delta * nn.y}, Vec2{p.x + tend * nn.x, p.y + tend * nn.y}});
        }
    }
    return out;
}

}  // namespace

// ---------------------------------------------------------------------------

struct pd_ctx {
    pd_params prm{};
    cudaStream_t stream = nullptr;
    int state = 0;  // 0 created, 1 meshed, 2 bonded, 3 bound
    // mesh (host)
    int G = 0;
    int64_t N = 0;
    std::vector<double> X;     // 2N
    std::vector<int32_t> lat;  // 2N
    std::vector<int32_t> grain;
    std::vector<double> V, v0;  // N, 2N
    std::vector<double> g_h, g_cw, g_s0, g_eps, g_cx, g_cy, g_R;
    // materials (pd_set_materials): per grain density and bulk modulus
    std::vector<double> g_rho, g_k;
    bool has_mat = false;
    std::vector<int64_t> g_start;
    std::vector<Outline> g_outline;  // per grain, local frame, physical units
    // bonds (host)
    std::vector<int32_t> row_ptr, col;
    std::vector<double> xi;
    int max_row = 0, wpn = 1;
    size_t stn_irregular = 0;   // FP32 split: nodes whose bonds do not follow the lattice stencil
    // derived
    double h_min = 0, Rc = 0, Kn = 0;   // of aggregate 0 (reported by pd_info)
    unsigned T = 0;
    // aggregates: independent wall boxes (one by default)
    int n_agg = 1;
    std::vector<int32_t> g_agg;          // per grain
    std::vector<double> agg_walls;       // 8 per aggregate: x_lo, x_hi, y_lo, y_hi, v(x_lo), v(x_hi), v(y_lo), v(y_hi)
    std::vector<pd::AggParams> aggp;
    // step path: 0 = graph of separate kernels, 1 = persistent cooperative kernel
    int mode = 2, block = 128;
    pd::KParams kp{};
    pd::DevPtrs d{};
    size_t arena_bytes = 0;
    int vcur = 0;
    int64_t steps_done = 0;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t body_stream = nullptr;    // captures the bodies of the rebuild conditionals
    cudaStream_t sur_stream = nullptr;     // captures the surrogate chain beside the lane sums
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    cudaGraphExec_t single[2] = {nullptr, nullptr};
    cudaGraphExec_t timed[2] = {nullptr, nullptr};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int timing = 0;
    // learned modal surrogate
    std::vector<int32_t> g_shape, g_tmpl, g_slot, tmpl_first, tmpl_count, tmpl_nodes;
    std::vector<double> g_theta;
    int n_tmpl = 0;
    bool sur_cfg = false;
    int sur_modes = 32, sur_judge = 50;
    double sur_gate = 0.5, sur_tol = 1e-3;
    std::vector<float> sur_basis, sur_lambda;   // basis: per template mode-major, padded rows
    std::vector<uint16_t> bnm_hi, bnm_lo, bmm_hi, bmm_lo;
    std::vector<int32_t> tmpl_rows, slot_grain;
    std::vector<int4> proj_work, exp_work, mlp_work;
    std::vector<pd_mlp *> sur_mlp;
};

namespace {

constexpr double kPiAgg = 3.14159265358979323846;

// Per-aggregate contact constants (Sec. 4.1): R_c = rc_ratio h_min and
// K_n = 18 k / (pi eps_c^5) with eps_c = horizon_ratio h_min, h_min the
// smallest lattice spacing of the aggregate's grains; hash grid anchored at
// the aggregate's lower-left wall corner with cells of side R_c.
void compute_aggregates(pd_ctx *c) {
    const pd_params &p = c->prm;
    c->aggp.assign(c->n_agg, pd::AggParams{});
    std::vector<double> hmin(c->n_agg, 1e300);
    for (int g = 0; g < c->G; ++g) hmin[c->g_agg[g]] = std::min(hmin[c->g_agg[g]], c->g_h[g]);
    for (int a = 0; a < c->n_agg; ++a) {
        pd::AggParams &A = c->aggp[a];
        double h = hmin[a] < 1e300 ? hmin[a] : c->g_h[0];
        double eps_c = p.horizon_ratio * h;
        A.Rc = p.rc_ratio * h;
        A.pe5 = kPiAgg * eps_c * eps_c * eps_c * eps_c * eps_c;
        A.Kn = 18.0 * p.k_bulk / A.pe5;
        const double *w = &c->agg_walls[8 * (size_t)a];
        A.w0[0] = w[0]; A.w0[1] = w[1]; A.w0[2] = w[2]; A.w0[3] = w[3];
        A.wv[0] = w[4]; A.wv[1] = w[5]; A.wv[2] = w[6]; A.wv[3] = w[7];
        A.ox = w[0];
        A.oy = w[2];
        // candidate lists of radius R_c + skin: a hair above it, two nodes closer
        // than R_c + skin never land two cells apart (FP32 split: 0.4 % above,
        // the margin of its float cell coordinates)
        const double skin = pd::kSkinRatio * A.Rc;
        A.cell = (A.Rc + skin) * (p.precision == PD_FP32_SPLIT ? 1.004 : 1.0 + 1e-9);
        A.rs2 = (float)((A.Rc + skin) * (A.Rc + skin));
        A.dmax2 = (float)(pd::kSkinTrigger * skin * pd::kSkinTrigger * skin);
        A.inv_cell = 1.0 / A.cell;
        // FP32 split: shift coordinates of the box into [L, 2L) so nearby
        // positions share a binade and their float differences are exact
        double Lx = std::max(w[1] - w[0], 1e-6), Ly = std::max(w[3] - w[2], 1e-6);
        A.sx = Lx - w[0];
        A.sy = Ly - w[2];
        double rc2 = A.Rc * A.Rc;
        A.rc2_hi = (float)rc2;
        A.rc2_lo = (float)(rc2 - (double)A.rc2_hi);
        A.rcf = (float)A.Rc;
        A.knf = (float)A.Kn;
        A.oxs = (float)(A.ox + A.sx);
        A.oys = (float)(A.oy + A.sy);
        A.inv_cell_f = (float)A.inv_cell;
    }
    c->h_min = hmin[0] < 1e300 ? hmin[0] : c->g_h[0];
    c->Rc = c->aggp[0].Rc;
    c->Kn = c->aggp[0].Kn;
}

}  // namespace

namespace {

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// BF16 (round to nearest even) of a finite float, and back.
uint16_t to_bf16(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float from_bf16(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
}

// v = hi + lo to about 2^-17 relative, both BF16.
void bf16_split(float v, uint16_t &hi, uint16_t &lo) {
    hi = to_bf16(v);
    lo = to_bf16(v - from_bf16(hi));
}

// Largest number of projection chunks of any template.
int sur_max_chunks(const pd_ctx *c) {
    int mx = 0;
    for (size_t t = 0; t + 1 < c->tmpl_rows.size(); ++t)
        mx = std::max(mx, (c->tmpl_rows[t + 1] - c->tmpl_rows[t]) / pd::kSurChunk);
    return mx;
}

template <class T>
void carve(char *base, size_t &off, T *&ptr, size_t count) {
    ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off = align_up(off + sizeof(T) * std::max<size_t>(count, 1));
}

size_t layout(pd_ctx *c, char *base) {
    size_t off = 0;
    pd::DevPtrs &d = c->d;
    size_t N = (size_t)c->N, nb = c->col.size(), G = (size_t)c->G;
    const bool fp32 = c->prm.precision == PD_FP32_SPLIT;
    carve(base, off, d.X, N);
    carve(base, off, d.ub[0], N);
    carve(base, off, d.ub[1], fp32 ? N : 0);
    if (!fp32) d.ub[1] = d.ub[0];
    carve(base, off, d.v[0], N);
    carve(base, off, d.v[1], N);
    carve(base, off, d.a, fp32 ? 0 : N);
    carve(base, off, d.af, fp32 ? N : 0);
    if (fp32) d.a = nullptr;
    else d.af = nullptr;
    carve(base, off, d.p, N);
    carve(base, off, d.F, c->prm.store_parts ? N : 0);
    carve(base, off, d.parts, c->prm.store_parts ? 4 * N : 0);
    carve(base, off, d.V, N);
    carve(base, off, d.grain, N);
    carve(base, off, d.row_ptr, N + 1);
    carve(base, off, d.col, nb);
    carve(base, off, d.xi, nb);
    carve(base, off, d.bits, N * (size_t)c->wpn);
    carve(base, off, d.g_cw, G);
    carve(base, off, d.g_s0, G);
    carve(base, off, d.g_eps, G);
    carve(base, off, d.g_agg, G);
    carve(base, off, d.g_rho, G);
    carve(base, off, d.g_k, G);
    carve(base, off, d.g_kf, G);
    carve(base, off, d.agg, (size_t)c->n_agg);
    carve(base, off, d.key, N);
    carve(base, off, d.cell, N);
    carve(base, off, d.wall_cell, (size_t)c->n_agg);
    carve(base, off, d.count, c->T);
    carve(base, off, d.start, (size_t)c->T + 1);
    carve(base, off, d.cursor, c->T);
    carve(base, off, d.sorted, N);
    carve(base, off, d.srec, N);
    carve(base, off, d.nbr_cnt, N);
    carve(base, off, d.nbr, N * (size_t)pd::kMaxList);
    carve(base, off, d.sref, N);
    carve(base, off, d.rebuild, 1);
    carve(base, off, d.pred_done, 1);
    carve(base, off, d.rebuild_next, 1);
    carve(base, off, d.pred_ok, 1);
    carve(base, off, d.fsum, 6 * N * (c->prm.precision == PD_FP32_SPLIT ? 4 : 8));
    // block sums of the scan: one per scan tile (multi-kernel path) or per
    // block of the persistent kernel (at most 16 blocks per SM)
    carve(base, off, d.blocksums, std::max<size_t>(c->T / pd::kScanTile + 2, 16 * 1024));
    carve(base, off, d.step, 1);
    carve(base, off, d.t_now, 1);
    carve(base, off, d.bar, 2);
    carve(base, off, d.status, PD_STATUS_COUNT);
    carve(base, off, d.diag_part, (size_t)c->kp.n_diag_blocks * PD_DIAG_COUNT);
    carve(base, off, d.diag_out, PD_DIAG_COUNT);
    carve(base, off, d.g_start, G + 1);
    carve(base, off, d.obs_gdam, G);
    carve(base, off, d.obs_wall, 16 * (size_t)c->n_agg);
    if (c->prm.precision == PD_FP32_SPLIT) {
        carve(base, off, d.lat, N);
        carve(base, off, d.gq, G);
        carve(base, off, d.pqb[0], N);
        carve(base, off, d.pqb[1], N);
        carve(base, off, d.xs, N);
        carve(base, off, d.colx, nb);
        carve(base, off, d.stn, N);
        carve(base, off, d.gc, G);
    } else {
        d.lat = nullptr;
        d.gq = nullptr;
        d.pqb[0] = d.pqb[1] = nullptr;
        d.xs = nullptr;
        d.colx = nullptr;
        d.stn = nullptr;
        d.gc = nullptr;
    }
    carve(base, off, d.g_invm, G);
    carve(base, off, d.g_invmf, G);
    carve(base, off, d.bu, N);
    carve(base, off, d.bv, N);
    carve(base, off, d.ba, N);
    carve(base, off, d.bbits, N * (size_t)c->wpn);
    if (c->sur_cfg) {
        const size_t M = (size_t)c->sur_modes, T = (size_t)c->n_tmpl;
        carve(base, off, d.g_tmpl, G);
        carve(base, off, d.g_slot, G);
        carve(base, off, d.tmpl_node, T + 1);
        carve(base, off, d.tmpl_slot, T + 1);
        carve(base, off, d.basis, c->sur_basis.size());
        carve(base, off, d.bnm_hi, c->bnm_hi.size());
        carve(base, off, d.bnm_lo, c->bnm_lo.size());
        carve(base, off, d.bmm_hi, c->bmm_hi.size());
        carve(base, off, d.bmm_lo, c->bmm_lo.size());
        carve(base, off, d.tmpl_rows, T + 1);
        carve(base, off, d.slot_grain, G);
        carve(base, off, d.proj_work, c->proj_work.size());
        carve(base, off, d.exp_work, c->exp_work.size());
        carve(base, off, d.sur_w, N);
        carve(base, off, d.sur_f, N);
        carve(base, off, d.sur_xpart, (size_t)(c->tmpl_rows.empty() ? 0 : sur_max_chunks(c)) * G * M);
        carve(base, off, d.sur_merr, G);
        carve(base, off, d.mlp_refs, T);
        carve(base, off, d.mlp_work, (G + pd::kSurTile - 1) / pd::kSurTile + T);
        carve(base, off, d.mlp_err, 1);
        carve(base, off, d.sur_lambda, T * M);
        carve(base, off, d.g_theta, G);
        carve(base, off, d.sur_fc, G);
        carve(base, off, d.sur_active, G);
        carve(base, off, d.sur_rot, G);
        carve(base, off, d.sur_x, G * M);
        carve(base, off, d.sur_y, G * M);
        carve(base, off, d.sur_fb, N);
        carve(base, off, d.sur_err, G);
        carve(base, off, d.sur_maxs, G);
        carve(base, off, d.sur_qs, G * M);
        carve(base, off, d.sur_fs, G * M);
    } else {
        d.g_tmpl = d.g_slot = d.tmpl_node = d.tmpl_slot = d.sur_active = nullptr;
        d.tmpl_rows = d.slot_grain = nullptr;
        d.bnm_hi = d.bnm_lo = d.bmm_hi = d.bmm_lo = nullptr;
        d.proj_work = d.exp_work = nullptr;
        d.sur_w = d.sur_f = nullptr;
        d.sur_xpart = d.sur_merr = nullptr;
        d.mlp_refs = nullptr;
        d.mlp_work = nullptr;
        d.mlp_err = nullptr;
        d.basis = d.sur_x = d.sur_y = d.sur_err = d.sur_maxs = d.sur_qs = d.sur_fs = d.sur_lambda = nullptr;
        d.g_theta = nullptr;
        d.sur_fc = nullptr;
        d.sur_rot = d.sur_fb = nullptr;
    }
    d.u = d.ub[c->vcur];
    d.pq = d.pqb[c->vcur];
    return off;
}

int check_ctx(pd_ctx *c, int min_state) {
    if (!c) return fail(PD_EINVAL, "null context");
    if (c->state < min_state) return fail(PD_ESTATE, "call out of order");
    return PD_OK;
}

// Surrogate phases before the force kernel: co-rotated local deformation of
// the active grains, its projection on the basis (tensor cores), the chunk
// partials summed in a fixed order, every template's network on its batch of
// grains with f = -Lambda q + net(q) in its output epilogue, and the
// expansion of f to nodal bond forces (tensor cores).
// The host-side current displacement and positions follow the velocity parity.
void set_current(pd_ctx *c) {
    c->d.u = c->d.ub[c->vcur];
    c->d.pq = c->d.pqb[c->vcur];
}

// Device pointers for the kernels of a step recorded with velocity parity vin:
// its displacement update writes, and its force phase reads, the displacement
// and positions of parity vin ^ 1.
pd::DevPtrs step_ptrs(const pd_ctx *c, int vin) {
    pd::DevPtrs d = c->d;
    d.u = d.ub[vin ^ 1];
    d.pq = d.pqb[vin ^ 1];
    return d;
}

cudaError_t record_surrogate(pd_ctx *c, const pd::DevPtrs &d, cudaStream_t s) {
    cudaError_t e;
    // the kernels after the frame begin while their predecessor finishes
    // (programmatic dependent launch) and stage their basis or weight operands
    if ((e = pd::launch_sur_frame(d, c->kp, 0, s)) != cudaSuccess) return e;
    if ((e = pd::launch_sur_project_tc(d, c->kp, s, true)) != cudaSuccess) return e;
    if ((e = pd::launch_sur_reduce(d, c->kp, s, true)) != cudaSuccess) return e;
    if ((e = pd::launch_mlp_grouped(d.mlp_refs, d.mlp_work, (int)c->mlp_work.size(), d.sur_x, d.sur_y, d.mlp_err, s,
                                    true)) != cudaSuccess)
        return e;
    return pd::launch_sur_expand_tc(d, c->kp, s, true);
}

// Record one time step (Algorithm 1) on the capturing stream s: displacement
// update and positions, the rebuild of the contact candidate lists as the
// body of a conditional node (run only when the displacement update raised
// the rebuild flag), forces + acceleration + velocity update.  With `timed`,
// event records bracket the three kernel groups.
cudaError_t record_step(pd_ctx *c, int vin, cudaStream_t s, bool timed = false) {
    cudaError_t e;
    const pd::DevPtrs dv = step_ptrs(c, vin);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g)) != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureUnmatched;
    const int use_cond = (c->mode & 4) ? 0 : 1;
    cudaGraphConditionalHandle cond = 0;
    if (use_cond && (e = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = pd::launch_predict(dv, c->kp, vin, 1, s, cond, use_cond)) != cudaSuccess) return e;
    // surrogate with the split force phase: its chain (frame, projection,
    // networks, expansion) runs on a second stream beside the rebuild and the
    // lane sums, which skip the bond loop of surrogate grains; the epilogue,
    // which adds the surrogate forces, waits for it
    const bool fork = c->kp.sur && c->kp.split;
    if (fork) {
        if ((e = cudaEventRecord(c->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->sur_stream, c->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = record_surrogate(c, dv, c->sur_stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->ev_join, c->sur_stream)) != cudaSuccess) return e;
    }
    if (timed && (e = cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (c->mode & 4) {
        // path modes 4-7: the rebuild kernels run every step and return at once
        // when the flag is clear (no conditional node)
        if ((e = pd::launch_rebuild(dv, c->kp, s)) != cudaSuccess) return e;
    } else {
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return e;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)) != cudaSuccess) return e;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return e;
        const cudaError_t eb = pd::launch_rebuild(dv, c->kp, c->body_stream);
        cudaGraph_t done = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->body_stream, &done);
        if (eb != cudaSuccess) return eb;
        if (ee != cudaSuccess) return ee;
    }
    if (c->kp.sur && !fork && (e = record_surrogate(c, dv, s)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (fork) {
        if ((e = pd::launch_force(dv, c->kp, vin, 1, s, 1)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, c->ev_join, 0)) != cudaSuccess) return e;
        if ((e = pd::launch_force(dv, c->kp, vin, 1, s, 2)) != cudaSuccess) return e;
    } else if ((e = pd::launch_force(dv, c->kp, vin, 1, s)) != cudaSuccess) {
        return e;
    }
    if (c->kp.sur && (e = pd::launch_sur_judge(dv, c->kp, s)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    return cudaSuccess;
}

// nsteps time steps as one persistent cooperative launch; timing brackets the
// whole launch as the force group.
cudaError_t record_persistent(pd_ctx *c, int vin, int nsteps, cudaStream_t s, bool timed = false) {
    cudaError_t e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = pd::launch_persistent(c->d, c->kp, vin, nsteps, c->block, s)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal)) != cudaSuccess) return e;
    return cudaSuccess;
}

int capture(pd_ctx *c, int vstart, int nsteps, cudaGraphExec_t *out, bool timed = false) {
    cudaGraph_t g = nullptr;
    PD_CUDA(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    int v = vstart;
    cudaError_t e = cudaSuccess;
    if ((c->mode & 1) && !c->kp.sur) {
        e = record_persistent(c, v, nsteps, c->capture_stream, timed);
    } else {
        for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
            e = record_step(c, v, c->capture_stream, timed);
            v ^= 1;
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &g);
    if (e != cudaSuccess) return fail(PD_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(PD_ECUDA, std::string("end capture: ") + cudaGetErrorString(e2));
    PD_CUDA(cudaGraphInstantiate(out, g, 0));
    cudaGraphDestroy(g);
    return PD_OK;
}

int capture_all(pd_ctx *c) {
    for (int v = 0; v < 2; ++v) {
        for (cudaGraphExec_t *g : {&c->chunk[v], &c->single[v], &c->timed[v]})
            if (*g) {
                cudaGraphExecDestroy(*g);
                *g = nullptr;
            }
        if (int r = capture(c, v, kChunk, &c->chunk[v])) return r;
        if (int r = capture(c, v, 1, &c->single[v])) return r;
        if (int r = capture(c, v, 1, &c->timed[v], true)) return r;
    }
    return PD_OK;
}

size_t field_bytes(pd_ctx *c, int f) {
    size_t N = (size_t)c->N;
    switch (f) {
        case PD_FIELD_X: case PD_FIELD_DISP: case PD_FIELD_VEL: case PD_FIELD_ACC: case PD_FIELD_POS:
        case PD_FIELD_FORCE:
            return 16 * N;
        case PD_FIELD_FORCE_PARTS: return 64 * N;
        case PD_FIELD_BROKEN: return c->col.size();
        case PD_FIELD_DAMAGE: case PD_FIELD_VOLUME: return 8 * N;
        case PD_FIELD_GRAIN: return 4 * N;
        case PD_FIELD_ROW_PTR: return 4 * (N + 1);
        case PD_FIELD_COL: return 4 * c->col.size();
        case PD_FIELD_LATTICE: return 8 * N;
        case PD_FIELD_STEP: return 8;
        case PD_FIELD_GRAIN_TEMPLATE: return 4 * (size_t)c->G;
        default: return 0;
    }
}

}  // namespace

int pd::set_error(int code, const char *msg) { return fail(code, msg); }

// Template data for the modal basis of the surrogate (pd_basis.cpp).
namespace pd {
struct TemplateView {
    int n_tmpl;
    const int32_t *tmpl_first, *tmpl_nodes;
    const int64_t *g_start;
    const int32_t *lat, *row_ptr, *col;
    const double *g_cw, *g_eps, *g_h;
    double E, horizon_ratio;
    int micromodulus;
};
int template_view(pd_ctx *c, TemplateView *out) {
    if (!c || !out) return fail(PD_EINVAL, "null context");
    if (c->state < 2) return fail(PD_ESTATE, "the modal basis needs the bond lists (after pd_build_bonds)");
    if (c->has_mat) return fail(PD_EINVAL, "the surrogate runs with one material");
    out->n_tmpl = c->n_tmpl;
    out->tmpl_first = c->tmpl_first.data();
    out->tmpl_nodes = c->tmpl_nodes.data();
    out->g_start = c->g_start.data();
    out->lat = c->lat.data();
    out->row_ptr = c->row_ptr.data();
    out->col = c->col.data();
    out->g_cw = c->g_cw.data();
    out->g_eps = c->g_eps.data();
    out->g_h = c->g_h.data();
    out->E = c->prm.E;
    out->horizon_ratio = c->prm.horizon_ratio;
    out->micromodulus = c->prm.micromodulus;
    return PD_OK;
}
}  // namespace pd

// ===========================================================================
// C ABI

extern "C" {

const char *pd_last_error(void) { return g_err.c_str(); }

int pd_create(pd_ctx **out, const pd_params *params, void *cuda_stream) {
    if (!out || !params) return fail(PD_EINVAL, "null argument");
    const pd_params &p = *params;
    if (!(p.dt > 0) || !(p.rho > 0) || !(p.E > 0) || !(p.horizon_ratio > 0) || !(p.rc_ratio > 0) ||
        !(p.nu < 1) || !(p.Gc > 0) || !(p.k_bulk > 0))
        return fail(PD_EINVAL, "invalid parameters (dt, rho, E, Gc, k, horizon_ratio, rc_ratio must be > 0, nu < 1)");
    if (p.precision != PD_FP64 && p.precision != PD_FP32_SPLIT) return fail(PD_EINVAL, "unknown precision");
    if (p.micromodulus != PD_MICRO_CONSTANT && p.micromodulus != PD_MICRO_CONIC)
        return fail(PD_EINVAL, "unknown micromodulus");
    if (p.lanes != 0 && p.lanes != 1 && p.lanes != 2 && p.lanes != 4 && p.lanes != 8)
        return fail(PD_EINVAL, "lanes must be 0, 1, 2, 4 or 8");
    pd_ctx *c = new (std::nothrow) pd_ctx();
    if (!c) return fail(PD_ENOMEM, "out of host memory");
    c->prm = p;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return PD_OK;
}

int pd_destroy(pd_ctx *c) {
    if (!c) return PD_OK;
    if (c->state >= 3) {
        cudaStreamSynchronize(c->stream);
        for (int k = 0; k < 2; ++k) {
            if (c->chunk[k]) cudaGraphExecDestroy(c->chunk[k]);
            if (c->single[k]) cudaGraphExecDestroy(c->single[k]);
            if (c->timed[k]) cudaGraphExecDestroy(c->timed[k]);
        }
        for (auto &e : c->ev)
            if (e) cudaEventDestroy(e);
        if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
        if (c->body_stream) cudaStreamDestroy(c->body_stream);
        if (c->sur_stream) cudaStreamDestroy(c->sur_stream);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
    }
    delete c;
    return PD_OK;
}

int pd_mesh_grains(pd_ctx *c, int n_shapes, const int32_t *shape_loop_start, const int32_t *loop_vtx_start,
                   const double *vtx, int n_grains, const int32_t *grain_shape, const double *geom,
                   int64_t *n_nodes_out) {
    if (int r = check_ctx(c, 0)) return r;
    if (c->state != 0) return fail(PD_ESTATE, "pd_mesh_grains called twice");
    if (n_shapes <= 0 || n_grains <= 0 || !shape_loop_start || !loop_vtx_start || !vtx || !grain_shape || !geom)
        return fail(PD_EINVAL, "empty or null mesh input");
    for (int s = 0; s < n_shapes; ++s) {
        if (shape_loop_start[s + 1] <= shape_loop_start[s]) return fail(PD_EINVAL, "shape without loops");
        for (int l = shape_loop_start[s]; l < shape_loop_start[s + 1]; ++l)
            if (loop_vtx_start[l + 1] - loop_vtx_start[l] < 3) return fail(PD_EINVAL, "loop with < 3 vertices");
    }
    try {
        c->G = n_grains;
        c->g_h.resize(n_grains);
        c->g_cx.resize(n_grains);
        c->g_cy.resize(n_grains);
        c->g_R.resize(n_grains);
        c->g_outline.resize(n_grains);
        c->g_start.assign(n_grains + 1, 0);
        for (int g = 0; g < n_grains; ++g) {
            const double *q = geom + 7 * (size_t)g;
            double cx = q[0], cy = q[1], R = q[2], th = q[3], vx = q[4], vy = q[5], h = q[6];
            int s = grain_shape[g];
            if (s < 0 || s >= n_shapes) return fail(PD_EINVAL, "grain shape index out of range");
            if (!(R > 0) || !(h > 0) || !(R / h < 1e4)) return fail(PD_EINVAL, "grain radius / spacing invalid");
            Outline &o = c->g_outline[g];
            o.loops.clear();
            for (int l = shape_loop_start[s]; l < shape_loop_start[s + 1]; ++l) {
                std::vector<Vec2> lp;
                for (int k = loop_vtx_start[l]; k < loop_vtx_start[l + 1]; ++k)
                    lp.push_back(Vec2{R * vtx[2 * k], R * vtx[2 * k + 1]});
                o.loops.push_back(lp);
            }
            c->g_h[g] = h;
            c->g_shape.push_back(s);
            c->g_theta.push_back(th);
            c->g_cx[g] = cx;
            c->g_cy[g] = cy;
            c->g_R[g] = R;
            int m = (int)std::ceil(R / h) + 1;
            double cs = std::cos(th), sn = std::sin(th);
            for (int j = -m; j <= m; ++j) {
                for (int i = -m; i <= m; ++i) {
                    double lx = (double)i * h, ly = (double)j * h;
                    Vec2 ql{lx, ly};
                    if (winding(o, ql) == 0) continue;
                    if (boundary_dist(o, ql) < kMeshClear * h) continue;
                    c->X.push_back(cx + (cs * lx - sn * ly));
                    c->X.push_back(cy + (sn * lx + cs * ly));
                    c->lat.push_back(i);
                    c->lat.push_back(j);
                    c->grain.push_back(g);
                    c->V.push_back(h * h);
                    c->v0.push_back(vx);
                    c->v0.push_back(vy);
                }
            }
            c->g_start[g + 1] = (int64_t)c->grain.size();
        }
    } catch (const std::bad_alloc &) {
        return fail(PD_ENOMEM, "out of host memory while meshing");
    }
    c->N = (int64_t)c->grain.size();
    if (c->N == 0) return fail(PD_EINVAL, "no lattice node inside any grain");
    if (c->N >= (int64_t(1) << 31)) return fail(PD_EINVAL, "too many nodes for 32-bit indices");
    // material constants per grain (Table 1) and contact constants (Sec. 4.1)
    const pd_params &p = c->prm;
    c->g_cw.resize(c->G);
    c->g_s0.resize(c->G);
    c->g_eps.resize(c->G);
    c->h_min = *std::min_element(c->g_h.begin(), c->g_h.end());
    for (int g = 0; g < c->G; ++g) {
        double eps = p.horizon_ratio * c->g_h[g];
        c->g_eps[g] = eps;
        if (p.micromodulus == PD_MICRO_CONSTANT) {
            c->g_cw[g] = 6.0 * p.E / (kPi * eps * eps * eps * (1.0 - p.nu));
            c->g_s0[g] = std::sqrt(4.0 * kPi * p.Gc / (9.0 * p.E * eps));
        } else {
            c->g_cw[g] = 24.0 * p.E / (kPi * eps * eps * eps * (1.0 - p.nu));
            c->g_s0[g] = std::sqrt(5.0 * kPi * p.Gc / (9.0 * p.E * eps));
        }
    }
    c->g_rho.assign(c->G, p.rho);
    c->g_k.assign(c->G, p.k_bulk);
    c->has_mat = false;
    c->n_agg = 1;
    c->g_agg.assign(c->G, 0);
    c->agg_walls = {p.wall_lo[0], p.wall_hi[0], p.wall_lo[1], p.wall_hi[1],
                    p.wall_vel_lo[0], p.wall_vel_hi[0], p.wall_vel_lo[1], p.wall_vel_hi[1]};
    compute_aggregates(c);
    c->state = 1;
    if (n_nodes_out) *n_nodes_out = c->N;
    return PD_OK;
}

int pd_build_bonds(pd_ctx *c, int64_t *n_bonds_out) {
    if (int r = check_ctx(c, 1)) return r;
    if (c->state != 1) return fail(PD_ESTATE, "pd_build_bonds called twice");
    const double hr = c->prm.horizon_ratio;
    const int rr = (int)std::ceil(hr);
    std::vector<std::vector<int32_t>> g_row(c->G), g_col(c->G);
    auto work = [&](int g) {
        int64_t s0 = c->g_start[g], s1 = c->g_start[g + 1];
        int n = (int)(s1 - s0);
        double h = c->g_h[g];
        std::vector<Seg> bar = barriers(c->g_outline[g], kExtend * h);
        int imin = 1 << 30, imax = -(1 << 30), jmin = 1 << 30, jmax = -(1 << 30);
        for (int k = 0; k < n; ++k) {
            imin = std::min(imin, c->lat[2 * (s0 + k)]);
            imax = std::max(imax, c->lat[2 * (s0 + k)]);
            jmin = std::min(jmin, c->lat[2 * (s0 + k) + 1]);
            jmax = std::max(jmax, c->lat[2 * (s0 + k) + 1]);
        }
        int W = imax - imin + 1, H = jmax - jmin + 1;
        std::vector<int> map((size_t)W * H, -1);
        for (int k = 0; k < n; ++k)
            map[(size_t)(c->lat[2 * (s0 + k) + 1] - jmin) * W + (c->lat[2 * (s0 + k)] - imin)] = k;
        auto &row = g_row[g];
        auto &col = g_col[g];
        row.assign(n + 1, 0);
        std::vector<int> nb;
        for (int x = 0; x < n; ++x) {
            nb.clear();
            int ix = c->lat[2 * (s0 + x)], jx = c->lat[2 * (s0 + x) + 1];
            Vec2 a{(double)ix * h, (double)jx * h};
            for (int dj = -rr; dj <= rr; ++dj)
                for (int di = -rr; di <= rr; ++di) {
                    if ((di | dj) == 0 || (double)(di * di + dj * dj) >= hr * hr) continue;
                    int iy = ix + di, jy = jx + dj;
                    if (iy < imin || iy > imax || jy < jmin || jy > jmax) continue;
                    int y = map[(size_t)(jy - jmin) * W + (iy - imin)];
                    if (y < 0) continue;
                    Vec2 b{(double)iy * h, (double)jy * h};
                    bool cut = false;
                    for (const Seg &sg : bar)
                        if (segs_meet(a, b, sg.a, sg.b)) {
                            cut = true;
                            break;
                        }
                    if (!cut) nb.push_back(y);
                }
            std::sort(nb.begin(), nb.end());
            for (int y : nb) col.push_back((int32_t)(y + s0));
            row[x + 1] = (int32_t)col.size();
        }
    };
    try {
        unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                for (int g = (int)t; g < c->G; g += (int)nt) work(g);
            });
        for (auto &t : th) t.join();
        size_t total = 0;
        for (int g = 0; g < c->G; ++g) total += g_col[g].size();
        if (total >= (size_t(1) << 31)) return fail(PD_EINVAL, "too many bonds for 32-bit indices");
        c->row_ptr.assign(c->N + 1, 0);
        c->col.clear();
        c->col.reserve(total);
        for (int g = 0; g < c->G; ++g) {
            int64_t s0 = c->g_start[g];
            int n = (int)(c->g_start[g + 1] - s0);
            int32_t base = (int32_t)c->col.size();
            for (int x = 0; x < n; ++x) c->row_ptr[s0 + x + 1] = base + g_row[g][x + 1];
            c->col.insert(c->col.end(), g_col[g].begin(), g_col[g].end());
        }
        c->xi.resize(c->col.size());
        c->max_row = 0;
        for (int64_t x = 0; x < c->N; ++x) {
            c->max_row = std::max(c->max_row, c->row_ptr[x + 1] - c->row_ptr[x]);
            for (int32_t b = c->row_ptr[x]; b < c->row_ptr[x + 1]; ++b) {
                int32_t y = c->col[b];
                double dx = c->X[2 * y] - c->X[2 * x], dy = c->X[2 * y + 1] - c->X[2 * x + 1];
                c->xi[b] = std::sqrt(dx * dx + dy * dy);
            }
        }
    } catch (const std::bad_alloc &) {
        return fail(PD_ENOMEM, "out of host memory while building bonds");
    }
    c->wpn = std::max(1, (c->max_row + 31) / 32);
    // bond-network templates: grains of one shape meshed at the same h/R have
    // the same lattice (and so the same bonds) -- verified node by node
    c->g_tmpl.assign(c->G, -1);
    c->tmpl_first.clear();
    c->tmpl_count.clear();
    c->tmpl_nodes.clear();
    c->g_slot.assign(c->G, 0);
    for (int g = 0; g < c->G; ++g) {
        const int64_t a0 = c->g_start[g], n = c->g_start[g + 1] - a0;
        for (int t = 0; t < (int)c->tmpl_first.size() && c->g_tmpl[g] < 0; ++t) {
            const int r = c->tmpl_first[t];
            const int64_t b0 = c->g_start[r];
            if (c->g_shape[r] != c->g_shape[g] || c->g_start[r + 1] - b0 != n) continue;
            if (std::fabs(c->g_R[r] / c->g_h[r] - c->g_R[g] / c->g_h[g]) > 1e-9 * (c->g_R[g] / c->g_h[g])) continue;
            if (!std::equal(c->lat.begin() + 2 * a0, c->lat.begin() + 2 * (a0 + n), c->lat.begin() + 2 * b0)) continue;
            bool same = true;
            for (int64_t x = 0; x < n && same; ++x) {
                const int32_t ra = c->row_ptr[a0 + x + 1] - c->row_ptr[a0 + x], rb = c->row_ptr[b0 + x + 1] - c->row_ptr[b0 + x];
                same = ra == rb;
                for (int32_t q = 0; q < ra && same; ++q)
                    same = c->col[c->row_ptr[a0 + x] + q] - a0 == c->col[c->row_ptr[b0 + x] + q] - b0;
            }
            if (same) c->g_tmpl[g] = t;
        }
        if (c->g_tmpl[g] < 0) {
            c->g_tmpl[g] = (int)c->tmpl_first.size();
            c->tmpl_first.push_back(g);
            c->tmpl_count.push_back(0);
            c->tmpl_nodes.push_back((int)n);
        }
        c->g_slot[g] = c->tmpl_count[c->g_tmpl[g]]++;
    }
    c->n_tmpl = (int)c->tmpl_first.size();
    // contact hash: power of two >= 2N buckets
    if (c->N > (int64_t(1) << 29)) return fail(PD_EINVAL, "too many nodes for the contact grid (at most 2^29)");
    unsigned T = 1024;
    while ((int64_t)T < 2 * c->N) T <<= 1;
    c->T = T;
    c->state = 2;
    if (n_bonds_out) *n_bonds_out = (int64_t)c->col.size();
    return PD_OK;
}

int pd_arena_bytes(pd_ctx *c, size_t *bytes) {
    if (int r = check_ctx(c, 2)) return r;
    if (!bytes) return fail(PD_EINVAL, "null bytes");
    c->kp.n_diag_blocks = (int)std::min<int64_t>(1024, (c->N + pd::kBlock - 1) / pd::kBlock);
    *bytes = layout(c, nullptr);
    return PD_OK;
}

int pd_bind_arena(pd_ctx *c, void *arena, size_t bytes) {
    if (int r = check_ctx(c, 2)) return r;
    if (c->state != 2) return fail(PD_ESTATE, "arena already bound");
    if (!arena || ((uintptr_t)arena & 255)) return fail(PD_EINVAL, "arena null or not 256-byte aligned");
    c->kp.n_diag_blocks = (int)std::min<int64_t>(1024, (c->N + pd::kBlock - 1) / pd::kBlock);
    size_t need = layout(c, nullptr);
    if (bytes < need) return fail(PD_EINVAL, "arena too small");
    c->arena_bytes = layout(c, (char *)arena);
    const pd_params &p = c->prm;
    pd::KParams &k = c->kp;
    k.N = (int)c->N;
    k.G = c->G;
    k.wpn = c->wpn;
    k.T = c->T;
    k.n_agg = c->n_agg;
    k.rho = p.rho;
    k.rd = p.damping_ratio;
    k.mu = p.friction;
    k.gx = p.gravity[0];
    k.gy = p.gravity[1];
    k.dt = p.dt;
    k.half_dt = 0.5 * p.dt;
    k.half_dt2 = 0.5 * p.dt * p.dt;
    k.rhof = (float)p.rho;
    k.rdf = (float)p.damping_ratio;
    k.muf = (float)p.friction;
    k.dtf = (float)p.dt;
    k.gxf = (float)p.gravity[0];
    k.gyf = (float)p.gravity[1];
    k.guard = 1e-4f;
    k.mat = c->has_mat ? 1 : 0;
    // one rebuild trigger for all aggregates: the smallest (the most cautious)
    k.dmax2 = c->aggp[0].dmax2;
    for (const pd::AggParams &A : c->aggp) k.dmax2 = std::min(k.dmax2, A.dmax2);
    k.fp32 = p.precision == PD_FP32_SPLIT ? 1 : 0;
    k.sur = 0;
    k.n_modes = c->sur_modes;
    k.judge_every = c->sur_judge;
    k.E = (float)p.E;
    k.gate = (float)c->sur_gate;
    k.err_tol = (float)c->sur_tol;
    k.n_proj_work = (int)c->proj_work.size();
    k.n_exp_work = (int)c->exp_work.size();
    k.n_rows = (int)c->slot_grain.size();
    k.bar_spins = pd::kBarrierSpins;
    k.withhold_block = -1;
    k.micro = p.micromodulus;
    k.store = p.store_parts ? 1 : 0;
    k.lanes = p.lanes == 0 ? 4 : p.lanes;
    k.split = 1;          // default path: kernel graph, split force phase (pd_set_path mode 2)
    {
        // L2 prefetch of the force phase's read-only arrays when they fit well in L2
        const size_t nb = c->col.size();
        const size_t pf = (size_t)c->N * (16 + 4 * (size_t)c->wpn + 4 * pd::kPrefetchListRows) +
                          nb * (k.fp32 ? 4 : 12);
        k.pf_bonds = (nb > 0 && nb < ((size_t)1 << 31) && pf < pd::kPrefetchMaxBytes) ? (int)nb : 0;
    }
    cudaStream_t s = c->stream;
    const pd::DevPtrs &d = c->d;
    size_t N = (size_t)c->N, nb = c->col.size(), G = (size_t)c->G;
    // host staging (kept alive until the stream drains below)
    std::vector<uint32_t> bits(N * c->wpn, 0u);
    PD_CUDA(cudaMemcpyAsync(d.X, c->X.data(), 16 * N, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemsetAsync(d.u, 0, 16 * N, s));
    PD_CUDA(cudaMemcpyAsync(d.v[0], c->v0.data(), 16 * N, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemsetAsync(d.v[1], 0, 16 * N, s));
    if (d.af) PD_CUDA(cudaMemsetAsync(d.af, 0, 8 * N, s));
    else PD_CUDA(cudaMemsetAsync(d.a, 0, 16 * N, s));
    PD_CUDA(cudaMemcpyAsync(d.V, c->V.data(), 8 * N, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.grain, c->grain.data(), 4 * N, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.row_ptr, c->row_ptr.data(), 4 * (N + 1), cudaMemcpyHostToDevice, s));
    if (nb) {
        PD_CUDA(cudaMemcpyAsync(d.col, c->col.data(), 4 * nb, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.xi, c->xi.data(), 8 * nb, cudaMemcpyHostToDevice, s));
    }
    PD_CUDA(cudaMemcpyAsync(d.bits, bits.data(), 4 * bits.size(), cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_cw, c->g_cw.data(), 8 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_s0, c->g_s0.data(), 8 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_eps, c->g_eps.data(), 8 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_agg, c->g_agg.data(), 4 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_rho, c->g_rho.data(), 8 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.g_k, c->g_k.data(), 8 * G, cudaMemcpyHostToDevice, s));
    std::vector<float> gkf(G);
    for (size_t g = 0; g < G; ++g) gkf[g] = (float)(18.0 * c->g_k[g] / c->aggp[c->g_agg[g]].pe5);
    PD_CUDA(cudaMemcpyAsync(d.g_kf, gkf.data(), 4 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.agg, c->aggp.data(), sizeof(pd::AggParams) * c->aggp.size(), cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), s));
    PD_CUDA(cudaMemsetAsync(d.t_now, 0, sizeof(double), s));
    // bucket counts are zero between rebuilds; the first force evaluation rebuilds
    PD_CUDA(cudaMemsetAsync(d.count, 0, sizeof(int) * c->T, s));
    PD_CUDA(cudaMemsetAsync(d.nbr_cnt, 0, 4 * N, s));
    PD_CUDA(cudaMemsetAsync(d.sref, 0, 16 * N, s));
    PD_CUDA(cudaMemsetAsync(d.rebuild, 1, sizeof(int), s));
    PD_CUDA(cudaMemsetAsync(d.pred_done, 0, sizeof(unsigned), s));
    PD_CUDA(cudaMemsetAsync(d.rebuild_next, 0, sizeof(int), s));
    PD_CUDA(cudaMemsetAsync(d.pred_ok, 0, sizeof(int), s));
    std::vector<int32_t> gstart32(c->g_start.begin(), c->g_start.end()), tnode, tslot;
    PD_CUDA(cudaMemcpyAsync(d.g_start, gstart32.data(), 4 * (G + 1), cudaMemcpyHostToDevice, s));
    std::vector<float> fc;
    if (c->sur_cfg) {
        tnode.assign(c->n_tmpl + 1, 0);
        tslot.assign(c->n_tmpl + 1, 0);
        for (int t = 0; t < c->n_tmpl; ++t) {
            tnode[t + 1] = tnode[t] + c->tmpl_nodes[t];
            tslot[t + 1] = tslot[t] + c->tmpl_count[t];
        }
        // per grain: h as a float-float pair and the centroid of its lattice indices
        fc.assign(4 * G, 0.f);
        for (size_t g = 0; g < G; ++g) {
            double si = 0, sj = 0;
            for (int64_t x = c->g_start[g]; x < c->g_start[g + 1]; ++x) {
                si += c->lat[2 * x];
                sj += c->lat[2 * x + 1];
            }
            const double n = (double)(c->g_start[g + 1] - c->g_start[g]);
            const float hh = (float)c->g_h[g];
            fc[4 * g] = hh;
            fc[4 * g + 1] = (float)(c->g_h[g] - (double)hh);
            fc[4 * g + 2] = (float)(si / n);
            fc[4 * g + 3] = (float)(sj / n);
        }

        PD_CUDA(cudaMemcpyAsync(d.g_tmpl, c->g_tmpl.data(), 4 * G, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.g_slot, c->g_slot.data(), 4 * G, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.tmpl_node, tnode.data(), 4 * tnode.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.tmpl_slot, tslot.data(), 4 * tslot.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.basis, c->sur_basis.data(), 4 * c->sur_basis.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.bnm_hi, c->bnm_hi.data(), 2 * c->bnm_hi.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.bnm_lo, c->bnm_lo.data(), 2 * c->bnm_lo.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.bmm_hi, c->bmm_hi.data(), 2 * c->bmm_hi.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.bmm_lo, c->bmm_lo.data(), 2 * c->bmm_lo.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.tmpl_rows, c->tmpl_rows.data(), 4 * c->tmpl_rows.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.slot_grain, c->slot_grain.data(), 4 * c->slot_grain.size(), cudaMemcpyHostToDevice, s));
        if (!c->proj_work.empty())
            PD_CUDA(cudaMemcpyAsync(d.proj_work, c->proj_work.data(), sizeof(int4) * c->proj_work.size(),
                                    cudaMemcpyHostToDevice, s));
        if (!c->exp_work.empty())
            PD_CUDA(cudaMemcpyAsync(d.exp_work, c->exp_work.data(), sizeof(int4) * c->exp_work.size(),
                                    cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemsetAsync(d.sur_w, 0, 8 * N, s));
        PD_CUDA(cudaMemsetAsync(d.sur_f, 0, 8 * N, s));
        PD_CUDA(cudaMemsetAsync(d.sur_merr, 0, 4 * G, s));
        PD_CUDA(pd::sur_init_attributes());
        PD_CUDA(pd::mlp_init_attributes());
        PD_CUDA(cudaMemsetAsync(d.mlp_err, 0, sizeof(int), s));
        PD_CUDA(cudaMemcpyAsync(d.sur_lambda, c->sur_lambda.data(), 4 * c->sur_lambda.size(), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.g_theta, c->g_theta.data(), 8 * G, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.sur_fc, fc.data(), 16 * G, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemsetAsync(d.sur_active, 0, 4 * G, s));
        PD_CUDA(cudaMemsetAsync(d.sur_y, 0, 4 * G * c->sur_modes, s));
        PD_CUDA(cudaMemsetAsync(d.sur_err, 0, 4 * G, s));
        PD_CUDA(cudaMemsetAsync(d.sur_maxs, 0, 4 * G, s));
        c->sur_mlp.assign(c->n_tmpl, nullptr);
    }
    PD_CUDA(cudaMemsetAsync(d.step, 0, 8, s));
    PD_CUDA(cudaMemsetAsync(d.status, 0, 4 * PD_STATUS_COUNT, s));
    std::vector<float> gq, gcf;
    std::vector<double> invm;
    std::vector<uint32_t> colx;
    std::vector<uint4> stn;
    std::vector<double> xs;
    if (p.precision == PD_FP32_SPLIT) {
        // per grain: h, h^2 as a float-float pair, V as float
        gq.resize(4 * G);
        for (size_t g = 0; g < G; ++g) {
            double h = c->g_h[g], h2 = h * h;
            float hi = (float)h2;
            gq[4 * g] = (float)h;
            gq[4 * g + 1] = hi;
            gq[4 * g + 2] = (float)(h2 - (double)hi);
            gq[4 * g + 3] = (float)c->V[c->g_start[g]];
        }
        PD_CUDA(cudaMemcpyAsync(d.lat, c->lat.data(), 8 * N, cudaMemcpyHostToDevice, s));
        // bond columns with the lattice offset n = di^2 + dj^2 in the top bits
        // (the FP32 bond kernel's |xi|^2 = n h^2 needs no neighbour lattice load)
        if (N > (size_t)pd::kColMask) return fail(PD_EINVAL, "FP32-split path: at most 2^28 - 1 nodes");
        colx.resize(nb);
        for (size_t x = 0; x < N; ++x)
            for (int b = c->row_ptr[x]; b < c->row_ptr[x + 1]; ++b) {
                const int j = c->col[b];
                const int64_t di = c->lat[2 * (size_t)j] - c->lat[2 * x], dj = c->lat[2 * (size_t)j + 1] - c->lat[2 * x + 1];
                const int64_t n = di * di + dj * dj;
                if (n >= (int64_t)1 << (32 - pd::kColBits))
                    return fail(PD_EINVAL, "FP32-split path: horizons up to 4 lattice spacings");
                colx[b] = (uint32_t)j | ((uint32_t)n << pd::kColBits);
            }
        if (nb) PD_CUDA(cudaMemcpyAsync(d.colx, colx.data(), 4 * nb, cudaMemcpyHostToDevice, s));
        // lattice stencil of the bonds (horizons with exactly the 24 offsets of the 5 x 5 block)
        const double hr2 = p.horizon_ratio * p.horizon_ratio;
        c->kp.stencil = (hr2 > 8.0 && hr2 <= 9.0) ? 1 : 0;
        if (c->kp.stencil) {
            stn.assign(N, make_uint4(pd::kStnIrregular, 0u, 0u, 0u));
            size_t irregular = 0;
            for (size_t x = 0; x < N; ++x) {
                uint32_t mask = 0;
                int D[5] = {0, 0, 0, 0, 0};
                bool seen[5] = {false, false, false, false, false}, ok = true;
                int last = -1;
                for (int b = c->row_ptr[x]; b < c->row_ptr[x + 1] && ok; ++b) {
                    const int j = c->col[b];
                    const int di = c->lat[2 * (size_t)j] - c->lat[2 * x], dj = c->lat[2 * (size_t)j + 1] - c->lat[2 * x + 1];
                    if (di < -2 || di > 2 || dj < -2 || dj > 2) { ok = false; break; }
                    const int oo = (dj + 2) * 5 + (di + 2), o = oo < 12 ? oo : oo - 1;
                    const long long base = (long long)j - (long long)x - di;
                    if (o <= last) ok = false;                      // CSR order must be the offset order
                    last = o;
                    if (!seen[dj + 2]) { seen[dj + 2] = true; D[dj + 2] = (int)std::max<long long>(-40000, std::min<long long>(40000, base)); }
                    else if (D[dj + 2] != base) ok = false;
                    if (dj == 0 && base != 0) ok = false;
                    if (D[dj + 2] < -32768 || D[dj + 2] > 32767) ok = false;
                    mask |= 1u << o;
                }
                if (!ok) {
                    stn[x] = make_uint4(pd::kStnIrregular, 0u, 0u, (unsigned)c->row_ptr[x]);
                    ++irregular;
                    continue;
                }
                auto u16 = [](int v) { return (uint32_t)(uint16_t)(int16_t)v; };
                stn[x] = make_uint4(mask, u16(D[0]) | (u16(D[1]) << 16), u16(D[3]) | (u16(D[4]) << 16),
                                    (unsigned)c->row_ptr[x]);
            }
            c->stn_irregular = irregular;
            PD_CUDA(cudaMemcpyAsync(d.stn, stn.data(), 16 * N, cudaMemcpyHostToDevice, s));
        }
        // X + the aggregate's shift (FP64): the FP32-split positions are (X + shift) + u
        xs.resize(2 * N);
        for (size_t x = 0; x < N; ++x) {
            const pd::AggParams &A = c->aggp[c->g_agg[c->grain[x]]];
            xs[2 * x] = c->X[2 * x] + A.sx;
            xs[2 * x + 1] = c->X[2 * x + 1] + A.sy;
        }
        PD_CUDA(cudaMemcpyAsync(d.xs, xs.data(), 16 * N, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.gq, gq.data(), 16 * G, cudaMemcpyHostToDevice, s));
        gcf.resize(4 * G);
        for (size_t g = 0; g < G; ++g) {
            gcf[4 * g] = (float)c->g_cw[g];
            gcf[4 * g + 1] = (float)c->g_s0[g];
            gcf[4 * g + 2] = (float)c->g_eps[g];
            gcf[4 * g + 3] = (float)c->g_rho[g];
        }
        PD_CUDA(cudaMemcpyAsync(d.gc, gcf.data(), 16 * G, cudaMemcpyHostToDevice, s));
    }
    // per grain 1 / (rho V): the update multiplies by it (an FP64 division per
    // node and component costs about nine FP64 operations on GB300)
    invm.resize(G);
    for (size_t g = 0; g < G; ++g) invm[g] = 1.0 / (c->g_rho[g] * c->V[c->g_start[g]]);
    PD_CUDA(cudaMemcpyAsync(d.g_invm, invm.data(), 8 * G, cudaMemcpyHostToDevice, s));
    std::vector<float> invmf(invm.begin(), invm.end());
    PD_CUDA(cudaMemcpyAsync(d.g_invmf, invmf.data(), 4 * G, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaStreamSynchronize(s));
    c->vcur = 0;
    set_current(c);
    c->steps_done = 0;
    c->state = 3;
    // initial acceleration a^0 from the forces of the initial state
    if (int r = pd_eval_forces(c)) {
        c->state = 2;
        return r;
    }
    PD_CUDA(cudaStreamSynchronize(s));
    // capture the step graphs on a private stream (the caller's may be the legacy stream)
    PD_CUDA(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    PD_CUDA(cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking));
    PD_CUDA(cudaStreamCreateWithFlags(&c->sur_stream, cudaStreamNonBlocking));
    PD_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    PD_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    for (auto &e : c->ev) PD_CUDA(cudaEventCreate(&e));
    return capture_all(c);
}

int pd_eval_forces(pd_ctx *c) {
    if (int r = check_ctx(c, 3)) return r;
    cudaStream_t s = c->stream;
    PD_CUDA(pd::launch_predict(c->d, c->kp, c->vcur, 0, s, 0, 0));
    PD_CUDA(cudaMemsetAsync(c->d.rebuild, 1, sizeof(int), s));     // fresh candidate lists
    PD_CUDA(pd::launch_rebuild(c->d, c->kp, s));
    if (c->kp.sur) PD_CUDA(record_surrogate(c, c->d, s));
    PD_CUDA(pd::launch_force(c->d, c->kp, c->vcur, 0, s));
    return PD_OK;
}

int pd_step(pd_ctx *c, int n_steps) {
    if (int r = check_ctx(c, 3)) return r;
    if (n_steps < 0) return fail(PD_EINVAL, "negative step count");
    int n = n_steps;
    if (c->timing) {
        for (int k = 0; k < n; ++k) {
            PD_CUDA(cudaGraphLaunch(c->timed[c->vcur], c->stream));
            c->vcur ^= 1;
            set_current(c);
        }
        c->steps_done += n_steps;
        return PD_OK;
    }
    while (n >= kChunk) {
        PD_CUDA(cudaGraphLaunch(c->chunk[c->vcur], c->stream));
        // kChunk is even: the velocity buffer parity is unchanged
        n -= kChunk;
    }
    while (n > 0) {
        PD_CUDA(cudaGraphLaunch(c->single[c->vcur], c->stream));
        c->vcur ^= 1;
        set_current(c);
        --n;
    }
    c->steps_done += n_steps;
    return PD_OK;
}

int pd_get_state(pd_ctx *c, int field, void *dst, size_t bytes, int dst_on_device) {
    if (int r = check_ctx(c, 1)) return r;
    size_t fb = field_bytes(c, field);
    if (fb == 0 && field != PD_FIELD_BROKEN && field != PD_FIELD_COL) return fail(PD_EINVAL, "unknown field");
    if (bytes != fb) return fail(PD_EINVAL, "size mismatch for field");
    if (!dst && fb) return fail(PD_EINVAL, "null destination");
    if (fb == 0) return PD_OK;
    // host-side mesh fields are available from meshing on
    const void *host = nullptr;
    switch (field) {
        case PD_FIELD_X: host = c->X.data(); break;
        case PD_FIELD_GRAIN: host = c->grain.data(); break;
        case PD_FIELD_VOLUME: host = c->V.data(); break;
        case PD_FIELD_LATTICE: host = c->lat.data(); break;
        case PD_FIELD_ROW_PTR: if (c->state >= 2) host = c->row_ptr.data(); break;
        case PD_FIELD_COL: if (c->state >= 2) host = c->col.data(); break;
        case PD_FIELD_GRAIN_TEMPLATE: if (c->state >= 2) host = c->g_tmpl.data(); break;
        default: break;
    }
    if (dst_on_device < PD_MEM_HOST || dst_on_device > PD_MEM_HOST_ASYNC) return fail(PD_EINVAL, "unknown memory kind");
    if (host) {
        if (dst_on_device == PD_MEM_DEVICE) PD_CUDA(cudaMemcpyAsync(dst, host, fb, cudaMemcpyHostToDevice, c->stream));
        else std::memcpy(dst, host, fb);
        if (dst_on_device == PD_MEM_DEVICE) PD_CUDA(cudaStreamSynchronize(c->stream));
        return PD_OK;
    }
    if (c->state < 3) return fail(PD_ESTATE, "field needs a bound arena");
    cudaMemcpyKind kind = dst_on_device == PD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const pd::DevPtrs &d = c->d;
    cudaStream_t s = c->stream;
    switch (field) {
        case PD_FIELD_DISP: PD_CUDA(cudaMemcpyAsync(dst, d.u, fb, kind, s)); break;
        case PD_FIELD_VEL: PD_CUDA(cudaMemcpyAsync(dst, d.v[c->vcur], fb, kind, s)); break;
        case PD_FIELD_ACC:
            if (!d.af) {
                PD_CUDA(cudaMemcpyAsync(dst, d.a, fb, kind, s));
            } else if (dst_on_device == PD_MEM_DEVICE) {
                PD_CUDA(pd::launch_widen(d.af, static_cast<double2 *>(dst), (size_t)c->N, s));
            } else {
                // widened on the device into the backup buffer, then copied
                PD_CUDA(pd::launch_widen(d.af, d.ba, (size_t)c->N, s));
                PD_CUDA(cudaMemcpyAsync(dst, d.ba, fb, cudaMemcpyDeviceToHost, s));
            }
            break;
        case PD_FIELD_POS:
            PD_CUDA(pd::launch_positions(d, c->kp, s));
            PD_CUDA(cudaMemcpyAsync(dst, d.p, fb, kind, s));
            break;
        case PD_FIELD_FORCE:
            if (!c->prm.store_parts) return fail(PD_ESTATE, "forces are kept only with store_parts");
            PD_CUDA(cudaMemcpyAsync(dst, d.F, fb, kind, s));
            break;
        case PD_FIELD_FORCE_PARTS:
            if (!c->prm.store_parts) return fail(PD_ESTATE, "forces are kept only with store_parts");
            PD_CUDA(cudaMemcpyAsync(dst, d.parts, fb, kind, s));
            break;
        case PD_FIELD_STEP: PD_CUDA(cudaMemcpyAsync(dst, d.step, 8, kind, s)); break;
        case PD_FIELD_BROKEN:
        case PD_FIELD_DAMAGE: {
            if (dst_on_device == PD_MEM_DEVICE) return fail(PD_EINVAL, "BROKEN/DAMAGE are host-only fields");
            std::vector<uint32_t> bits((size_t)c->N * c->wpn);
            PD_CUDA(cudaMemcpyAsync(bits.data(), d.bits, 4 * bits.size(), cudaMemcpyDeviceToHost, s));
            PD_CUDA(cudaStreamSynchronize(s));
            for (int64_t x = 0; x < c->N; ++x) {
                int r0 = c->row_ptr[x], r1 = c->row_ptr[x + 1], nbk = 0;
                for (int b = r0; b < r1; ++b) {
                    int k = b - r0;
                    int br = (bits[(size_t)x * c->wpn + k / 32] >> (k % 32)) & 1u;
                    nbk += br;
                    if (field == PD_FIELD_BROKEN) ((uint8_t *)dst)[b] = (uint8_t)br;
                }
                if (field == PD_FIELD_DAMAGE) ((double *)dst)[x] = r1 > r0 ? (double)nbk / (double)(r1 - r0) : 0.0;
            }
            return PD_OK;
        }
        default: return fail(PD_EINVAL, "unknown field");
    }
    if (dst_on_device == PD_MEM_HOST) PD_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}

int pd_set_state(pd_ctx *c, int field, const void *src, size_t bytes, int src_on_device) {
    if (int r = check_ctx(c, 3)) return r;
    size_t fb = field_bytes(c, field);
    if (bytes != fb) return fail(PD_EINVAL, "size mismatch for field");
    if (!src && fb) return fail(PD_EINVAL, "null source");
    if (src_on_device < PD_MEM_HOST || src_on_device > PD_MEM_HOST_ASYNC) return fail(PD_EINVAL, "unknown memory kind");
    cudaMemcpyKind kind = src_on_device == PD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const pd::DevPtrs &d = c->d;
    cudaStream_t s = c->stream;
    // the persistent kernel's prediction of the next step was made from the old state
    PD_CUDA(cudaMemsetAsync(d.pred_ok, 0, sizeof(int), s));
    switch (field) {
        case PD_FIELD_DISP: PD_CUDA(cudaMemcpyAsync(d.u, src, fb, kind, s)); break;
        case PD_FIELD_VEL: PD_CUDA(cudaMemcpyAsync(d.v[c->vcur], src, fb, kind, s)); break;
        case PD_FIELD_ACC:
            if (!d.af) {
                PD_CUDA(cudaMemcpyAsync(d.a, src, fb, kind, s));
            } else if (src_on_device == PD_MEM_DEVICE) {
                PD_CUDA(pd::launch_narrow(static_cast<const double2 *>(src), d.af, (size_t)c->N, s));
            } else {
                // through the backup buffer, rounded to float on the device
                PD_CUDA(cudaMemcpyAsync(d.ba, src, fb, cudaMemcpyHostToDevice, s));
                PD_CUDA(pd::launch_narrow(d.ba, d.af, (size_t)c->N, s));
            }
            break;
        case PD_FIELD_STEP: {
            int64_t st = 0;
            if (src_on_device == PD_MEM_DEVICE) PD_CUDA(cudaMemcpy(&st, src, 8, cudaMemcpyDeviceToHost));
            else std::memcpy(&st, src, 8);
            PD_CUDA(cudaMemcpyAsync(d.step, src, 8, kind, s));
            c->steps_done = st;
            break;
        }
        case PD_FIELD_BROKEN: {
            if (src_on_device == PD_MEM_DEVICE) return fail(PD_EINVAL, "BROKEN is a host-only field");
            std::vector<uint32_t> bits((size_t)c->N * c->wpn, 0u);
            for (int64_t x = 0; x < c->N; ++x)
                for (int b = c->row_ptr[x]; b < c->row_ptr[x + 1]; ++b) {
                    int k = b - c->row_ptr[x];
                    if (((const uint8_t *)src)[b]) bits[(size_t)x * c->wpn + k / 32] |= 1u << (k % 32);
                }
            PD_CUDA(cudaMemcpyAsync(d.bits, bits.data(), 4 * bits.size(), cudaMemcpyHostToDevice, s));
            PD_CUDA(cudaStreamSynchronize(s));
            return PD_OK;
        }
        default: return fail(PD_EINVAL, "field is not settable");
    }
    if (src_on_device == PD_MEM_HOST || field == PD_FIELD_STEP) PD_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}

int pd_diagnostics(pd_ctx *c, double *out) {
    if (int r = check_ctx(c, 3)) return r;
    if (!out) return fail(PD_EINVAL, "null output");
    PD_CUDA(pd::launch_diagnostics(c->d, c->kp, c->vcur, c->stream));
    PD_CUDA(cudaMemcpyAsync(out, c->d.diag_out, 8 * PD_DIAG_COUNT, cudaMemcpyDeviceToHost, c->stream));
    PD_CUDA(cudaStreamSynchronize(c->stream));
    return PD_OK;
}

int pd_observables(pd_ctx *c, double *out) {
    if (int r = check_ctx(c, 3)) return r;
    if (!out) return fail(PD_EINVAL, "null output");
    const size_t G = (size_t)c->G, A = (size_t)c->n_agg;
    PD_CUDA(pd::launch_observables(c->d, c->kp, c->vcur, c->d.obs_gdam, c->d.obs_wall, c->stream));
    std::vector<double> gdam(G), wsum(16 * A);
    long long step = 0;
    PD_CUDA(cudaMemcpyAsync(gdam.data(), c->d.obs_gdam, 8 * G, cudaMemcpyDeviceToHost, c->stream));
    PD_CUDA(cudaMemcpyAsync(wsum.data(), c->d.obs_wall, 8 * 16 * A, cudaMemcpyDeviceToHost, c->stream));
    PD_CUDA(cudaMemcpyAsync(&step, c->d.step, 8, cudaMemcpyDeviceToHost, c->stream));
    PD_CUDA(cudaStreamSynchronize(c->stream));
    const double t = (double)step * c->prm.dt;
    std::vector<double> vol(A, 0.0), dsum(A, 0.0);
    std::vector<int> ng(A, 0);
    for (size_t g = 0; g < G; ++g) {
        const int a = c->g_agg[g];
        for (int64_t x = c->g_start[g]; x < c->g_start[g + 1]; ++x) vol[a] += c->V[x];
        dsum[a] += gdam[g];
        ng[a] += 1;
    }
    for (size_t a = 0; a < A; ++a) {
        const double *w = &c->agg_walls[8 * a];
        const double xlo = w[0] + w[4] * t, xhi = w[1] + w[5] * t, ylo = w[2] + w[6] * t, yhi = w[3] + w[7] * t;
        const double *ws = &wsum[16 * a];
        // force of wall l on the nodes: its own segment term less half of each
        // corner term it shares; the aggregate exerts the opposite force
        // (corners: 0 (x_lo,y_lo), 1 (x_lo,y_hi), 2 (x_hi,y_lo), 3 (x_hi,y_hi))
        const double top = ws[2 * 3 + 1] - 0.5 * (ws[8 + 2 * 1 + 1] + ws[8 + 2 * 3 + 1]);
        const double bottom = ws[2 * 2 + 1] - 0.5 * (ws[8 + 2 * 0 + 1] + ws[8 + 2 * 2 + 1]);
        out[PD_OBS_COUNT * a + PD_OBS_PHI] = vol[a] / ((xhi - xlo) * (yhi - ylo));
        out[PD_OBS_COUNT * a + PD_OBS_BULK_DAMAGE] = ng[a] ? dsum[a] / ng[a] : 0.0;
        out[PD_OBS_COUNT * a + PD_OBS_FORCE_TOP] = -top;
        out[PD_OBS_COUNT * a + PD_OBS_FORCE_BOTTOM] = -bottom;
    }
    return PD_OK;
}

int pd_status(pd_ctx *c, int32_t *out) {
    if (int r = check_ctx(c, 3)) return r;
    int32_t st[PD_STATUS_COUNT];
    PD_CUDA(cudaMemcpyAsync(st, c->d.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    PD_CUDA(cudaStreamSynchronize(c->stream));
    if (out) std::memcpy(out, st, sizeof(st));
    if (st[PD_STATUS_NONFINITE]) return fail(PD_ENUMERIC, "non-finite acceleration");
    if (st[PD_STATUS_OVERFLOW]) return fail(PD_EOVERFLOW, "contact candidate overflow");
    int mlp_err = 0;
    if (c->d.mlp_err) {
        PD_CUDA(cudaMemcpy(&mlp_err, c->d.mlp_err, sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (st[PD_STATUS_TIMEOUT] || mlp_err)
        return fail(PD_ETIMEOUT, "a bounded device wait gave up (the surrogate is off from then on)");
    return PD_OK;
}

int pd_clear_status(pd_ctx *c) {
    if (int r = check_ctx(c, 3)) return r;
    const pd::DevPtrs &d = c->d;
    cudaStream_t s = c->stream;
    PD_CUDA(cudaMemsetAsync(d.status, 0, sizeof(int) * PD_STATUS_COUNT, s));
    if (d.mlp_err) PD_CUDA(cudaMemsetAsync(d.mlp_err, 0, sizeof(int), s));
    PD_CUDA(cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), s));
    PD_CUDA(cudaMemsetAsync(d.pred_done, 0, sizeof(unsigned), s));
    PD_CUDA(cudaMemsetAsync(d.pred_ok, 0, sizeof(int), s));
    PD_CUDA(cudaMemsetAsync(d.rebuild_next, 0, sizeof(int), s));
    // a step that gave up inside a rebuild leaves bucket counts behind; they are
    // zero between rebuilds, and the next step rebuilds the candidate lists
    PD_CUDA(cudaMemsetAsync(d.count, 0, sizeof(int) * c->T, s));
    PD_CUDA(cudaMemsetAsync(d.rebuild, 1, sizeof(int), s));
    PD_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}

int pd_set_wait_test(pd_ctx *c, int withhold_block, long long max_spins) {
    if (int r = check_ctx(c, 3)) return r;
    if (withhold_block < -1) return fail(PD_EINVAL, "withhold_block must be -1 or a block index");
    if (max_spins < 0) return fail(PD_EINVAL, "negative spin limit");
    c->kp.withhold_block = withhold_block;
    c->kp.bar_spins = max_spins == 0 ? pd::kBarrierSpins : max_spins;
    return capture_all(c);
}

int pd_set_materials(pd_ctx *c, int n_mat, const double *props, const int32_t *grain_material) {
    if (int r = check_ctx(c, 1)) return r;
    if (c->state > 2) return fail(PD_ESTATE, "pd_set_materials must come before pd_bind_arena");
    if (c->sur_cfg) return fail(PD_ESTATE, "the surrogate runs with one material: set materials before it");
    if (n_mat < 1 || !props || !grain_material) return fail(PD_EINVAL, "n_mat >= 1 and non-null arrays required");
    for (int m = 0; m < n_mat; ++m)
        for (int q = 0; q < 4; ++q)
            if (!(props[4 * m + q] > 0.0) || !std::isfinite(props[4 * m + q]))
                return fail(PD_EINVAL, "material properties must be positive and finite");
    for (int g = 0; g < c->G; ++g)
        if (grain_material[g] < 0 || grain_material[g] >= n_mat) return fail(PD_EINVAL, "grain material out of range");
    const pd_params &p = c->prm;
    for (int g = 0; g < c->G; ++g) {
        const double *m = props + 4 * (size_t)grain_material[g];
        const double E = m[0], Gc = m[3], eps = c->g_eps[g];
        if (p.micromodulus == PD_MICRO_CONSTANT) {
            c->g_cw[g] = 6.0 * E / (kPi * eps * eps * eps * (1.0 - p.nu));
            c->g_s0[g] = std::sqrt(4.0 * kPi * Gc / (9.0 * E * eps));
        } else {
            c->g_cw[g] = 24.0 * E / (kPi * eps * eps * eps * (1.0 - p.nu));
            c->g_s0[g] = std::sqrt(5.0 * kPi * Gc / (9.0 * E * eps));
        }
        c->g_k[g] = m[1];
        c->g_rho[g] = m[2];
    }
    c->has_mat = true;
    return PD_OK;
}

int pd_set_aggregates(pd_ctx *c, int n_agg, const int32_t *grain_agg, const double *agg_walls) {
    if (int r = check_ctx(c, 1)) return r;
    if (c->state > 2) return fail(PD_ESTATE, "pd_set_aggregates must come before pd_bind_arena");
    if (n_agg < 1 || !grain_agg || !agg_walls) return fail(PD_EINVAL, "n_agg >= 1 and non-null arrays required");
    for (int g = 0; g < c->G; ++g)
        if (grain_agg[g] < 0 || grain_agg[g] >= n_agg) return fail(PD_EINVAL, "grain aggregate out of range");
    for (int a = 0; a < n_agg; ++a) {
        const double *w = agg_walls + 8 * (size_t)a;
        if (!(w[1] > w[0]) || !(w[3] > w[2])) return fail(PD_EINVAL, "aggregate wall box is empty");
    }
    c->n_agg = n_agg;
    c->g_agg.assign(grain_agg, grain_agg + c->G);
    c->agg_walls.assign(agg_walls, agg_walls + 8 * (size_t)n_agg);
    compute_aggregates(c);
    return PD_OK;
}

int pd_autotune(pd_ctx *c, double *report) {
    if (int r = check_ctx(c, 3)) return r;
    cudaStream_t s = c->stream;
    const pd::DevPtrs &d = c->d;
    const size_t N = (size_t)c->N;
    // back up the state; every trial starts from it and it is restored at the end
    PD_CUDA(cudaMemcpyAsync(d.bu, d.u, 16 * N, cudaMemcpyDeviceToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.bv, d.v[c->vcur], 16 * N, cudaMemcpyDeviceToDevice, s));
    if (d.af) PD_CUDA(cudaMemcpyAsync(d.ba, d.af, 8 * N, cudaMemcpyDeviceToDevice, s));
    else PD_CUDA(cudaMemcpyAsync(d.ba, d.a, 16 * N, cudaMemcpyDeviceToDevice, s));
    PD_CUDA(cudaMemcpyAsync(d.bbits, d.bits, 4 * N * c->wpn, cudaMemcpyDeviceToDevice, s));
    long long step0 = 0;
    int32_t st0[PD_STATUS_COUNT];
    PD_CUDA(cudaMemcpyAsync(&step0, d.step, 8, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaMemcpyAsync(st0, d.status, sizeof(st0), cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    auto restore = [&]() -> int {
        PD_CUDA(cudaMemcpyAsync(d.u, d.bu, 16 * N, cudaMemcpyDeviceToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.v[c->vcur], d.bv, 16 * N, cudaMemcpyDeviceToDevice, s));
        if (d.af) PD_CUDA(cudaMemcpyAsync(d.af, d.ba, 8 * N, cudaMemcpyDeviceToDevice, s));
        else PD_CUDA(cudaMemcpyAsync(d.a, d.ba, 16 * N, cudaMemcpyDeviceToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.bits, d.bbits, 4 * N * c->wpn, cudaMemcpyDeviceToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.step, &step0, 8, cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemcpyAsync(d.status, st0, sizeof(st0), cudaMemcpyHostToDevice, s));
        PD_CUDA(cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), s));
        PD_CUDA(cudaMemsetAsync(d.pred_ok, 0, sizeof(int), s));
        PD_CUDA(cudaStreamSynchronize(s));
        return PD_OK;
    };
    struct Cand {
        int mode, lanes, block;
    };
    std::vector<Cand> cands;
    // 1, 2, 4 or 8 threads per node for every mode
    // modes 4 and 6: the kernel graph with the rebuild kernels launched every
    // step (returning at once without the flag) instead of the conditional node
    for (int m : {0, 1, 2, 3, 4, 6}) {
        for (int lanes : {1, 2, 4, 8}) {
            if (c->prm.lanes && lanes != c->prm.lanes) continue;
            cands.push_back({m, lanes, 128});
            if (m & 1) cands.push_back({m, lanes, 256});
        }
    }
    const int kTune = 8;
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    Cand pick = {c->mode, c->kp.lanes, c->block};
    for (const Cand &cd : cands) {
        c->mode = cd.mode;
        c->kp.split = (cd.mode >> 1) & 1;
        c->kp.lanes = cd.lanes;
        c->block = cd.block;
        cudaGraphExec_t g = nullptr;
        if (capture(c, c->vcur, kTune, &g) != PD_OK) {
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        bool ok = cudaGraphLaunch(g, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
        if (int r = restore()) return r;
        if (ok) {
            ok = cudaEventRecord(e0, s) == cudaSuccess && cudaGraphLaunch(g, s) == cudaSuccess &&
                 cudaEventRecord(e1, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            int32_t st[PD_STATUS_COUNT];
            if (ok && cudaMemcpy(st, d.status, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess &&
                st[PD_STATUS_TIMEOUT] != 0)
                ok = false;
            if (int r = restore()) return r;
        }
        cudaGraphExecDestroy(g);
        cudaGetLastError();
        if (ok && ms / kTune < best) {
            best = ms / kTune;
            pick = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->mode = pick.mode;
    c->kp.split = (pick.mode >> 1) & 1;
    c->kp.lanes = pick.lanes;
    c->block = pick.block;
    if (int r = capture_all(c)) return r;
    if (report) {
        report[0] = pick.mode;
        report[1] = pick.lanes;
        report[2] = pick.block;
        report[3] = best;
    }
    return PD_OK;
}

int pd_set_path(pd_ctx *c, int mode, int lanes, int block) {
    if (int r = check_ctx(c, 3)) return r;
    if (mode < 0 || mode > 7 || (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) ||
        (block != 128 && block != 256))
        return fail(PD_EINVAL, "mode 0..7, lanes 1|2|4|8, block 128|256");
    c->mode = mode;
    c->kp.split = (mode >> 1) & 1;
    c->kp.lanes = lanes;
    c->block = block;
    return capture_all(c);
}

int pd_surrogate_setup(pd_ctx *c, int n_modes, const float *basis, const float *lambda, int judge_every, double gate,
                       double err_tol) {
    if (int r = check_ctx(c, 2)) return r;
    if (c->state != 2) return fail(PD_ESTATE, "pd_surrogate_setup must come before pd_bind_arena");
    if (c->prm.precision != PD_FP32_SPLIT) return fail(PD_EINVAL, "the surrogate runs in the FP32-split path");
    if (c->has_mat) return fail(PD_EINVAL, "the surrogate runs with one material");
    if (n_modes < 8 || n_modes > 32 || n_modes % 8 || !basis || !lambda || judge_every < 1 || !(gate > 0) ||
        !(err_tol > 0))
        return fail(PD_EINVAL,
                    "n_modes in {8,16,24,32}, basis and lambda non-null, judge_every >= 1, gate and err_tol > 0");
    const int T = c->n_tmpl, M = n_modes;
    // padded basis rows per template (2 n_t rounded up to the expansion tile)
    c->tmpl_rows.assign(T + 1, 0);
    for (int t = 0; t < T; ++t) {
        const int rows = 2 * c->tmpl_nodes[t];
        c->tmpl_rows[t + 1] = c->tmpl_rows[t] + (rows + pd::kSurExpandRows - 1) / pd::kSurExpandRows * pd::kSurExpandRows;
    }
    const size_t total = (size_t)c->tmpl_rows[T] * M;
    c->sur_basis.assign(total, 0.f);
    c->bnm_hi.assign(total, 0);
    c->bnm_lo.assign(total, 0);
    c->bmm_hi.assign(total, 0);
    c->bmm_lo.assign(total, 0);
    size_t in = 0;   // input: per template node l, x row then y row of M values
    for (int t = 0; t < T; ++t) {
        const size_t base = (size_t)c->tmpl_rows[t] * M;
        const int rp = c->tmpl_rows[t + 1] - c->tmpl_rows[t];
        for (int l = 0; l < c->tmpl_nodes[t]; ++l)
            for (int comp = 0; comp < 2; ++comp)
                for (int m = 0; m < M; ++m) {
                    const float v = basis[in++];
                    const int r = 2 * l + comp;
                    uint16_t hi, lo;
                    bf16_split(v, hi, lo);
                    c->sur_basis[base + (size_t)m * rp + r] = v;
                    c->bmm_hi[base + (size_t)m * rp + r] = hi;
                    c->bmm_lo[base + (size_t)m * rp + r] = lo;
                    c->bnm_hi[base + (size_t)r * M + m] = hi;
                    c->bnm_lo[base + (size_t)r * M + m] = lo;
                }
    }
    // network rows -> grains, and the tensor-core tiles
    c->slot_grain.assign(c->G, 0);
    int rows = 0;
    std::vector<int> slot0(T + 1, 0);
    for (int t = 0; t < T; ++t) slot0[t + 1] = slot0[t] + c->tmpl_count[t];
    for (int g = 0; g < c->G; ++g)
        if (c->g_tmpl[g] >= 0) {
            c->slot_grain[slot0[c->g_tmpl[g]] + c->g_slot[g]] = g;
            ++rows;
        }
    c->slot_grain.resize(rows);
    c->proj_work.clear();
    c->exp_work.clear();
    for (int t = 0; t < T; ++t) {
        const int rp = c->tmpl_rows[t + 1] - c->tmpl_rows[t];
        for (int s0 = 0; s0 < c->tmpl_count[t]; s0 += pd::kSurTile) {
            for (int r0 = 0, ch = 0; r0 < rp; r0 += pd::kSurChunk, ++ch) c->proj_work.push_back(make_int4(t, s0, r0, ch));
            for (int r0 = 0; r0 < rp; r0 += pd::kSurExpandRows) c->exp_work.push_back(make_int4(t, s0, r0, 0));
        }
    }
    c->sur_lambda.assign(lambda, lambda + (size_t)T * M);
    c->sur_modes = n_modes;
    c->sur_judge = judge_every;
    c->sur_gate = gate;
    c->sur_tol = err_tol;
    c->sur_cfg = true;
    return PD_OK;
}

int pd_surrogate_set_mlp(pd_ctx *c, int tmpl, pd_mlp *mlp) {
    if (int r = check_ctx(c, 3)) return r;
    if (!c->sur_cfg) return fail(PD_ESTATE, "pd_surrogate_setup was not called");
    if (tmpl < 0 || tmpl >= c->n_tmpl) return fail(PD_EINVAL, "template out of range");
    if (mlp && c->sur_modes != PD_MLP_IN)
        return fail(PD_EINVAL, "a network takes 32 modal coefficients: the surrogate needs n_modes = 32");
    pd::MlpRef ref{};
    if (mlp && pd::mlp_ref(mlp, &ref) != PD_OK) return fail(PD_ESTATE, "network not bound to device memory");
    // the linear modal part -Lambda q is applied in the network's output epilogue
    if (mlp) ref.lin = c->d.sur_lambda + (size_t)tmpl * PD_MLP_OUT;
    c->sur_mlp[tmpl] = mlp;
    // device table of the networks and the inference tiles (template, first row, end row)
    PD_CUDA(cudaMemcpyAsync(c->d.mlp_refs + tmpl, &ref, sizeof(ref), cudaMemcpyHostToDevice, c->stream));
    c->mlp_work.clear();
    for (int t = 0, row = 0; t < c->n_tmpl; row += c->tmpl_count[t], ++t)
        if (c->sur_mlp[t])
            for (int r0 = 0; r0 < c->tmpl_count[t]; r0 += pd::kSurTile)
                c->mlp_work.push_back(make_int4(t, row + r0, row + c->tmpl_count[t], 0));
    if (!c->mlp_work.empty())
        PD_CUDA(cudaMemcpyAsync(c->d.mlp_work, c->mlp_work.data(), sizeof(int4) * c->mlp_work.size(),
                                cudaMemcpyHostToDevice, c->stream));
    PD_CUDA(cudaStreamSynchronize(c->stream));
    if (!mlp) {
        // grains of a template without a network leave the surrogate
        std::vector<int32_t> act(c->G);
        PD_CUDA(cudaMemcpyAsync(act.data(), c->d.sur_active, 4 * act.size(), cudaMemcpyDeviceToHost, c->stream));
        PD_CUDA(cudaStreamSynchronize(c->stream));
        for (int g = 0; g < c->G; ++g)
            if (c->g_tmpl[g] == tmpl) act[g] = 0;
        PD_CUDA(cudaMemcpyAsync(c->d.sur_active, act.data(), 4 * act.size(), cudaMemcpyHostToDevice, c->stream));
        PD_CUDA(cudaStreamSynchronize(c->stream));
    }
    if (c->kp.sur) return capture_all(c);
    return PD_OK;
}

int pd_surrogate_enable(pd_ctx *c, int on) {
    if (int r = check_ctx(c, 3)) return r;
    if (!c->sur_cfg) return fail(PD_ESTATE, "pd_surrogate_setup was not called");
    std::vector<int32_t> act(c->G, 0);
    for (int g = 0; g < c->G; ++g) act[g] = (on && c->sur_mlp[c->g_tmpl[g]]) ? 1 : 0;
    PD_CUDA(cudaMemcpyAsync(c->d.sur_active, act.data(), 4 * act.size(), cudaMemcpyHostToDevice, c->stream));
    PD_CUDA(cudaStreamSynchronize(c->stream));
    c->kp.sur = on ? 1 : 0;
    return capture_all(c);
}

int pd_surrogate_sample(pd_ctx *c, float *q_host, float *f_host) {
    if (int r = check_ctx(c, 3)) return r;
    if (!c->sur_cfg || !c->prm.store_parts) return fail(PD_ESTATE, "sampling needs pd_surrogate_setup and store_parts");
    if (!q_host || !f_host) return fail(PD_EINVAL, "null output");
    const int sur = c->kp.sur;
    c->kp.sur = 0;                                       // full bond forces
    int r = pd_eval_forces(c);
    c->kp.sur = sur;
    if (r) return r;
    cudaStream_t s = c->stream;
    PD_CUDA(pd::launch_sur_frame(c->d, c->kp, 1, s));
    PD_CUDA(pd::launch_sur_project_cc(c->d, c->kp, nullptr, c->d.sur_qs, s));
    PD_CUDA(pd::launch_sur_project_cc(c->d, c->kp, c->d.parts, c->d.sur_fs, s));
    const size_t bytes = 4 * (size_t)c->G * c->sur_modes;
    PD_CUDA(cudaMemcpyAsync(q_host, c->d.sur_qs, bytes, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaMemcpyAsync(f_host, c->d.sur_fs, bytes, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}

int pd_surrogate_stats(pd_ctx *c, int32_t *active, float *err, float *merr, float *maxs) {
    if (int r = check_ctx(c, 3)) return r;
    if (!c->sur_cfg) return fail(PD_ESTATE, "pd_surrogate_setup was not called");
    cudaStream_t s = c->stream;
    if (active) PD_CUDA(cudaMemcpyAsync(active, c->d.sur_active, 4 * (size_t)c->G, cudaMemcpyDeviceToHost, s));
    if (err) PD_CUDA(cudaMemcpyAsync(err, c->d.sur_err, 4 * (size_t)c->G, cudaMemcpyDeviceToHost, s));
    if (merr) PD_CUDA(cudaMemcpyAsync(merr, c->d.sur_merr, 4 * (size_t)c->G, cudaMemcpyDeviceToHost, s));
    if (maxs) PD_CUDA(cudaMemcpyAsync(maxs, c->d.sur_maxs, 4 * (size_t)c->G, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}

int pd_surrogate_inspect(pd_ctx *c, float *q_host, float *y_host) {
    if (int r = check_ctx(c, 3)) return r;
    if (!c->sur_cfg || !c->kp.sur) return fail(PD_ESTATE, "the surrogate is not enabled");
    if (!q_host || !y_host) return fail(PD_EINVAL, "null output");
    if (int r = pd_eval_forces(c)) return r;
    const size_t M = (size_t)c->sur_modes, rows = c->slot_grain.size();
    std::vector<float> x(rows * M), y(rows * M);
    cudaStream_t s = c->stream;
    if (rows) {
        PD_CUDA(cudaMemcpyAsync(x.data(), c->d.sur_x, 4 * x.size(), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaMemcpyAsync(y.data(), c->d.sur_y, 4 * y.size(), cudaMemcpyDeviceToHost, s));
    }
    PD_CUDA(cudaStreamSynchronize(s));
    std::fill(q_host, q_host + (size_t)c->G * M, 0.f);
    std::fill(y_host, y_host + (size_t)c->G * M, 0.f);
    for (size_t row = 0; row < rows; ++row) {
        const int g = c->slot_grain[row];
        std::copy(x.begin() + row * M, x.begin() + (row + 1) * M, q_host + (size_t)g * M);
        std::copy(y.begin() + row * M, y.begin() + (row + 1) * M, y_host + (size_t)g * M);
    }
    return PD_OK;
}

int pd_set_timing(pd_ctx *c, int enable) {
    if (int r = check_ctx(c, 3)) return r;
    c->timing = enable ? 1 : 0;
    return PD_OK;
}

int pd_kernel_times(pd_ctx *c, double *out) {
    if (int r = check_ctx(c, 3)) return r;
    if (!out) return fail(PD_EINVAL, "null output");
    PD_CUDA(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    for (int k = 0; k < 3; ++k) {
        PD_CUDA(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        out[k] = ms;
    }
    PD_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[3]));
    out[3] = ms;
    return PD_OK;
}

int pd_info(pd_ctx *c, double *out) {
    if (int r = check_ctx(c, 0)) return r;
    if (!out) return fail(PD_EINVAL, "null output");
    out[0] = (double)c->N;
    out[1] = (double)c->col.size();
    out[2] = (double)c->G;
    out[3] = c->h_min;
    out[4] = c->Rc;
    out[5] = c->Kn;
    out[6] = c->prm.dt;
    out[7] = (double)c->steps_done;
    out[8] = (double)c->max_row;
    out[9] = (double)c->T;
    out[10] = (double)c->mode;
    out[11] = (double)(c->state >= 3 ? c->kp.lanes : (c->prm.lanes ? c->prm.lanes : 8));
    out[12] = (double)c->block;
    out[13] = (double)c->n_agg;
    out[14] = (double)c->n_tmpl;
    return PD_OK;
}

}  // extern "C"
