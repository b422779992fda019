// pd_device.cuh -- device code shared by the multi-kernel and the persistent
// step paths: per-node phase functions (displacement update, forces) and the
// contact / wall / precision helpers they use.
#pragma once

#include "pd_internal.h"
#include "peridem.h"

namespace pd {

// Loads of state that other blocks write in an earlier phase of the same
// persistent launch.  The persistent kernel's grid barrier orders them: every
// block fences its writes before it arrives and fences again once it has seen
// the new generation (the pattern of a cooperative grid synchronisation), so
// ordinary loads after the barrier, L1 included, see the other blocks' writes
// (the persistent-vs-graph tests compare FP64 trajectories bit for bit).
// PERSIST is kept to mark those loads.
template <bool PERSIST, class T>
__device__ __forceinline__ T ldm(const T *p) {
    return *p;
}

// ---------------------------------------------------------------------------
// contact search grid

// Square cells of side >= R_c hashed (with the aggregate id) into T buckets
// (T a power of two >= 2N): every pair closer than R_c lies in the 3x3 cell
// block around either node; aliasing cells only add candidates, which the
// distance test rejects.
// Hash-grid cell index of a coordinate (inv_cell = 1 / cell side).  Only the
// binning kernel calls this; the force kernels read the stored cells.
__device__ __forceinline__ int cell_coord_f(float x, float inv_cell) {
    float f = floorf(x * inv_cell);
    if (!(f > -1048576.0f)) return -1048576;  // also catches NaN
    if (f > 1048576.0f) return 1048576;
    return (int)f;
}

__device__ __forceinline__ int cell_coord(double x, double origin, double inv_cell) {
    double f = floor((x - origin) * inv_cell);
    if (!(f > -1048576.0)) return -1048576;  // also catches NaN
    if (f > 1048576.0) return 1048576;
    return (int)f;
}

constexpr unsigned kHashX = 73856093u, kHashY = 19349663u, kHashA = 83492791u;

__device__ __forceinline__ unsigned cell_bucket(int cx, int cy, int agg, unsigned T) {
    return ((unsigned)cx * kHashX ^ (unsigned)cy * kHashY ^ (unsigned)agg * kHashA) & (T - 1u);
}

// ---------------------------------------------------------------------------
// materials (Sec. 4.1): contact between bulk moduli k1, k2 uses the harmonic
// mean 2 k1 k2 / (k1 + k2) in K_n = 18 k / (pi eps_c^5); damping the harmonic
// mean of the two densities; equal values give the value itself
__device__ __forceinline__ double harmonic64(double a, double b) { return a == b ? a : 2.0 * a * b / (a + b); }
// (float: the contact stiffnesses reach 1e25, so a * b would overflow; a * (b / (a + b)) does not)
__device__ __forceinline__ float harmonic32(float a, float b) { return a == b ? a : 2.0f * a * (b / (a + b)); }

// ---------------------------------------------------------------------------
// FP64 laws

// Normal damping (Sec. 4.3, Kelvin-Voigt: -beta_d V_x V_y (v(x,y).e) e with
// beta_d = 2 r_d sqrt(K_n rho_d / V_y)) and regularised Coulomb friction
// (Sec. 4.2: slip -mu |F_r| v_perp/|v_perp| when |v_perp| > v_thr =
// mu |F_r| dt / (rho V_x), else the sticking force -(rho V_x / dt) v_perp).
// e points from x to y, (vrx, vry) = v(x) - v(y), Fr = |F_r|, Vy the partner
// volume (|S_l| for a wall); rho_d the pair's density (the harmonic mean of
// the two grains' densities), rho the density of x.  Adds to (fx, fy).
__device__ __forceinline__ void damping_friction64(const KParams &k, double Kn, double rho_d, double rho,
                                                   double ex, double ey, double vrx, double vry, double Fr, double Vx,
                                                   double Vy, double &fx, double &fy) {
    double beta = 2.0 * k.rd * sqrt(Kn * rho_d / Vy);
    double vn = vrx * ex + vry * ey;
    double cd = beta * Vx * Vy * vn;
    double Fdx = -cd * ex, Fdy = -cd * ey;
    double vtx = vrx - vn * ex, vty = vry - vn * ey;
    double vt = sqrt(vtx * vtx + vty * vty);
    double vthr = k.mu * Fr * k.dt / (rho * Vx);
    double c = (vt > vthr) ? (k.mu * Fr / vt) : (rho * Vx / k.dt);
    double Ffx = -c * vtx, Ffy = -c * vty;
    fx += Fdx + Ffx;
    fy += Fdy + Ffy;
}

// Taylor coefficients, about theta = 0, of the shape functions of the wall
// contact regions (Sec. 4.5), evaluated by the C++ front end at compile time:
//   h1(theta) / theta^3 = sum_{k>=1} H_k theta^(2k-2),
//       H_1 = 2/3, H_{k+1} = -4 H_k / ((2k+2)(2k+3))  (theta - sin theta cos theta);
//   g(theta) / theta^5 = sum_{k>=2} G_k theta^(2k-4),  G_k = a_k - b_k - e_k, the
//       terms of 3^(2k+1)/6, 4^k and 1/2 over (2k+1)! with alternating signs
//       (h1 - 2/3 sin^3 theta);
//   f(x) / x^3 = sum_{k>=1} F_k x^(2k-2),  F_1 = 1/6, F_{k+1} = -F_k / ((2k+2)(2k+3))
//       (x - sin x).
// Below theta = 0.3 (x = 0.5) nine, nine and eight terms leave a tail below
// 1e-18 of the sum.
__host__ __device__ constexpr double seg_h1_coef(int k) {
    double c = 4.0 / 6.0;
    for (int m = 1; m < k; ++m) c *= -4.0 / ((2.0 * m + 2.0) * (2.0 * m + 3.0));
    return c;
}
__host__ __device__ constexpr double seg_g_coef(int k) {
    double a = 243.0 / 6.0 / 120.0, b = 16.0 / 120.0, e = 0.5 / 120.0;
    for (int m = 2; m < k; ++m) {
        const double den = (2.0 * m + 2.0) * (2.0 * m + 3.0);
        a *= -9.0 / den;
        b *= -4.0 / den;
        e *= -1.0 / den;
    }
    return a - b - e;
}
__host__ __device__ constexpr double seg_f_coef(int k) {
    double c = 1.0 / 6.0;
    for (int m = 1; m < k; ++m) c *= -1.0 / ((2.0 * m + 2.0) * (2.0 * m + 3.0));
    return c;
}
constexpr int kSegH1Terms = 9, kSegGTerms = 9, kSegFTerms = 8;

// Horner evaluation of sum_{k=K..KMAX} C_k t2^(k-K0) with the coefficients above
// (WHICH: 0 = H, 1 = G, 2 = F), one FMA per term: a dependent chain of FMAs
// instead of the recurrence's chain of divisions, which at GB300's FP64 rate
// held a whole step back on the one node that touched a wall.
template <int WHICH, int K, int KMAX>
__device__ __forceinline__ double seg_horner(double t2) {
    constexpr double c = WHICH == 0 ? seg_h1_coef(K) : (WHICH == 1 ? seg_g_coef(K) : seg_f_coef(K));
    if constexpr (K == KMAX) return c;
    else return fma(seg_horner<WHICH, K + 1, KMAX>(t2), t2, c);
}

// Circular segment of B_R(p) beyond a line at distance d < R (Sec. 4.5).
// With theta = acos(d/R) = atan2(sqrt(R^2 - d^2), d) the paper's closed forms
// read |S| = R^2 (theta - sin theta cos theta) and
// R - |c - p| = R (h1 - 2/3 sin^3 theta) / h1; both are evaluated without
// cancellation (Taylor series in theta below 0.3), because the printed
// pi R^2/2 - R^2 asin(d/R) - d sqrt(R^2 - d^2) loses all digits as d -> R.
__device__ __forceinline__ void wall_segment_stable(double d, double R, double &area, double &gap) {
    const double y = sqrt((R - d) * (R + d));
    const double th = atan2(y, d);
    double h1, g;
    if (th < 0.3) {
        const double t2 = th * th;
        h1 = (th * t2) * seg_horner<0, 1, kSegH1Terms>(t2);
        g = (t2 * t2 * th) * seg_horner<1, 2, kSegGTerms + 1>(t2);
    } else {
        // sin and cos of the rounded angle itself: with sqrt(R^2 - d^2) / R and
        // d / R instead, the cancellation in g (about 30-fold at theta = 0.3)
        // doubles the rounding error of the gap
        double sn, cs;
        sincos(th, &sn, &cs);
        h1 = th - sn * cs;
        g = h1 - (2.0 / 3.0) * sn * sn * sn;
    }
    area = R * R * h1;
    gap = R * g / h1;
}

// Corner region S_li cap S_lj (Sec. 4.5) in the frame x -> wall i, y -> wall j:
// {x >= di, y >= dj, |.| <= R}, split into the triangle Q P1 P2 (Q = (di, dj),
// P1 = (b, dj), P2 = (di, c) on the circle) and the circular segment cut by
// the chord P1 P2, so the area and the centroid stay accurate as the corner
// point approaches the circle (the paper's polar integrals cancel there).
__device__ __forceinline__ void corner_region_stable(double di, double dj, double R, double &area, double &cx,
                                                     double &cy) {
    const double b = sqrt((R - dj) * (R + dj)), c = sqrt((R - di) * (R + di));
    const double w = (R - di) * (R + di) - dj * dj;
    const double bmi = w / (b + di), cmj = w / (c + dj);
    const double T = 0.5 * bmi * cmj;
    const double dth = atan2(b * cmj + dj * bmi, b * di + dj * c);
    double f;
    if (dth < 0.5) {
        const double t2 = dth * dth;
        f = (dth * t2) * seg_horner<2, 1, kSegFTerms>(t2);
    } else {
        f = dth - sin(dth);
    }
    const double Sg = 0.5 * R * R * f;
    const double mx = b + di, my = dj + c, ml = sqrt(mx * mx + my * my);
    const double s2 = sin(0.5 * dth);
    const double sd = (dth > 0.0) ? R * (4.0 * s2 * s2 * s2) / (3.0 * f) : R;
    const double A = Sg + T;
    area = A;
    cx = (Sg * (sd * mx / ml) + T * ((di + b + di) / 3.0)) / A;
    cy = (Sg * (sd * my / ml) + T * ((dj + dj + c) / 3.0)) / A;
}

// Wall contact (Sec. 4.5, eq:wall-repulsive, eq:wall-total) of a node at p
// with velocity v, volume Vx, contact stiffness Kn and density rho (its own
// material: a wall is rigid) against the four walls of its aggregate at
// time t (position w0 + v_w t, normal velocity v_w).  The repulsion of each
// wall uses the circular segment S_l of B_Rc(p) beyond it; corners subtract
// the S_li cap S_lj term (inclusion-exclusion); friction and damping follow by
// substituting e -> e^l, V_y -> |S_l|, p(y) -> c_l.  A node past a wall is
// treated as touching it and counted in status[PD_STATUS_PENETRATION].
__device__ __forceinline__ void wall_terms64(const KParams &k, const AggParams &A, double Kn, double rho, double t,
                                             double px, double py, double vx, double vy, double Vx,
                                             double (&single)[4][2], double (&corner)[4][2], int *status) {
    const double Rc = A.Rc;
    double d[4], ex[4], ey[4];
    d[0] = px - (A.w0[0] + A.wv[0] * t); ex[0] = -1.0; ey[0] = 0.0;
    d[1] = (A.w0[1] + A.wv[1] * t) - px; ex[1] = 1.0;  ey[1] = 0.0;
    d[2] = py - (A.w0[2] + A.wv[2] * t); ex[2] = 0.0;  ey[2] = -1.0;
    d[3] = (A.w0[3] + A.wv[3] * t) - py; ex[3] = 0.0;  ey[3] = 1.0;
    bool near = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        single[l][0] = single[l][1] = corner[l][0] = corner[l][1] = 0.0;
        if (d[l] < 0.0) {
            if (status) atomicAdd(&status[PD_STATUS_PENETRATION], 1);
            d[l] = 0.0;
        }
        near |= d[l] < Rc;
    }
    if (!near) return;
    for (int l = 0; l < 4; ++l) {
        if (!(d[l] < Rc)) continue;
        double Ar, gap;
        wall_segment_stable(d[l], Rc, Ar, gap);
        if (!(Ar > 0.0) || !(gap > 0.0)) continue;
        double Fr = Kn * gap * Vx * Ar;
        double wvx = (l < 2) ? A.wv[l] : 0.0, wvy = (l < 2) ? 0.0 : A.wv[l];
        double gx = -Fr * ex[l], gy = -Fr * ey[l];
        damping_friction64(k, Kn, rho, rho, ex[l], ey[l], vx - wvx, vy - wvy, Fr, Vx, Ar, gx, gy);
        single[l][0] = gx;
        single[l][1] = gy;
    }
    for (int c = 0; c < 4; ++c) {
        const int i = c >> 1, j = 2 + (c & 1);  // (x_lo|x_hi) x (y_lo|y_hi)
        double di = d[i], dj = d[j];
        if (!(sqrt(di * di + dj * dj) < Rc)) continue;
        double Ar, lx, ly;
        corner_region_stable(di, dj, Rc, Ar, lx, ly);
        if (!(Ar > 0.0)) continue;
        double cx = lx * ex[i] + ly * ex[j], cy = lx * ey[i] + ly * ey[j];
        double cd = sqrt(cx * cx + cy * cy);
        if (!(cd < Rc) || !(cd > 0.0)) continue;
        double ux = cx / cd, uy = cy / cd;
        double Fr = Kn * (Rc - cd) * Vx * Ar;
        double gx = -Fr * ux, gy = -Fr * uy;
        damping_friction64(k, Kn, rho, rho, ux, uy, vx - A.wv[i], vy - A.wv[j], Fr, Vx, Ar, gx, gy);
        corner[c][0] = gx;
        corner[c][1] = gy;
    }
}

// Wall force on a node at (px, py) with velocity (vx, vy) and volume Vx:
// eq:wall-total, the walls' own segments in order minus the corner terms.
__device__ __forceinline__ void wall_force64(const KParams &k, const AggParams &A, double Kn, double rho, double t,
                                             double px, double py, double vx, double vy, double Vx, double &Fx_out,
                                             double &Fy_out, int *status) {
    double single[4][2], corner[4][2];
    wall_terms64(k, A, Kn, rho, t, px, py, vx, vy, Vx, single, corner, status);
    double Fx = 0.0, Fy = 0.0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        Fx += single[l][0];
        Fy += single[l][1];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        Fx -= corner[c][0];
        Fy -= corner[c][1];
    }
    Fx_out = Fx;
    Fy_out = Fy;
}

// ---------------------------------------------------------------------------
// float-float helpers of the FP32-split path

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |d|^2 of d = (dxh + dxl, dyh + dyl) as a float-float pair (hi, lo).  The low
// parts are not small against one ulp of the high parts (they carry the
// position bits below the float grid of the box coordinates), so the square
// keeps dxl^2 + dyl^2 as well as the cross terms.
__device__ __forceinline__ void len2_ff(float dxh, float dxl, float dyh, float dyl, float &hi, float &lo) {
    float px, ex, py, ey, s, es;
    two_prod(dxh, dxh, px, ex);
    two_prod(dyh, dyh, py, ey);
    two_sum(px, py, s, es);
    float r = es + (ex + ey) + (2.f * (dxh * dxl + dyh * dyl) + (dxl * dxl + dyl * dyl));
    hi = __fadd_rn(s, r);
    lo = __fsub_rn(r, __fsub_rn(hi, s));
}

// (ah + al) - (bh + bl) rounded to float; the high-part difference is exact
// when the two values are within a factor of two of each other.
__device__ __forceinline__ float ff_diff(float ah, float al, float bh, float bl) {
    return __fsub_rn(ah, bh) + (al - bl);
}

// Square root and quotient of the bond loop by the approximate special-function
// instructions (relative error about 2^-22) instead of the correctly rounded
// sequences: the FP32-split bond force carries a 1e-5 tolerance, and stretches
// within 1e-4 of the critical one are re-decided in FP64 after the loop, so
// the break decisions do not change.  (The operands here are far from the
// ranges where __fdividef returns 0.)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void damping_friction32(float rd, float Kn, float rho_d, float rho, float dt, float mu,
                                                   float ex, float ey, float vrx, float vry, float Fr, float Vx,
                                                   float Vy, float &fx, float &fy) {
    // sqrt(K_n) sqrt(rho_d / V_y): K_n of GPa-range materials (~1e28) times a
    // density over a node volume would overflow float
    float beta = 2.0f * rd * sqrtf(Kn) * sqrtf(rho_d / Vy);
    float vn = vrx * ex + vry * ey;
    float cd = beta * Vx * Vy * vn;
    float vtx = vrx - vn * ex, vty = vry - vn * ey;
    float vt = sqrtf(vtx * vtx + vty * vty);
    float vthr = mu * Fr * dt / (rho * Vx);
    float c = (vt > vthr) ? (mu * Fr / vt) : (rho * Vx / dt);
    fx += -cd * ex - c * vtx;
    fy += -cd * ey - c * vty;
}

// Float Horner evaluation of the wall-region series (coefficients as above).
template <int WHICH, int K, int KMAX>
__device__ __forceinline__ float seg_horner_f(float t2) {
    constexpr float c = (float)(WHICH == 0 ? seg_h1_coef(K) : (WHICH == 1 ? seg_g_coef(K) : seg_f_coef(K)));
    if constexpr (K == KMAX) return c;
    else return fmaf(seg_horner_f<WHICH, K + 1, KMAX>(t2), t2, c);
}

// Wall force of the FP32-split path (Sec. 4.5, eq:wall-total): the same terms
// as wall_force64, with the single-wall segments in float.  Each wall distance
// d is formed in FP64 and the segment is evaluated from R_c - d and R_c + d,
// each rounded once to float, so the small-angle quantities keep float's
// relative precision (the gap to about 1e-6 relative).  The small-angle series
// covers theta < 0.6 (six and eight terms leave a tail below 1e-8), where
// the closed form's cancellation in g stays below tenfold.  A node within R_c
// of a corner takes the FP64 terms.  Knf, rhof: the node's own contact
// stiffness and density as floats; Kn, rho, V: the same in FP64.
__device__ __forceinline__ void wall_force32(const KParams &k, const AggParams &A, float Knf, float rhof, double Kn,
                                             double rho, double t, double px, double py, double vx, double vy,
                                             double V, double &Fx_out, double &Fy_out, int *status) {
    const double Rc = A.Rc;
    double d[4];
    d[0] = px - (A.w0[0] + A.wv[0] * t);
    d[1] = (A.w0[1] + A.wv[1] * t) - px;
    d[2] = py - (A.w0[2] + A.wv[2] * t);
    d[3] = (A.w0[3] + A.wv[3] * t) - py;
    bool near = false, corner = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) near |= d[l] < Rc;
    if (!near) {
        Fx_out = Fy_out = 0.0;
        return;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double di = fmax(d[c >> 1], 0.0), dj = fmax(d[2 + (c & 1)], 0.0);
        corner |= di * di + dj * dj < Rc * Rc;
    }
    if (corner) {
        wall_force64(k, A, Kn, rho, t, px, py, vx, vy, V, Fx_out, Fy_out, status);
        return;
    }
    const float Rf = (float)Rc, Vx = (float)V, rd = k.rdf, dt = k.dtf, mu = k.muf;
    float Fx = 0.f, Fy = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (d[l] < 0.0) {
            if (status) atomicAdd(&status[PD_STATUS_PENETRATION], 1);
            d[l] = 0.0;
        }
        if (!(d[l] < Rc)) continue;
        const float e = (float)(Rc - d[l]), sp = (float)(Rc + d[l]), df = (float)d[l];
        const float y = sqrtf(e * sp);
        const float th = atan2f(y, df);
        float h1, g;
        if (th < 0.6f) {
            const float t2 = th * th;
            h1 = (th * t2) * seg_horner_f<0, 1, 6>(t2);
            g = (t2 * t2 * th) * seg_horner_f<1, 2, 9>(t2);
        } else {
            float sn, cs;
            sincosf(th, &sn, &cs);
            h1 = th - sn * cs;
            g = h1 - (2.0f / 3.0f) * sn * sn * sn;
        }
        const float Ar = Rf * Rf * h1, gap = Rf * g / h1;
        // (a region below 1e-30 R_c^2 carries no force float can represent)
        if (!(h1 > 1e-30f) || !(gap > 0.f)) continue;
        const float Fr = ((Knf * gap) * Vx) * Ar;
        const float ex = (l == 0) ? -1.f : (l == 1 ? 1.f : 0.f), ey = (l == 2) ? -1.f : (l == 3 ? 1.f : 0.f);
        const float vrx = (float)(vx - ((l < 2) ? A.wv[l] : 0.0)), vry = (float)(vy - ((l < 2) ? 0.0 : A.wv[l]));
        float gx = -Fr * ex, gy = -Fr * ey;
        damping_friction32(rd, Knf, rhof, rhof, dt, mu, ex, ey, vrx, vry, Fr, Vx, Ar, gx, gy);
        Fx += gx;
        Fy += gy;
    }
    Fx_out = (double)Fx;
    Fy_out = (double)Fy;
}

// ---------------------------------------------------------------------------
// plain FP64 path on GB300's narrow FP64 pipe
//
// GB300 issues FP64 at 2 lanes per SM cycle, against 64 for 32-bit integer and
// 128 for FP32 arithmetic.  The FP64 bond loop therefore keeps in FP64 only the
// operations whose rounding the stretch s = (L - |xi|) / |xi| depends on (the
// coordinate differences, |d|^2 and L - |xi|, which cancels), takes the correctly
// rounded L = sqrt(|d|^2) from integer and FP32 arithmetic, and forms the rest of
// the bond force in float-float arithmetic (about 2^-47 relative), far inside the
// 1e-12 per-step force tolerance of the path.

// Float-float (hi + lo) of a double from its bits: hi holds the top 24
// significand bits, lo the next 24 (the last five are dropped: 2^-48 relative).
// Integer operations and one conversion of a 24-bit integer, no FP64
// instruction.  Magnitudes below 2^-79 lose lo, below 2^-126 become 0.
__device__ __forceinline__ void dbl_to_ff(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 897) {
        hi = lo = 0.f;
        return;
    }
    if (e > 1150) {                     // beyond the float range, inf or NaN: carried as inf or NaN
        hi = lo = e == 2047 && (b & 0xFFFFFFFFFFFFFull) ? __int_as_float(0x7FC00000) : __uint_as_float(sign | 0x7F800000u);
        return;
    }
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
    // fraction bits 28..5 carry the weight 2^(e - 1023 - 47)
    const float scale = e > 943 ? __uint_as_float((unsigned)(e - 943) << 23) : 0.f;
    lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn((unsigned)(m >> 5) & 0xFFFFFFu) * scale));
}

// Correctly rounded (to nearest) square root of a positive normal double, in
// integer and FP32 arithmetic.  With x = M 2^(E - 52), M the 53-bit significand,
// let N = M 2^(52 + (E & 1)); then sqrt(x) = sqrt(N) 2^(floor(E / 2) - 52) with
// sqrt(N) in [2^52, 2^53), and the result's significand is Q = round(sqrt(N)).
//  1. y = sqrt(A), A = N 2^-104 in [1, 4): the FP32 reciprocal square root, one
//     FP32 Newton step, then one Newton step with the float-float residual
//     A - y^2 (relative error below 2^-44): Y = y 2^52 is within 2^9 of sqrt(N).
//  2. Newton's correction in integers: Q = Y + round((N - Y^2) / (2 Y)), with the
//     residual exact in 128 bits (|N - Y^2| < 2^63) and its top bits converted,
//     leaves |Q - sqrt(N)| < 1.
//  3. Exact decision from R = N - Q^2 (|R| < 2^55): Q - 1 if R < 0 (then
//     R += 2 Q - 1), and round up when R > Q, since (Q + 1/2)^2 = Q^2 + Q + 1/4
//     and sqrt(N) is never a half-integer.
// The result equals the IEEE square root (checked against the hardware's on
// random inputs by pd_check_sqrt).
__device__ __forceinline__ double sqrt_rn_int(double x) {
    const unsigned long long D = (unsigned long long)__double_as_longlong(x);
    if (D == 0ull || (D >> 52) >= 0x7FFull) return x;   // 0, inf, NaN (negative inputs do not occur)
    const int E = (int)(D >> 52) - 1023;
    const unsigned long long M = (D & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int odd = E & 1;
    const int eL = (E - odd) / 2;
    // A = M 2^(odd - 52) as a float-float: the top 24 bits and the remaining 29
    const float a_hi = __uint_as_float(((unsigned)(127 + odd) << 23) | (unsigned)((M >> 29) & 0x7FFFFFu));
    const float a_lo = __uint2float_rn((unsigned)(M & 0x1FFFFFFFu)) * __uint_as_float((unsigned)(75 + odd) << 23);
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a_hi));
    r = r * fmaf(-0.5f * a_hi, r * r, 1.5f);
    const float y0 = a_hi * r;
    float p, pe;
    two_prod(y0, y0, p, pe);
    const float res = (__fsub_rn(a_hi, p) - pe) + a_lo;     // A - y0^2
    const unsigned yb = __float_as_uint(y0);
    const int ey = (int)(yb >> 23) - 127;                   // -1, 0 or 1
    long long Y = (long long)((yb & 0x7FFFFFu) | 0x800000u) << (29 + ey);
    Y += (long long)__float2int_rn(res * (0.5f * r) * 4503599627370496.0f);   // + (A - y0^2) / (2 y0) 2^52
    // R = N - Y^2 in 128 bits (hi:lo)
    const unsigned long long n_lo = M << (52 + odd), n_hi = M >> (12 - odd);
    const unsigned long long yy_lo = (unsigned long long)Y * (unsigned long long)Y;
    const unsigned long long yy_hi = __umul64hi((unsigned long long)Y, (unsigned long long)Y);
    const unsigned long long r_lo = n_lo - yy_lo;
    const unsigned long long r_hi = n_hi - yy_hi - (n_lo < yy_lo ? 1ull : 0ull);
    // R / 2^32 fits 32 bits (|R| < 2^63); its dropped low bits move R / (2 Y) by < 2^-21
    // (32-bit conversions only: GB300 converts 64-bit integers at the FP64 rate)
    const float rf = __int2float_rn((int)(long long)((r_hi << 32) | (r_lo >> 32))) * 4294967296.0f;
    long long Q = Y + __float2int_rn(rf * (r * 1.1102230246251565e-16f));   // R / (2 Y), 1 / (2 Y) = r 2^-53
    long long R = (long long)(n_lo - (unsigned long long)Q * (unsigned long long)Q);
    if (R < 0) {
        Q -= 1;
        R += 2 * Q + 1;
    }
    Q += R > Q ? 1 : 0;
    return __longlong_as_double(((long long)(eL + 1023) << 52) + (Q - (1ll << 52)));
}

// float-float arithmetic (Dekker / Knuth error-free transformations with FMA)
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
// 1 / a to about 2^-46 relative: the approximate reciprocal and two Newton
// steps x + x (1 - a x) with the residual formed in float-float.
__device__ __forceinline__ ff ff_rcp(ff a) {
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(a.hi));
    float t = fmaf(-a.hi, x, 1.0f) - a.lo * x;
    x = fmaf(x, t, x);
    t = fmaf(-a.hi, x, 1.0f) - a.lo * x;
    const float c = x * t;
    const float h = __fadd_rn(x, c);
    return {h, __fsub_rn(c, __fsub_rn(h, x))};
}
__device__ __forceinline__ ff to_ff(double x) {
    ff r;
    dbl_to_ff(x, r.hi, r.lo);
    return r;
}

// Exact widening of a float to a double by bit operations: a conversion
// instruction occupies GB300's 2-lane FP64 pipe like an FP64 operation.
// Subnormal floats become zero; inf and NaN stay inf and NaN.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if (e == 0u) return __longlong_as_double((long long)sign);
    const unsigned long long ed = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}
// The float part of a double's float-float split (its top 24 significand bits).
__device__ __forceinline__ float d2f_hi_bits(double x) {
    float hi, lo;
    dbl_to_ff(x, hi, lo);
    return hi;
}

// ---------------------------------------------------------------------------
// per-node phases

// The persistent kernel's current displacement and positions: the buffers of
// its step's parity, set by thread 0 of every block at the start of the step
// (one kernel body serves both parities).
__shared__ double2 *s_cur_u;
__shared__ float4 *s_cur_pq;

// Current displacement / positions of the kernel: the device pointers' own on
// the multi-kernel path (the host sets them per launch), the persistent
// kernel's per-step choice otherwise.
template <bool PERSIST>
__device__ __forceinline__ double2 *cur_u(const DevPtrs &d) {
    if constexpr (PERSIST) return s_cur_u;
    else return d.u;
}
template <bool PERSIST>
__device__ __forceinline__ float4 *cur_pq(const DevPtrs &d) {
    if constexpr (PERSIST) return s_cur_pq;
    else return d.pq;
}

// Shifted position xs + u of node i as a float-float pair into q_out[i], and
// the rebuild test: the displacement since the last rebuild from the float-float
// positions (error ~1e-7 of the displacement, far below the trigger's margin).
template <bool PERSIST>
__device__ __forceinline__ bool position32(const DevPtrs &d, const KParams &k, int i, double2 u, float4 *q_out) {
    const double2 xs = __ldg(&d.xs[i]);
    const double qx = xs.x + u.x, qy = xs.y + u.y;
    // float-float split by bit operations (no FP64-pipe conversions)
    float4 q;
    dbl_to_ff(qx, q.x, q.z);
    dbl_to_ff(qy, q.y, q.w);
    q_out[i] = q;
    const float4 r = ldm<PERSIST>(&d.sref[i]);
    const float ex = __fsub_rn(q.x, r.x) + (q.z - r.z), ey = __fsub_rn(q.y, r.y) + (q.w - r.w);
    return !(ex * ex + ey * ey <= k.dmax2);
}

// FP32-split displacement update of node i (Algorithm 1): u += dt v + dt^2/2 a
// with the FP32 acceleration widened exactly, written to u_out, and its shifted
// position as a float-float pair to q_out; true when the node has moved
// kSkinTrigger * skin since the last rebuild.  The persistent kernel's velocity
// update calls it for the next step with the same operands that the update
// phase would load, so both give the same bits.
template <bool PERSIST>
__device__ __forceinline__ bool advance_node32(const DevPtrs &d, const KParams &k, int i, double2 u, double2 v,
                                               float ax, float ay, double2 *u_out, float4 *q_out) {
    u.x = fma(k.dt, v.x, fma(k.half_dt2, f2d_bits(ax), u.x));
    u.y = fma(k.dt, v.y, fma(k.half_dt2, f2d_bits(ay), u.y));
    u_out[i] = u;
    return position32<PERSIST>(d, k, i, u, q_out);
}

// Algorithm 1: u <- u + dt v + dt^2/2 a (when advancing) and the positions.
// Returns true when the node has moved farther than kSkinTrigger * skin since
// the last rebuild of the candidate lists (or its position is not finite).
//  * FP64 path: p = X + u in FP64, every operation rounded as written (no FMA).
//  * FP32 split: u advances in FP64 with fused multiply-adds; the shifted
//    position q = (X + shift) + u is kept only as a float-float pair (the FP64
//    p is formed where it is needed: walls, near-threshold bonds, readout).
//    GB300 issues FP64 at 2 lanes per SM cycle, so the node update is written
//    with as few FP64 operations as the FP64 state allows.
// With advance, u^(n-1) is read from ub[vin] and u^n written to d.u
// (= ub[vin ^ 1]); without, only the positions of d.u.
template <bool PERSIST>
__device__ __forceinline__ bool predict_node(const DevPtrs &d, const KParams &k, int i, int vin, int advance) {
    double2 *const uc = cur_u<PERSIST>(d);
    double2 u = advance ? ldm<PERSIST>(&d.ub[vin][i]) : ldm<PERSIST>(&uc[i]);
    const float dmax2 = k.dmax2;
    if (d.pq) {
        if (advance) {
            const double2 v = ldm<PERSIST>(&d.v[vin][i]);
            const float2 a = ldm<PERSIST>(&d.af[i]);       // FP32 acceleration, widened exactly
            return advance_node32<PERSIST>(d, k, i, u, v, a.x, a.y, uc, cur_pq<PERSIST>(d));
        }
        return position32<PERSIST>(d, k, i, u, cur_pq<PERSIST>(d));
    }
    if (advance) {
        // explicit round-to-nearest operations: never contracted into FMAs
        const double2 v = ldm<PERSIST>(&d.v[vin][i]), a = ldm<PERSIST>(&d.a[i]);
        u.x = __dadd_rn(__dadd_rn(u.x, __dmul_rn(k.dt, v.x)), __dmul_rn(k.half_dt2, a.x));
        u.y = __dadd_rn(__dadd_rn(u.y, __dmul_rn(k.dt, v.y)), __dmul_rn(k.half_dt2, a.y));
        uc[i] = u;
    }
    const double2 X = __ldg(&d.X[i]);
    d.p[i] = make_double2(__dadd_rn(X.x, u.x), __dadd_rn(X.y, u.y));
    // |u - u at the last rebuild| in float: its rounding (1e-7 |u|) is far below the margin
    // (1/2 - kSkinTrigger) skin of the trigger
    const float4 r = ldm<PERSIST>(&d.sref[i]);
    const float ex = d2f_hi_bits(u.x) - r.x, ey = d2f_hi_bits(u.y) - r.y;
    return !(ex * ex + ey * ey <= dmax2);
}

// FP64 position X + u of node i (the FP32-split path does not store p).
template <bool PERSIST>
__device__ __forceinline__ double2 position64(const DevPtrs &d, int i) {
    const double2 X = __ldg(&d.X[i]), u = ldm<PERSIST>(&cur_u<PERSIST>(d)[i]);
    return make_double2(__dadd_rn(X.x, u.x), __dadd_rn(X.y, u.y));
}

// Rebuild, step 1: hash-grid cell and bucket of node i at its current
// position, counted into its bucket.
template <bool PERSIST>
__device__ __forceinline__ void bin_node(const DevPtrs &d, const KParams &k, int i) {
    const int ag = __ldg(&d.g_agg[__ldg(&d.grain[i])]);
    const AggParams &A = d.agg[ag];
    int cx, cy;
    if (d.pq) {
        // FP32-split: the cell from the shifted float position (error below 1e-3
        // cell; the cells of this path are 0.4 % wider to absorb it)
        const float4 q = ldm<PERSIST>(&cur_pq<PERSIST>(d)[i]);
        cx = cell_coord_f((q.x - A.oxs) + q.z, A.inv_cell_f);
        cy = cell_coord_f((q.y - A.oys) + q.w, A.inv_cell_f);
    } else {
        const double2 p = ldm<PERSIST>(&d.p[i]);
        cx = cell_coord(p.x, A.ox, A.inv_cell);
        cy = cell_coord(p.y, A.oy, A.inv_cell);
    }
    d.cell[i] = make_int2(cx, cy);
    unsigned b = cell_bucket(cx, cy, ag, k.T);
    d.key[i] = (int)b;
    atomicAdd(&d.count[b], 1);
}

// L2 prefetch of a byte range, one 128-byte line per index of a grid stride g
// that counts on from range to range (a hint: it never faults, and every
// address issued lies inside the range).
__device__ __forceinline__ void prefetch_range(const void *p, size_t bytes, long long &g, long long nt) {
    const long long lines = (long long)((bytes + 127) >> 7);
    for (; g < lines; g += nt) asm volatile("prefetch.global.L2 [%0];" ::"l"((const char *)p + (g << 7)));
    g -= lines;
}

// The read-only arrays of the force phase (CSR rows, grain ids, broken-bond
// words, candidate-list lengths and first rows, bond columns, per-grain and
// per-aggregate constants) and the lines of the step counter, rebuild flag,
// status words and grid barrier, prefetched into L2 by all threads of a grid
// before the displacement update: their DRAM latency then overlaps the update
// instead of lengthening the dependent load chains that follow.  Off
// (k.pf_bonds = 0) when the arrays do not fit comfortably in L2.
__device__ __forceinline__ void prefetch_force_inputs(const DevPtrs &d, const KParams &k, long long t, long long nt) {
    if (k.pf_bonds <= 0) return;
    const size_t N = (size_t)k.N, nb = (size_t)k.pf_bonds, G = (size_t)k.G;
    long long g = t;
    prefetch_range(d.step, sizeof(long long), g, nt);
    prefetch_range(d.rebuild, sizeof(int), g, nt);
    prefetch_range(d.status, sizeof(int) * PD_STATUS_COUNT, g, nt);
    prefetch_range(d.bar, 2 * sizeof(unsigned), g, nt);
    prefetch_range(d.g_agg, 4 * G, g, nt);
    prefetch_range(d.agg, sizeof(AggParams) * (size_t)k.n_agg, g, nt);
    if (d.pq) {
        prefetch_range(d.gq, 16 * G, g, nt);
        prefetch_range(d.gc, 16 * G, g, nt);
        prefetch_range(d.g_invm, 8 * G, g, nt);
        if (k.mat) prefetch_range(d.g_kf, 4 * G, g, nt);
    } else {
        prefetch_range(d.g_cw, 8 * G, g, nt);
        prefetch_range(d.g_s0, 8 * G, g, nt);
        prefetch_range(d.g_eps, 8 * G, g, nt);
        if (k.mat) {
            prefetch_range(d.g_rho, 8 * G, g, nt);
            prefetch_range(d.g_k, 8 * G, g, nt);
        }
    }
    prefetch_range(d.row_ptr, 4 * (N + 1), g, nt);
    prefetch_range(d.grain, 4 * N, g, nt);
    prefetch_range(d.bits, 4 * N * (size_t)k.wpn, g, nt);
    prefetch_range(d.nbr_cnt, 4 * N, g, nt);
    prefetch_range(d.nbr, 4 * N * (size_t)kPrefetchListRows, g, nt);
    if (d.pq) {
        prefetch_range(d.colx, 4 * nb, g, nt);
    } else {
        prefetch_range(d.col, 4 * nb, g, nt);
        prefetch_range(d.xi, 8 * nb, g, nt);
    }
}

// Hash-grid cells of the four walls of every aggregate at time t (written once
// per force evaluation by the threads of one block, one aggregate each): a node
// two or more cells away from all of them is farther than R_c from every wall
// and feels no wall force.
__device__ __forceinline__ void wall_cells(const DevPtrs &d, const KParams &k, double t) {
    for (int a = threadIdx.x; a < k.n_agg; a += blockDim.x) {
        const AggParams &A = d.agg[a];
        d.wall_cell[a] = make_int4(cell_coord(A.w0[0] + A.wv[0] * t, A.ox, A.inv_cell),
                                   cell_coord(A.w0[1] + A.wv[1] * t, A.ox, A.inv_cell),
                                   cell_coord(A.w0[2] + A.wv[2] * t, A.oy, A.inv_cell),
                                   cell_coord(A.w0[3] + A.wv[3] * t, A.oy, A.inv_cell));
    }
}

// The node cell is the one of the last rebuild: the node has moved less than
// kSkinTrigger * skin since, and cells are wider than R_c + skin, so two cells
// from a wall's cell still means farther than R_c from the wall.
template <bool PERSIST>
__device__ __forceinline__ bool far_from_walls(const DevPtrs &d, int i, int ag) {
    const int2 c = ldm<PERSIST>(&d.cell[i]);
    const int4 w = ldm<PERSIST>(&d.wall_cell[ag]);
    return c.x - w.x >= 2 && w.y - c.x >= 2 && c.y - w.z >= 2 && w.w - c.y >= 2;
}

// The same test on a cell and wall-cell record already loaded.
__device__ __forceinline__ bool cells_far_from_walls(int2 c, int4 w) {
    return c.x - w.x >= 2 && w.y - c.x >= 2 && c.y - w.z >= 2 && w.w - c.y >= 2;
}

// Counting-sort scatter of node i into its bucket, with its position record.
template <bool PERSIST>
__device__ __forceinline__ void scatter_node(const DevPtrs &d, const KParams &k, int i) {
    const int pos = atomicAdd(&d.cursor[ldm<PERSIST>(&d.key[i])], 1);
    d.sorted[pos] = i;
    uint4 rec;
    if (k.fp32) {
        const float4 q = ldm<PERSIST>(&cur_pq<PERSIST>(d)[i]);
        rec = make_uint4(__float_as_uint(q.x), __float_as_uint(q.y), __float_as_uint(q.z), __float_as_uint(q.w));
    } else {
        const double2 p = ldm<PERSIST>(&d.p[i]);
        rec = make_uint4((unsigned)__double2loint(p.x), (unsigned)__double2hiint(p.x), (unsigned)__double2loint(p.y),
                         (unsigned)__double2hiint(p.y));
    }
    d.srec[pos] = rec;
}

// Rebuild, last step: the candidate list of node i -- every node y != i of
// its aggregate with |p(y) - p(i)| < R_c + skin, gathered from the 3x3 block
// of hash-grid cells around its cell (cells are wider than R_c + skin) and
// kept in ascending node index -- and the position it was built at.  The
// bucket records hold the positions in bucket order, so only nodes inside
// the radius are looked up.  The three buckets of a row of the block are
// walked as one range of records, so that the threads of a warp step through
// rows rather than through nine buckets of different lengths.
template <bool PERSIST>
__device__ __forceinline__ void build_list_node(const DevPtrs &d, const KParams &k, int i) {
    const int ag = __ldg(&d.g_agg[__ldg(&d.grain[i])]);
    const AggParams &A = d.agg[ag];
    const int2 cc = ldm<PERSIST>(&d.cell[i]);
    const unsigned ha = (unsigned)ag * kHashA, mask = k.T - 1u;
    unsigned hx[3], bk[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) hx[c] = (unsigned)(cc.x + c - 1) * kHashX;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const unsigned hy = (unsigned)(cc.y + r - 1) * kHashY ^ ha;
#pragma unroll
        for (int c = 0; c < 3; ++c) bk[3 * r + c] = (hx[c] ^ hy) & mask;
    }
    float4 qi = make_float4(0.f, 0.f, 0.f, 0.f);
    double2 pi = make_double2(0.0, 0.0);
    if (d.pq) qi = ldm<PERSIST>(&cur_pq<PERSIST>(d)[i]);
    else pi = ldm<PERSIST>(&d.p[i]);
    int lst[kMaxList];
    int n = 0, over = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int t0[3], m[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int cell = 3 * r + c;
            bool dup = false;      // two cells of the block hashed to one bucket: visit it once
#pragma unroll
            for (int q = 0; q < cell; ++q) dup |= bk[q] == bk[cell];
            t0[c] = dup ? 0 : ldm<PERSIST>(&d.start[bk[cell]]);
            m[c] = dup ? 0 : ldm<PERSIST>(&d.start[bk[cell] + 1]) - t0[c];
        }
        const int tot = m[0] + m[1] + m[2];
        for (int e = 0; e < tot; ++e) {
            const int t = e < m[0] ? t0[0] + e : (e < m[0] + m[1] ? t0[1] + (e - m[0]) : t0[2] + (e - m[0] - m[1]));
            const uint4 rec = ldm<PERSIST>(&d.srec[t]);
            float dx, dy;
            if (d.pq) {
                dx = (__uint_as_float(rec.x) - qi.x) + (__uint_as_float(rec.z) - qi.z);
                dy = (__uint_as_float(rec.y) - qi.y) + (__uint_as_float(rec.w) - qi.w);
            } else {
                dx = (float)(__hiloint2double((int)rec.y, (int)rec.x) - pi.x);
                dy = (float)(__hiloint2double((int)rec.w, (int)rec.z) - pi.y);
            }
            if (!(dx * dx + dy * dy < A.rs2)) continue;
            const int j = ldm<PERSIST>(&d.sorted[t]);
            // hash aliasing can bring nodes of another aggregate: never in contact
            if (j == i || __ldg(&d.g_agg[__ldg(&d.grain[j])]) != ag) continue;
            if (n < kMaxList) {
                int w = n++;
                while (w > 0 && lst[w - 1] > j) {
                    lst[w] = lst[w - 1];
                    --w;
                }
                lst[w] = j;
            } else {
                over = 1;
            }
        }
    }
    const size_t N = (size_t)k.N;
    for (int q = 0; q < n; ++q) d.nbr[q * N + i] = lst[q];
    d.nbr_cnt[i] = n;
    if (d.pq) {
        d.sref[i] = qi;
    } else {
        const double2 u = ldm<PERSIST>(&cur_u<PERSIST>(d)[i]);
        d.sref[i] = make_float4((float)u.x, (float)u.y, 0.f, 0.f);
    }
    if (over) atomicAdd(&d.status[PD_STATUS_OVERFLOW], 1);
}

// Is the bond x -> j intact?  (row columns ascending: binary search; broken
// flags read past L1, since other lanes may have just set them.)
__device__ __forceinline__ bool bonded_intact(const DevPtrs &d, const KParams &k, int i, int r0, int r1, int j) {
    int lo = r0, hi = r1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(&d.col[mid]) < j) lo = mid + 1; else hi = mid;
    }
    if (lo < r1 && __ldg(&d.col[lo]) == j) {
        const int kk = lo - r0;
        return !((__ldcg(&d.bits[(size_t)i * k.wpn + (kk >> 5)]) >> (kk & 31)) & 1u);
    }
    return false;
}

// Acceleration and velocity update of node i (Algorithm 1) plus the optional
// per-part force output; run by one lane per node.  m = rho V, or with RECIP
// inv_m = 1 / (rho V): a = F (1 / m) + g and the velocity update fused, about
// one ulp of a from the quotient (the forces themselves are unchanged), for
// the two FP64 divisions per node that GB300's FP64 pipe makes costly.
template <bool PERSIST, bool RECIP = false>
__device__ __forceinline__ void finish_node(const DevPtrs &d, const KParams &k, int i, int vin, int update_v,
                                            double2 vi, double m, double Fbx, double Fby, double Fsx, double Fsy,
                                            double Fnx, double Fny, double Fwx, double Fwy, double inv_m = 0.0) {
    const double Fx = __dadd_rn(__dadd_rn(__dadd_rn(Fbx, Fsx), Fnx), Fwx);
    const double Fy = __dadd_rn(__dadd_rn(__dadd_rn(Fby, Fsy), Fny), Fwy);
    double ax, ay;
    if constexpr (RECIP) {
        ax = fma(Fx, inv_m, k.gx);
        ay = fma(Fy, inv_m, k.gy);
    } else {
        ax = __dadd_rn(__ddiv_rn(Fx, m), k.gx);
        ay = __dadd_rn(__ddiv_rn(Fy, m), k.gy);
    }
    if (update_v) {
        const double2 ao = ldm<PERSIST>(&d.a[i]);
        double2 vn;
        if constexpr (RECIP) {
            vn.x = fma(k.half_dt, ao.x + ax, vi.x);
            vn.y = fma(k.half_dt, ao.y + ay, vi.y);
        } else {
            vn.x = __dadd_rn(vi.x, __dmul_rn(k.half_dt, __dadd_rn(ao.x, ax)));
            vn.y = __dadd_rn(vi.y, __dmul_rn(k.half_dt, __dadd_rn(ao.y, ay)));
        }
        d.v[vin ^ 1][i] = vn;
    }
    d.a[i] = make_double2(ax, ay);
    if ((((unsigned)__double2hiint(ax) | 0x800FFFFFu) == 0xFFFFFFFFu) || (((unsigned)__double2hiint(ay) | 0x800FFFFFu) == 0xFFFFFFFFu))   // inf or NaN
        atomicAdd(&d.status[PD_STATUS_NONFINITE], 1);
    if (k.store) {
        d.F[i] = make_double2(Fx, Fy);
        d.parts[i] = make_double2(Fbx, Fby);
        d.parts[k.N + i] = make_double2(Fsx, Fsy);
        d.parts[2 * (size_t)k.N + i] = make_double2(Fnx, Fny);
        d.parts[3 * (size_t)k.N + i] = make_double2(Fwx, Fwy);
    }
}

// FP32-split update: the lane-summed parts are added in FP32 (their rounding is
// far below the path's force error), the wall force in FP64 where there is one;
// a = F (1 / m) + g is formed and stored in FP32 (the force carries FP32
// precision already), the velocity-Verlet increment dt/2 (a_old + a) is
// formed in FP32 and added to the FP64 velocity: two FP64 additions per node
// on GB300's narrow FP64 pipe.  (ao: the previous acceleration, loaded by the
// caller with the node's other independent loads.)
//
// The persistent kernel (PERSIST) also takes the next step's displacement
// update here, from the velocity and acceleration just formed and the node's
// current displacement ui: u and pq of the next step go to ub[vin] / pqb[vin]
// (free: this step reads ub[vin ^ 1] / pqb[vin ^ 1]), and a node past the
// rebuild trigger raises the next step's flag.  The next step then skips its
// update phase, which would have read u, v and a back from memory.
template <bool PERSIST>
__device__ __forceinline__ void finish_node32_total(const DevPtrs &d, const KParams &k, int i, int vin, int update_v,
                                                    double2 vi, float2 ao, float fx, float fy, bool walls,
                                                    double Fwx, double Fwy, float inv_m, double2 ui = {}) {
    float ax, ay;
    if (walls) {
        ax = fmaf(__double2float_rn(f2d_bits(fx) + Fwx), inv_m, k.gxf);
        ay = fmaf(__double2float_rn(f2d_bits(fy) + Fwy), inv_m, k.gyf);
    } else {
        ax = fmaf(fx, inv_m, k.gxf);
        ay = fmaf(fy, inv_m, k.gyf);
    }
    if (update_v) {
        const float hdt = 0.5f * k.dtf;
        const double2 vn = make_double2(vi.x + f2d_bits(hdt * (ao.x + ax)), vi.y + f2d_bits(hdt * (ao.y + ay)));
        d.v[vin ^ 1][i] = vn;
        if constexpr (PERSIST) {
            if (advance_node32<PERSIST>(d, k, i, ui, vn, ax, ay, d.ub[vin], d.pqb[vin]))
                *(volatile int *)d.rebuild_next = 1;
        }
    }
    d.af[i] = make_float2(ax, ay);
    // finiteness from the exponent bits (no FP64 compare)
    if (((__float_as_uint(ax) | 0x807FFFFFu) == 0xFFFFFFFFu) || ((__float_as_uint(ay) | 0x807FFFFFu) == 0xFFFFFFFFu))
        atomicAdd(&d.status[PD_STATUS_NONFINITE], 1);
}

// FP64 update from the total of the lane-summed parts, T = (F_b + F_s) + F_n
// (as finish_node forms it), and the wall force: the same roundings as
// finish_node with the reciprocal mass, without the per-part output.
template <bool PERSIST>
__device__ __forceinline__ void finish_node64_total(const DevPtrs &d, const KParams &k, int i, int vin, int update_v,
                                                    double2 vi, double2 ao, double Tx, double Ty, bool walls,
                                                    double Fwx, double Fwy, double inv_m) {
    const double Fx = walls ? __dadd_rn(Tx, Fwx) : Tx, Fy = walls ? __dadd_rn(Ty, Fwy) : Ty;
    const double ax = fma(Fx, inv_m, k.gx), ay = fma(Fy, inv_m, k.gy);
    if (update_v)
        d.v[vin ^ 1][i] = make_double2(fma(k.half_dt, ao.x + ax, vi.x), fma(k.half_dt, ao.y + ay, vi.y));
    d.a[i] = make_double2(ax, ay);
    if ((((unsigned)__double2hiint(ax) | 0x800FFFFFu) == 0xFFFFFFFFu) || (((unsigned)__double2hiint(ay) | 0x800FFFFFu) == 0xFFFFFFFFu))   // inf or NaN
        atomicAdd(&d.status[PD_STATUS_NONFINITE], 1);
}

template <int LANES, class T>
__device__ __forceinline__ T lane_sum(T v) {
#pragma unroll
    for (int off = 1; off < LANES; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// FP64 forces of node i (eq:full, Algorithm 1), LANES threads per node: lane l
// takes bonds l, l + LANES, ... and grid cells l, l + LANES, ...; partial sums
// meet in a fixed xor-butterfly (deterministic).  With LANES = 1 every sum is
// in the textbook order (bonds in CSR order, contacts in ascending index).
// Every thread of the warp must call this (shuffles); inactive lanes pass
// active = false.
// Lane-summed per-node force parts (bond, self-contact, contact), handed from
// the lanes of a node to the node's epilogue thread.
struct Sums64 {
    double bx, by, sx, sy, nx, ny;
};
struct Sums32 {
    float bx, by, sx, sy, nx, ny;
};

template <bool PERSIST, int LANES>
__device__ __forceinline__ void force_node64(const DevPtrs &d, const KParams &k, int i, int lane, bool active,
                                             int vin, Sums64 &out) {
    const int ii = active ? i : 0;
    const double2 pi = ldm<PERSIST>(&d.p[ii]);
    const double2 Xi = __ldg(&d.X[ii]);
    const double Vi = __ldg(&d.V[ii]);
    const int gi = __ldg(&d.grain[ii]);
    const int ag = __ldg(&d.g_agg[gi]);
    const AggParams &A = d.agg[ag];
    const double cw = __ldg(&d.g_cw[gi]), s0 = __ldg(&d.g_s0[gi]), eps = __ldg(&d.g_eps[gi]);
    const int r0 = active ? __ldg(&d.row_ptr[ii]) : 0, r1 = active ? __ldg(&d.row_ptr[ii + 1]) : 0;
    uint32_t *bw = d.bits + (size_t)ii * k.wpn;

    // peridynamic bonds with breaking (eq:peri, eq:pmb, Sec. 3.1).  The
    // stretch's cancelling difference L - |xi| is formed exactly as the FP64
    // definition rounds it: dx, dy and |d|^2 in FP64, L = sqrt(|d|^2) correctly
    // rounded (integer square root), L - |xi| in FP64.  The quotient by |xi|,
    // the break decision away from the threshold and the bond force
    // c_w w s V_x V_y (d / L) are float-float (relative error ~1e-14; a bond
    // whose stretch lies within 1e-6 of s0 is decided by the FP64 quotient).
    ff Fbx = {0.f, 0.f}, Fby = {0.f, 0.f};
    const uint32_t w0 = active ? __ldcg(bw) : 0u;      // the row's first 32 broken bits (own bonds only)
    const float s0f = (float)s0;
    const ff cwVV = to_ff(cw * Vi * Vi);                // one grain: V_y = V_x
    const ff inv_eps = ff_rcp(to_ff(eps));
    constexpr int kBondBatch64 = 4;
    for (int b0 = r0 + lane; b0 < r1; b0 += kBondBatch64 * LANES) {
        int jb[kBondBatch64];
        uint32_t wb[kBondBatch64];
        double xb[kBondBatch64];
        double2 pb[kBondBatch64];
#pragma unroll
        for (int m = 0; m < kBondBatch64; ++m) {
            const int b = b0 + m * LANES;
            jb[m] = b < r1 ? __ldg(&d.col[b]) : -1;
            xb[m] = b < r1 ? __ldg(&d.xi[b]) : 1.0;
            wb[m] = b - r0 < 32 ? w0 : (b < r1 ? __ldcg(&bw[(b - r0) >> 5]) : 0u);
        }
#pragma unroll
        for (int m = 0; m < kBondBatch64; ++m) pb[m] = ldm<PERSIST>(&d.p[jb[m] < 0 ? ii : jb[m]]);
#pragma unroll
        for (int m = 0; m < kBondBatch64; ++m) {
            const int kk = b0 + m * LANES - r0;
            if (jb[m] < 0 || ((wb[m] >> (kk & 31)) & 1u)) continue;
            const double xi = xb[m];
            const double dx = __dsub_rn(pb[m].x, pi.x), dy = __dsub_rn(pb[m].y, pi.y);
            const double L = sqrt_rn_int(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            const double diff = __dsub_rn(L, xi);                       // |xi| s, exact as in FP64
            const ff dff = to_ff(diff), xff = to_ff(xi);
            // break test |diff| > s0 |xi| in float, the FP64 quotient near the threshold
            const float lhs = fabsf(dff.hi), rhs = s0f * xff.hi;
            bool brk = lhs > rhs;
            if (fabsf(lhs - rhs) <= 1e-6f * rhs) brk = fabs(__ddiv_rn(diff, xi)) > s0;
            if (brk) {
                atomicOr(&bw[kk >> 5], 1u << (kk & 31));
                continue;
            }
            // c_w w V_x V_y (diff / |xi|) / L  (w = 1 - |xi| / eps for the conic micromodulus)
            ff c = cwVV;
            if (k.micro) c = ff_mul(c, ff_add({1.0f, 0.f}, ff_mul({-xff.hi, -xff.lo}, inv_eps)));
            const ff t = ff_mul(ff_mul(c, dff), ff_rcp(ff_mul(xff, to_ff(L))));
            Fbx = ff_add(Fbx, ff_mul(t, to_ff(dx)));
            Fby = ff_add(Fby, ff_mul(t, to_ff(dy)));
        }
    }
    __syncwarp();

    // contact candidates (the node's list: every pair closer than R_c is in it,
    // ascending node index), self-contact (Sec. 4.4), inter-grain contact
    // (Secs. 4.1-4.3)
    const double Rc = A.Rc;
    // |d|^2 above R_c^2 (1 + 1e-12) means sqrt(|d|^2) rounds to R_c or more:
    // candidates that far are dropped before the square root
    const double rc2_out = Rc * Rc * (1.0 + 1e-12);
    const double rho_i = k.mat ? __ldg(&d.g_rho[gi]) : k.rho;
    const int nc = active ? ldm<PERSIST>(&d.nbr_cnt[ii]) : 0;
    const double2 vi = ldm<PERSIST>(&d.v[vin][ii]);
    double Fsx = 0.0, Fsy = 0.0, Fnx = 0.0, Fny = 0.0;
    for (int q = lane; q < nc; q += LANES) {
        const int j = ldm<PERSIST>(&d.nbr[(size_t)q * k.N + ii]);
        const double2 pj = ldm<PERSIST>(&d.p[j]);
        double dx = pj.x - pi.x, dy = pj.y - pi.y;
        const double dd2 = dx * dx + dy * dy;
        if (!(dd2 <= rc2_out)) continue;
        double dd = dd2 > 0.0 ? sqrt_rn_int(dd2) : 0.0;
        if (!(dd < Rc)) continue;
        if (dd == 0.0) {
            atomicAdd(&d.status[PD_STATUS_COINCIDENT], 1);
            continue;
        }
        double ex = dx / dd, ey = dy / dd;
        const double Vj = __ldg(&d.V[j]);
        const double2 vj = ldm<PERSIST>(&d.v[vin][j]);
        double vrx = vi.x - vj.x, vry = vi.y - vj.y;
        const int gj = __ldg(&d.grain[j]);
        if (gj == gi) {
            if (bonded_intact(d, k, ii, r0, r1, j)) continue;
            const double2 Xj = __ldg(&d.X[j]);
            double xix = Xj.x - Xi.x, xiy = Xj.y - Xi.y;
            double xi = sqrt(xix * xix + xiy * xiy);
            double m;
            if (xi < Rc)
                m = (dd < xi) ? cw * (dd - xi) / xi : 0.0;
            else
                m = cw * (dd - Rc) / Rc;
            if (m == 0.0) continue;
            double f = m * Vi * Vj;
            double gx = f * ex, gy = f * ey;
            const double Kn = k.mat ? 18.0 * __ldg(&d.g_k[gi]) / A.pe5 : A.Kn;
            damping_friction64(k, Kn, rho_i, rho_i, ex, ey, vrx, vry, -f, Vi, Vj, gx, gy);
            Fsx += gx;
            Fsy += gy;
        } else {
            double Kn = A.Kn, rho_d = rho_i;
            if (k.mat) {
                Kn = 18.0 * harmonic64(__ldg(&d.g_k[gi]), __ldg(&d.g_k[gj])) / A.pe5;
                rho_d = harmonic64(rho_i, __ldg(&d.g_rho[gj]));
            }
            double Fr = Kn * (Rc - dd) * Vi * Vj;
            double gx = -Fr * ex, gy = -Fr * ey;
            damping_friction64(k, Kn, rho_d, rho_i, ex, ey, vrx, vry, Fr, Vi, Vj, gx, gy);
            Fnx += gx;
            Fny += gy;
        }
    }
    out.bx = lane_sum<LANES>(f2d_bits(Fbx.hi) + f2d_bits(Fbx.lo));
    out.by = lane_sum<LANES>(f2d_bits(Fby.hi) + f2d_bits(Fby.lo));
    out.sx = lane_sum<LANES>(Fsx);
    out.sy = lane_sum<LANES>(Fsy);
    out.nx = lane_sum<LANES>(Fnx);
    out.ny = lane_sum<LANES>(Fny);
}

// Wall forces and the update of node i from its lane sums, one thread per node
// (the FP64 work runs with converged warps).
template <bool PERSIST>
__device__ __forceinline__ void node_epilogue64(const DevPtrs &d, const KParams &k, int i, int vin, int update_v,
                                                const Sums64 &f, bool total = false) {
    // the node's independent loads first, all in flight together (the pass is
    // bound by memory latency): velocity, previous acceleration, grain, cell
    const double2 vi = ldm<PERSIST>(&d.v[vin][i]);
    const double2 ao = update_v ? ldm<PERSIST>(&d.a[i]) : make_double2(0.0, 0.0);
    const int gi = __ldg(&d.grain[i]);
    const int2 cell = ldm<PERSIST>(&d.cell[i]);
    const int ag = __ldg(&d.g_agg[gi]);
    const double inv_m = __ldg(&d.g_invm[gi]);
    const int4 wc = ldm<PERSIST>(&d.wall_cell[ag]);
    double Fwx = 0.0, Fwy = 0.0;
    const bool walls = !cells_far_from_walls(cell, wc);
    if (walls) {
        const double2 pi = ldm<PERSIST>(&d.p[i]);
        const AggParams &A = d.agg[ag];
        const double rho = k.mat ? __ldg(&d.g_rho[gi]) : k.rho;
        const double Kn = k.mat ? 18.0 * __ldg(&d.g_k[gi]) / A.pe5 : A.Kn;
        wall_force64(k, A, Kn, rho, ldm<PERSIST>(d.t_now), pi.x, pi.y, vi.x, vi.y, __ldg(&d.V[i]), Fwx, Fwy,
                     d.status);
    }
    if (k.store) {
        finish_node<PERSIST, true>(d, k, i, vin, update_v, vi, 0.0, f.bx, f.by, f.sx, f.sy, f.nx, f.ny, Fwx, Fwy,
                                   inv_m);
    } else {
        // total: the parts were summed by the lane-sum pass, f.bx / f.by hold T
        const double Tx = total ? f.bx : __dadd_rn(__dadd_rn(f.bx, f.sx), f.nx);
        const double Ty = total ? f.by : __dadd_rn(__dadd_rn(f.by, f.sy), f.ny);
        finish_node64_total<PERSIST>(d, k, i, vin, update_v, vi, ao, Tx, Ty, walls, Fwx, Fwy, inv_m);
    }
}

// FP32-split geometry of one bond to a neighbour at qj (float-float shifted
// position), lattice offset code nn = di^2 + dj^2 and sqn = sqrt(nn):
// num = |d|^2 - |xi|^2 (float-float difference, |xi|^2 = n h^2 exact to
// float-float), den = |xi| (L + |xi|), so that s = num / den.  Returns 0 =
// intact, 1 = broken at this evaluation (|s| > s0), 2 = |s| in the guard band
// around s0 (decided in FP64 after the loop).  The tests compare |num| with
// s0 den: no division.
struct BondGeom32 {
    float dx, dy, L, num, den, xi;
};
// (pow2: n is a power of two, so n h^2 is exact in float-float without a
// product residual; callers that know n at compile time pass it as a constant)
__device__ __forceinline__ int bond_classify32(float4 qj, float2 phi, float2 pli, float nn, float sqn, float4 gq,
                                               float s0_lo, float s0_hi, BondGeom32 &g, bool pow2 = false) {
    const float dxh = __fsub_rn(qj.x, phi.x), dxl = qj.z - pli.x;
    const float dyh = __fsub_rn(qj.y, phi.y), dyl = qj.w - pli.y;
    float L2h, L2l;
    len2_ff(dxh, dxl, dyh, dyl, L2h, L2l);
    float q, eq;                                         // |xi|^2 = n h^2 as a float-float pair
    if (pow2) {
        q = nn * gq.y;
        eq = nn * gq.z;
    } else {
        two_prod(nn, gq.y, q, eq);
        eq = fmaf(nn, gq.z, eq);
    }
    g.num = ff_diff(L2h, L2l, q, eq);
    g.xi = gq.x * sqn;
    g.L = sqrt_approx(L2h);
    g.den = g.xi * (g.L + g.xi);
    g.dx = dxh + dxl;
    g.dy = dyh + dyl;
    // intact and clear of the guard band (the common case): one comparison; a
    // NaN stretch counts as intact, as in the band tests
    const float an = fabsf(g.num);
    if (!(an > s0_lo * g.den)) return 0;
    return an < s0_hi * g.den ? 2 : 1;
}

// Adds the bond force c_w w V^2 s (d / L) of an intact bond (w = 1 - |xi| / eps
// for the conic micromodulus).
__device__ __forceinline__ void bond_add32(const BondGeom32 &g, float cw, float eps, float VV, int micro, float &Fbx,
                                           float &Fby) {
    const float c = micro ? cw * (1.0f - __fdividef(g.xi, eps)) : cw;
    const float qf = __fdividef(c * VV * g.num, g.den * g.L);
    Fbx += qf * g.dx;
    Fby += qf * g.dy;
}

// sqrt(di^2 + dj^2) of the stencil offsets (compile-time for a fixed offset)
__host__ __device__ constexpr float stn_sqrt_n(int n) {
    return n == 1 ? 1.0f : (n == 2 ? 1.41421356f : (n == 4 ? 2.0f : (n == 5 ? 2.23606798f : 2.82842712f)));
}

// Offset o (0..23) of the bond stencil: the 5 x 5 lattice block without its
// centre, in (dj, di) order.
__host__ __device__ constexpr int stn_di(int o) { return (o + (o >= 12 ? 1 : 0)) % 5 - 2; }
__host__ __device__ constexpr int stn_dj(int o) { return (o + (o >= 12 ? 1 : 0)) / 5 - 2; }

// FP32-split forces of node i: the same laws and lane layout, with the bond,
// self-contact and contact arithmetic on the FP32 pipe.  Positions are
// float-float pairs of the shifted position (every coordinate of a box lies in
// [L, 2L), so high-part differences of nearby nodes are exact), |d|^2 is a
// float-float pair built with exact FMA products, and the reference
// |xi|^2 = h^2 (di^2 + dj^2) comes from the integer lattice offset: the stretch
// s = (|d|^2 - |xi|^2) / (|xi| (|d| + |xi|)) (eq:pmb, rearranged) and the
// contact overlap R_c - |d| = (R_c^2 - |d|^2) / (R_c + |d|) keep ~1e-7 relative
// accuracy.  Bonds whose FP32 stretch lies within guard * s0 of s0 are
// re-decided with the FP64 stretch, so break decisions are the FP64 ones.
// The learned surrogate is used only while none of its bounded tensor-core
// waits has given up (status[PD_STATUS_TIMEOUT], the networks' error word): a
// step in which one gives up still runs on the surrogate in the kernels that
// started before it, every later step uses the full bond kernel.
__device__ __forceinline__ bool sur_healthy(const DevPtrs &d) {
    return __ldcg(&d.status[PD_STATUS_TIMEOUT]) == 0 && (d.mlp_err == nullptr || __ldcg(d.mlp_err) == 0);
}

template <bool PERSIST, int LANES>
__device__ __forceinline__ void force_node32(const DevPtrs &d, const KParams &k, int i, int lane, bool active,
                                             int vin, Sums32 &out) {
    const int ii = active ? i : 0;
    const float4 qi = ldm<PERSIST>(&cur_pq<PERSIST>(d)[ii]);
    const float2 phi = make_float2(qi.x, qi.y), pli = make_float2(qi.z, qi.w);
    const int gi = __ldg(&d.grain[ii]);
    const int ag = __ldg(&d.g_agg[gi]);
    const AggParams &A = d.agg[ag];
    const float4 gq = __ldg(&d.gq[gi]);                   // (h, h^2 hi, h^2 lo, V)
    const float Vi = gq.w;
    const float4 gc = __ldg(&d.gc[gi]);                   // (c_w, s0, eps) as floats
    const float cw = gc.x, s0 = gc.y, eps = gc.z;
    const float s0_lo = s0 * (1.0f - k.guard), s0_hi = s0 * (1.0f + k.guard);
    // lattice stencil of the node's bonds (regular nodes: the neighbour at
    // offset o is node ii + di + D[dj], no column load), else the CSR columns
    const uint4 st = (k.stencil && active) ? __ldg(&d.stn[ii]) : make_uint4(kStnIrregular, 0u, 0u, 0u);
    const bool stencil = !(st.x & kStnIrregular);
    int r0 = 0, r1 = 0;
    if (stencil) {
        r0 = (int)st.w;
        r1 = r0 + __popc(st.x);
    } else if (active) {
        r0 = __ldg(&d.row_ptr[ii]);
        r1 = __ldg(&d.row_ptr[ii + 1]);
    }
    uint32_t *bw = d.bits + (size_t)ii * k.wpn;
    const float Rc = A.rcf, Kn = A.knf;

    float Fbx = 0.f, Fby = 0.f;
    const float VV = Vi * Vi;
    // learned modal surrogate: between judge steps an active grain skips the
    // bond loop; the epilogue adds its surrogate bond force instead
    bool sur = false, judge = false;
    if constexpr (!PERSIST) {
        if (k.sur && active) {
            sur = d.sur_active[gi] != 0 && sur_healthy(d);
            judge = (*d.step) % k.judge_every == 0;
        }
    }
    // broken-bond bits of the node's first 32 bonds: only the node's own threads
    // set them, each for its own bonds, so one load at the start serves the loop
    const uint32_t w0 = active ? __ldcg(bw) : 0u;
    bool pending = false;      // a bond of this lane lies in the guard band
    // bonds in batches of kBondBatch per lane: the column indices, broken words and
    // neighbour positions of a batch are all in flight before any is used (the
    // per-lane summation order is unchanged: bonds lane, lane + LANES, ...)
    constexpr int kBondBatch = 4;
    if (stencil && !(sur && !judge)) {
        const uint32_t mask = st.x;
        // the intact bonds by stencil offset: the broken-bond bits follow the
        // order of the node's bonds (the rank of the offset among the stencil
        // bits), so each set bit clears the stencil bit of that rank (a node
        // seldom has a broken bond: the loop is skipped)
        uint32_t alive = mask;
        for (uint32_t wb = w0; wb; wb &= wb - 1u) {
            uint32_t m = mask;
            for (int t = __ffs(wb) - 1; t > 0; --t) m &= m - 1u;
            alive &= ~(m & (0u - m));
        }
        const int Dm2 = (int)(short)(st.y & 0xFFFFu), Dm1 = (int)(short)(st.y >> 16);
        const int Dp1 = (int)(short)(st.z & 0xFFFFu), Dp2 = (int)(short)(st.z >> 16);
        constexpr int kPerLane = (24 + LANES - 1) / LANES;
        // fully unrolled: offsets, lattice codes and sqrt(n) are constants for one
        // lane per node (a loop over the batches was 30 % slower on the compaction)
#pragma unroll
        for (int m0 = 0; m0 < kPerLane; m0 += kBondBatch) {
            float4 qb[kBondBatch];
            bool live[kBondBatch];
#pragma unroll
            for (int m = 0; m < kBondBatch; ++m) {
                const int o = (m0 + m) * LANES + lane;
                const int dj = stn_dj(o), di = stn_di(o);
                const int D = dj == -2 ? Dm2 : (dj == -1 ? Dm1 : (dj == 0 ? 0 : (dj == 1 ? Dp1 : Dp2)));
                live[m] = (m0 + m) < kPerLane && o < 24 && ((alive >> o) & 1u);
                qb[m] = ldm<PERSIST>(&cur_pq<PERSIST>(d)[live[m] ? ii + di + D : ii]);
            }
#pragma unroll
            for (int m = 0; m < kBondBatch; ++m) {
                if (!live[m]) continue;
                const int o = (m0 + m) * LANES + lane;
                const int dj = stn_dj(o), di = stn_di(o);
                const int n = di * di + dj * dj;
                BondGeom32 bg;
                const int r = bond_classify32(qb[m], phi, pli, (float)n, stn_sqrt_n(n), gq, s0_lo, s0_hi, bg,
                                              (n & (n - 1)) == 0);
                if (r == 0) bond_add32(bg, cw, eps, VV, k.micro, Fbx, Fby);
                else if (r == 2) pending = true;
                else atomicOr(bw, 1u << __popc(mask & ((1u << o) - 1u)));
            }
        }
    }
    for (int b0 = r0 + lane; b0 < r1 && !stencil && !(sur && !judge); b0 += kBondBatch * LANES) {
        uint32_t cb[kBondBatch], wb[kBondBatch];
#pragma unroll
        for (int m = 0; m < kBondBatch; ++m) {
            const int b = b0 + m * LANES;
            cb[m] = b < r1 ? __ldg(&d.colx[b]) : 0xFFFFFFFFu;
            // the node's first broken-bond word is loaded once (rows of up to 32 bonds)
            wb[m] = b - r0 < 32 ? w0 : (b < r1 ? __ldcg(&bw[(b - r0) >> 5]) : 0u);
        }
        float4 qb[kBondBatch];
#pragma unroll
        for (int m = 0; m < kBondBatch; ++m) {
            const int j = cb[m] == 0xFFFFFFFFu ? ii : (int)(cb[m] & kColMask);
            qb[m] = ldm<PERSIST>(&cur_pq<PERSIST>(d)[j]);
        }
#pragma unroll
        for (int m = 0; m < kBondBatch; ++m) {
            const int b = b0 + m * LANES;
            const int kk = b - r0;
            if (cb[m] == 0xFFFFFFFFu || ((wb[m] >> (kk & 31)) & 1u)) continue;
            const float nn = (float)(cb[m] >> kColBits);         // lattice offset di^2 + dj^2
            BondGeom32 bg;
            const int r = bond_classify32(qb[m], phi, pli, nn, sqrt_approx(nn), gq, s0_lo, s0_hi, bg);
            if (r == 0) bond_add32(bg, cw, eps, VV, k.micro, Fbx, Fby);
            else if (r == 2) pending = true;
            else atomicOr(&bw[kk >> 5], 1u << (kk & 31));
        }
    }
    if (pending) {
        // the lane's bonds in the guard band, in its order: FP64 break decision,
        // else the FP32 force
        for (int b = r0 + lane; b < r1; b += LANES) {
            const int kk = b - r0;
            if ((__ldcg(&bw[kk >> 5]) >> (kk & 31)) & 1u) continue;
            const uint32_t c = __ldg(&d.colx[b]);
            const int j = (int)(c & kColMask);
            const float4 qj = ldm<PERSIST>(&cur_pq<PERSIST>(d)[j]);
            const float nn = (float)(c >> kColBits);
            // the same classification as the loop (stencil: sqrt(n) from the table)
            const float sqn = stencil ? stn_sqrt_n((int)nn) : sqrt_approx(nn);
            BondGeom32 bg;
            if (bond_classify32(qj, phi, pli, nn, sqn, gq, s0_lo, s0_hi, bg) != 2) continue;
            const double2 pi = position64<PERSIST>(d, ii), pj = position64<PERSIST>(d, j);
            const double ddx = __dsub_rn(pj.x, pi.x), ddy = __dsub_rn(pj.y, pi.y);
            const double L64 = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)));
            const double xi64 = __ldg(&d.xi[b]);
            if (fabs(__ddiv_rn(__dsub_rn(L64, xi64), xi64)) > __ldg(&d.g_s0[gi])) {
                atomicOr(&bw[kk >> 5], 1u << (kk & 31));
                continue;
            }
            bond_add32(bg, cw, eps, VV, k.micro, Fbx, Fby);
        }
    }
    __syncwarp();

    // contact candidates from the node's list (ascending node index); the
    // R_c test is exact in float-float
    const int nc = active ? ldm<PERSIST>(&d.nbr_cnt[ii]) : 0;
    // start-of-step velocity (FP64; read only by nodes with candidates)
    const double2 vi64 = nc > 0 ? ldm<PERSIST>(&d.v[vin][ii]) : make_double2(0.0, 0.0);
    const float rd = k.rdf, rho = gc.w, dt = k.dtf, mu = k.muf;     // rho: this grain's density
    float Fsx = 0.f, Fsy = 0.f, Fnx = 0.f, Fny = 0.f;
    for (int q = lane; q < nc; q += LANES) {
        const int j = ldm<PERSIST>(&d.nbr[(size_t)q * k.N + ii]);
        const float4 qj = ldm<PERSIST>(&cur_pq<PERSIST>(d)[j]);
        const float dxh = __fsub_rn(qj.x, phi.x), dxl = qj.z - pli.x;
        const float dyh = __fsub_rn(qj.y, phi.y), dyl = qj.w - pli.y;
        float L2h, L2l;
        len2_ff(dxh, dxl, dyh, dyl, L2h, L2l);
        if (!(ff_diff(A.rc2_hi, A.rc2_lo, L2h, L2l) > 0.f)) continue;
        const float dd = sqrtf(L2h);
        if (dd == 0.f) {
            atomicAdd(&d.status[PD_STATUS_COINCIDENT], 1);
            continue;
        }
        const float ex = (dxh + dxl) / dd, ey = (dyh + dyl) / dd;
        const float overlap = ff_diff(A.rc2_hi, A.rc2_lo, L2h, L2l) / (Rc + dd);   // R_c - |d|
        const int gj = __ldg(&d.grain[j]);
        const float Vj = __ldg(&d.gq[gj]).w;
        // v(x) - v(y) in FP64, rounded once to float (nearby nodes move alike:
        // a float difference of float velocities would cancel)
        const double2 vj64 = ldm<PERSIST>(&d.v[vin][j]);
        const float vrx = (float)__dsub_rn(vi64.x, vj64.x), vry = (float)__dsub_rn(vi64.y, vj64.y);
        if (gj == gi) {
            if (bonded_intact(d, k, ii, r0, r1, j)) continue;
            const int2 li = __ldg(&d.lat[ii]), lj = __ldg(&d.lat[j]);
            const int di = lj.x - li.x, dj = lj.y - li.y;
            const float nn = (float)(di * di + dj * dj);
            const float xi = gq.x * sqrtf(nn);
            float m;
            if (xi < Rc) {
                float q2, eq2;
                two_prod(nn, gq.y, q2, eq2);
                const float dl = ff_diff(L2h, L2l, q2, eq2 + nn * gq.z) / (dd + xi);   // |d| - |xi|
                m = (dl < 0.f) ? cw * dl / xi : 0.f;
            } else {
                m = -cw * overlap / Rc;
            }
            if (m == 0.f) continue;
            const float f = m * Vi * Vj;
            float gx = f * ex, gy = f * ey;
            const float Kns = k.mat ? __ldg(&d.g_kf[gi]) : Kn;
            damping_friction32(rd, Kns, rho, rho, dt, mu, ex, ey, vrx, vry, -f, Vi, Vj, gx, gy);
            Fsx += gx;
            Fsy += gy;
        } else {
            // the harmonic mean of the grains' own K_n is K_n of the harmonic-mean modulus
            const float Knp = k.mat ? harmonic32(__ldg(&d.g_kf[gi]), __ldg(&d.g_kf[gj])) : Kn;
            const float Fr = Knp * overlap * Vi * Vj;
            float gx = -Fr * ex, gy = -Fr * ey;
            damping_friction32(rd, Knp, harmonic32(rho, __ldg(&d.gc[gj]).w), rho, dt, mu, ex, ey, vrx, vry, Fr, Vi,
                               Vj, gx, gy);
            Fnx += gx;
            Fny += gy;
        }
    }
    out.bx = lane_sum<LANES>(Fbx);
    out.by = lane_sum<LANES>(Fby);
    out.sx = lane_sum<LANES>(Fsx);
    out.sy = lane_sum<LANES>(Fsy);
    out.nx = lane_sum<LANES>(Fnx);
    out.ny = lane_sum<LANES>(Fny);
    if (sur && judge && lane == 0) d.sur_fb[i] = make_float2(out.bx, out.by);   // full bond force for the judge
}

template <bool PERSIST>
__device__ __forceinline__ void node_epilogue32(const DevPtrs &d, const KParams &k, int i, int vin, int update_v,
                                                const Sums32 &fin, bool total = false) {
    // the node's independent loads first, all in flight together (the pass is
    // bound by memory latency): velocity, previous acceleration, grain, cell
    const double2 vi = ldm<PERSIST>(&d.v[vin][i]);
    const float2 ao = update_v ? ldm<PERSIST>(&d.af[i]) : make_float2(0.f, 0.f);
    const int gi = __ldg(&d.grain[i]);
    const int2 cell = ldm<PERSIST>(&d.cell[i]);
    const int ag = __ldg(&d.g_agg[gi]);
    const float inv_m = __ldg(&d.g_invmf[gi]);
    const int4 wc = ldm<PERSIST>(&d.wall_cell[ag]);
    // the displacement for the next step's update (persistent kernel)
    const double2 ui = PERSIST && update_v ? ldm<PERSIST>(&cur_u<PERSIST>(d)[i]) : double2{};
    Sums32 f = fin;
    if constexpr (!PERSIST) {
        // learned modal surrogate: between judge steps an active grain's bond force
        // is R(theta + phi) Phi f E h (expanded on the tensor cores), in place of
        // the bond loop the sums skipped
        if (k.sur && d.sur_active[gi] && (*d.step) % k.judge_every != 0 && sur_healthy(d)) {
            const float2 sf = d.sur_f[i];                     // Phi f, lattice frame, units of E h
            const float2 rot = d.sur_rot[gi];
            const float Eh = k.E * __ldg(&d.gq[gi]).x;
            f.bx += (rot.x * sf.x - rot.y * sf.y) * Eh;
            f.by += (rot.y * sf.x + rot.x * sf.y) * Eh;
        }
    }
    double Fwx = 0.0, Fwy = 0.0;
    const bool walls = !cells_far_from_walls(cell, wc);
    if (walls) {
        const double2 pi = position64<PERSIST>(d, i);
        const AggParams &A = d.agg[ag];
        const double Kn = k.mat ? 18.0 * __ldg(&d.g_k[gi]) / A.pe5 : A.Kn;
        const double rho = k.mat ? __ldg(&d.g_rho[gi]) : k.rho;
        const float Knf = k.mat ? __ldg(&d.g_kf[gi]) : A.knf, rhof = __ldg(&d.gc[gi]).w;
        wall_force32(k, A, Knf, rhof, Kn, rho, ldm<PERSIST>(d.t_now), pi.x, pi.y, vi.x, vi.y, __ldg(&d.V[i]), Fwx,
                     Fwy, d.status);
    }
    // the lane-sum pass may have summed the parts already (f.bx / f.by hold the total)
    const float fx = total ? f.bx : (f.bx + f.sx) + f.nx, fy = total ? f.by : (f.by + f.sy) + f.ny;
    if (k.store) {
        // per-part output in FP64 (the parts as the lanes summed them, the total as the update uses it)
        d.F[i] = make_double2(f2d_bits(fx) + Fwx, f2d_bits(fy) + Fwy);
        d.parts[i] = make_double2((double)f.bx, (double)f.by);
        d.parts[k.N + i] = make_double2((double)f.sx, (double)f.sy);
        d.parts[2 * (size_t)k.N + i] = make_double2((double)f.nx, (double)f.ny);
        d.parts[3 * (size_t)k.N + i] = make_double2(Fwx, Fwy);
    }
    finish_node32_total<PERSIST>(d, k, i, vin, update_v, vi, ao, fx, fy, walls, Fwx, Fwy, inv_m, ui);
}

}  // namespace pd
