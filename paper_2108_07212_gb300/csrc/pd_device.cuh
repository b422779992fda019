// pd_device.cuh -- device helpers shared by the step kernels.
#pragma once

#include "pd_internal.h"
#include "peridem.h"

namespace pd {

// Contact search grid: square cells of side >= R_c hashed into T buckets
// (T a power of two >= 2N), so every pair closer than R_c lies in the 3x3
// cell block around either node.  Aliasing cells only add candidates, which
// the distance test rejects.
__device__ __forceinline__ int cell_coord(double x, double origin, double cell) {
    double f = floor((x - origin) / cell);
    if (!(f > -1048576.0)) return -1048576;  // also catches NaN
    if (f > 1048576.0) return 1048576;
    return (int)f;
}

__device__ __forceinline__ unsigned cell_bucket(int cx, int cy, unsigned T) {
    return ((unsigned)cx * 73856093u ^ (unsigned)cy * 19349663u) & (T - 1u);
}

// Normal damping (Sec. 4.3, Kelvin-Voigt: -beta_d V_x V_y (v(x,y).e) e with
// beta_d = 2 r_d sqrt(K_n rho / V_y)) and regularised Coulomb friction
// (Sec. 4.2: slip -mu |F_r| v_perp/|v_perp| when |v_perp| > v_thr =
// mu |F_r| dt / (rho V_x), else the sticking force -(rho V_x / dt) v_perp).
// e points from x to y, (vrx, vry) = v(x) - v(y), Fr = |F_r|, Vy the partner
// volume (|S_l| for a wall).  Adds to (fx, fy).
__device__ __forceinline__ void damping_friction64(const KParams &k, double ex, double ey, double vrx, double vry,
                                                   double Fr, double Vx, double Vy, double &fx, double &fy) {
    double beta = 2.0 * k.rd * sqrt(k.Kn * k.rho / Vy);
    double vn = vrx * ex + vry * ey;
    double cd = beta * Vx * Vy * vn;
    double Fdx = -cd * ex, Fdy = -cd * ey;
    double vtx = vrx - vn * ex, vty = vry - vn * ey;
    double vt = sqrt(vtx * vtx + vty * vty);
    double vthr = k.mu * Fr * k.dt / (k.rho * Vx);
    double c = (vt > vthr) ? (k.mu * Fr / vt) : (k.rho * Vx / k.dt);
    double Ffx = -c * vtx, Ffy = -c * vty;
    fx += Fdx + Ffx;
    fy += Fdy + Ffy;
}

// Circular segment of B_R(p) beyond a line at distance d < R (Sec. 4.5).
// With theta = acos(d/R) = atan2(sqrt(R^2 - d^2), d) the paper's closed forms
// read |S| = R^2 (theta - sin theta cos theta) and
// R - |c - p| = R (h1 - 2/3 sin^3 theta) / h1; both are evaluated without
// cancellation (Taylor series in theta below 0.3), because the printed
// pi R^2/2 - R^2 asin(d/R) - d sqrt(R^2 - d^2) loses all digits as d -> R.
__device__ __forceinline__ void wall_segment_stable(double d, double R, double &area, double &gap) {
    const double th = atan2(sqrt((R - d) * (R + d)), d);
    double h1, g;
    if (th < 0.3) {
        const double t2 = th * th;
        double term = (4.0 / 6.0) * th * t2;
        h1 = 0.0;
#pragma unroll
        for (int k = 1; k <= 12; ++k) {
            h1 += term;
            term *= -4.0 * t2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
        const double t5 = t2 * t2 * th;
        double a = (243.0 / 6.0 / 120.0) * t5, b = (16.0 / 120.0) * t5, e = (0.5 / 120.0) * t5;
        g = 0.0;
#pragma unroll
        for (int k = 2; k <= 14; ++k) {
            g += a - b - e;
            const double den = (2.0 * k + 2.0) * (2.0 * k + 3.0);
            a *= -9.0 * t2 / den;
            b *= -4.0 * t2 / den;
            e *= -t2 / den;
        }
    } else {
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
        double term = dth * t2 / 6.0;
        f = 0.0;
#pragma unroll
        for (int k = 1; k <= 12; ++k) {
            f += term;
            term *= -t2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
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
// with velocity v and volume Vx against the four walls at positions wn[0..3]
// (x_lo, x_hi, y_lo, y_hi) moving with normal velocities k.wv.  The repulsion
// of each wall uses the circular segment S_l of B_Rc(p) beyond the wall;
// corners subtract the S_li cap S_lj term (inclusion-exclusion); friction and
// damping follow by substituting e -> e^l, V_y -> |S_l|, p(y) -> c_l.  A node
// past a wall is treated as touching it and counted in
// status[PD_STATUS_PENETRATION].
__device__ __forceinline__ void wall_force64(const KParams &k, const double *wn, double px, double py, double vx,
                                             double vy, double Vx, double &Fx_out, double &Fy_out, int *status) {
    const double Rc = k.Rc, Kn = k.Kn;
    double d[4], ex[4], ey[4];
    d[0] = px - wn[0]; ex[0] = -1.0; ey[0] = 0.0;
    d[1] = wn[1] - px; ex[1] = 1.0;  ey[1] = 0.0;
    d[2] = py - wn[2]; ex[2] = 0.0;  ey[2] = -1.0;
    d[3] = wn[3] - py; ex[3] = 0.0;  ey[3] = 1.0;
    bool near = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (d[l] < 0.0) {
            atomicAdd(&status[PD_STATUS_PENETRATION], 1);
            d[l] = 0.0;
        }
        near |= d[l] < Rc;
    }
    double Fx = 0.0, Fy = 0.0;
    if (near) {
        for (int l = 0; l < 4; ++l) {
            if (!(d[l] < Rc)) continue;
            double A, gap;
            wall_segment_stable(d[l], Rc, A, gap);
            if (!(A > 0.0) || !(gap > 0.0)) continue;
            double Fr = Kn * gap * Vx * A;
            double wvx = (l < 2) ? k.wv[l] : 0.0, wvy = (l < 2) ? 0.0 : k.wv[l];
            double gx = -Fr * ex[l], gy = -Fr * ey[l];
            damping_friction64(k, ex[l], ey[l], vx - wvx, vy - wvy, Fr, Vx, A, gx, gy);
            Fx += gx;
            Fy += gy;
        }
        for (int c = 0; c < 4; ++c) {
            const int i = c >> 1, j = 2 + (c & 1);  // (x_lo|x_hi) x (y_lo|y_hi)
            double di = d[i], dj = d[j];
            if (!(sqrt(di * di + dj * dj) < Rc)) continue;
            double A, lx, ly;
            corner_region_stable(di, dj, Rc, A, lx, ly);
            if (!(A > 0.0)) continue;
            double cx = lx * ex[i] + ly * ex[j], cy = lx * ey[i] + ly * ey[j];
            double cd = sqrt(cx * cx + cy * cy);
            if (!(cd < Rc) || !(cd > 0.0)) continue;
            double ux = cx / cd, uy = cy / cd;
            double Fr = Kn * (Rc - cd) * Vx * A;
            double gx = -Fr * ux, gy = -Fr * uy;
            damping_friction64(k, ux, uy, vx - k.wv[i], vy - k.wv[j], Fr, Vx, A, gx, gy);
            Fx -= gx;
            Fy -= gy;
        }
    }
    Fx_out = Fx;
    Fy_out = Fy;
}

}  // namespace pd
