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

// Wall contact (Sec. 4.5, eq:wall-repulsive, eq:wall-total) of a node at p
// with velocity v and volume Vx against the four walls at positions wn[0..3]
// (x_lo, x_hi, y_lo, y_hi) moving with normal velocities k.wv.  The repulsion
// of each wall uses the circular segment S_l of B_Rc(p) beyond the wall (area
// and centroid distance in closed form); corners subtract the S_li cap S_lj
// term (inclusion-exclusion); friction and damping follow by substituting
// e -> e^l, V_y -> |S_l|, p(y) -> c_l.  A node past a wall is treated as
// touching it and counted in status[PD_STATUS_PENETRATION].
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
        const double R2 = Rc * Rc;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (!(d[l] < Rc)) continue;
            double q = R2 - d[l] * d[l];
            double A = 0.5 * 3.14159265358979323846 * Rc * Rc - Rc * Rc * asin(d[l] / Rc) - sqrt(q) * d[l];
            double cd = (2.0 / 3.0) * (q * sqrt(q)) / A;
            if (!(A > 0.0) || !(cd < Rc)) continue;
            double Fr = Kn * (Rc - cd) * Vx * A;
            double wvx = (l < 2) ? k.wv[l] : 0.0, wvy = (l < 2) ? 0.0 : k.wv[l];
            double gx = -Fr * ex[l], gy = -Fr * ey[l];
            damping_friction64(k, ex[l], ey[l], vx - wvx, vy - wvy, Fr, Vx, A, gx, gy);
            Fx += gx;
            Fy += gy;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = c >> 1, j = 2 + (c & 1);  // (x_lo|x_hi) x (y_lo|y_hi)
            double di = d[i], dj = d[j];
            if (!(sqrt(di * di + dj * dj) < Rc)) continue;
            double qi = R2 - di * di, qj = R2 - dj * dj;
            double A = -0.5 * R2 * asin(di / Rc) + 0.5 * R2 * asin(sqrt(qj) / Rc) + di * dj - 0.5 * sqrt(qi) * di -
                       0.5 * sqrt(qj) * dj;
            if (!(A > 0.0)) continue;
            double Ix = dj * dj * dj / 6.0 - 0.5 * qi * dj + (qi * sqrt(qi)) / 3.0;
            double Iy = -0.5 * R2 * di + di * di * di / 6.0 + 0.5 * di * dj * dj + (qj * sqrt(qj)) / 3.0;
            double cx = (Ix * ex[i] + Iy * ex[j]) / A, cy = (Ix * ey[i] + Iy * ey[j]) / A;
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
