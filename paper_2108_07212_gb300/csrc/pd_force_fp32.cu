// pd_force_fp32.cu -- FP32-split force kernel of one time step.
//
// Same laws and order as the FP64 kernel (eq:full, Algorithm 1), but the bond,
// self-contact and inter-grain contact arithmetic and the force accumulation
// run on the FP32 pipe; FP64 is kept for the wall terms, the acceleration and
// the velocity update (and for the displacement update in the predict kernel).
//
// Precision design (each force term keeps ~1e-7 relative accuracy):
//  - positions are float-float pairs of the shifted position p + shift, all
//    inside [L, 2L) per axis, so the difference of the high parts of two nearby
//    nodes is exact (Sterbenz) and d = p(y) - p(x) = xi + eta is exact to
//    ~1e-15 relative however far a grain has moved or turned;
//  - |d|^2 is formed as a float-float pair with exact FMA products, and the
//    reference |xi|^2 = h^2 (di^2 + dj^2) from the integer lattice offset of
//    the two nodes, so the stretch s = (|d|^2 - |xi|^2) / (|xi| (|d| + |xi|))
//    (algebraically (|xi+eta| - |xi|)/|xi|, eq:pmb) has no cancellation;
//  - the contact overlap R_c - |d| = (R_c^2 - |d|^2) / (R_c + |d|) likewise;
//  - breaking (Sec. 3.1) is re-decided in FP64, from the FP64 positions and
//    reference lengths, for every bond whose FP32 stretch lies within
//    guard * s0 of s0, so break decisions are the FP64 ones.
#include "pd_device.cuh"

namespace pd {

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |d|^2 of d = (dxh + dxl, dyh + dyl) as a float-float pair (hi, lo).
__device__ __forceinline__ void len2_ff(float dxh, float dxl, float dyh, float dyl, float &hi, float &lo) {
    float px, ex, py, ey, s, es;
    two_prod(dxh, dxh, px, ex);
    two_prod(dyh, dyh, py, ey);
    two_sum(px, py, s, es);
    float r = es + (ex + ey) + 2.f * (dxh * dxl + dyh * dyl);
    hi = __fadd_rn(s, r);
    lo = __fsub_rn(r, __fsub_rn(hi, s));
}

// (ah + al) - (bh + bl) rounded to float; exact high-part difference when the
// two values are within a factor of two of each other.
__device__ __forceinline__ float ff_diff(float ah, float al, float bh, float bl) {
    return __fsub_rn(ah, bh) + (al - bl);
}

__device__ __forceinline__ void damping_friction32(float rd, float Kn, float rho, float dt, float mu, float ex,
                                                   float ey, float vrx, float vry, float Fr, float Vx, float Vy,
                                                   float &fx, float &fy) {
    float beta = 2.0f * rd * sqrtf(Kn * rho / Vy);
    float vn = vrx * ex + vry * ey;
    float cd = beta * Vx * Vy * vn;
    float vtx = vrx - vn * ex, vty = vry - vn * ey;
    float vt = sqrtf(vtx * vtx + vty * vty);
    float vthr = mu * Fr * dt / (rho * Vx);
    float c = (vt > vthr) ? (mu * Fr / vt) : (rho * Vx / dt);
    fx += -cd * ex - c * vtx;
    fy += -cd * ey - c * vty;
}

__global__ void __launch_bounds__(kBlock) k_force32(DevPtrs d, KParams k, int vin, int update_v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.N) return;
    const double2 *__restrict__ vI = d.v[vin];
    const float2 phi = d.ph[i], pli = d.pl[i];
    const int2 li = d.lat[i];
    const int gi = d.grain[i];
    const float4 gq = d.gq[gi];               // (h, h^2 hi, h^2 lo, V)
    const float Vi = gq.w;
    const float cw = (float)d.g_cw[gi], s0 = (float)d.g_s0[gi], eps = (float)d.g_eps[gi];
    const float s0_lo = s0 * (1.0f - k.guard), s0_hi = s0 * (1.0f + k.guard);
    const int r0 = d.row_ptr[i], r1 = d.row_ptr[i + 1];
    uint32_t *bw = d.bits + (size_t)i * k.wpn;
    const float Rc = (float)k.Rc, Kn = (float)k.Kn;

    // ---- bonds
    float Fbx = 0.f, Fby = 0.f;
    {
        int wk = -1;
        uint32_t word = 0;
        bool dirty = false;
        const float VV = Vi * Vi;
        for (int b = r0; b < r1; ++b) {
            const int kk = b - r0;
            if ((kk >> 5) != wk) {
                if (dirty) bw[wk] = word;
                wk = kk >> 5;
                word = bw[wk];
                dirty = false;
            }
            if ((word >> (kk & 31)) & 1u) continue;
            const int j = d.col[b];
            const float2 phj = d.ph[j], plj = d.pl[j];
            const int2 lj = d.lat[j];
            const float dxh = __fsub_rn(phj.x, phi.x), dxl = plj.x - pli.x;
            const float dyh = __fsub_rn(phj.y, phi.y), dyl = plj.y - pli.y;
            float L2h, L2l;
            len2_ff(dxh, dxl, dyh, dyl, L2h, L2l);
            const int di = lj.x - li.x, dj = lj.y - li.y;
            const float nn = (float)(di * di + dj * dj);
            float q, eq;
            two_prod(nn, gq.y, q, eq);                       // |xi|^2 = n h^2
            const float num = ff_diff(L2h, L2l, q, eq + nn * gq.z);
            const float xi = gq.x * sqrtf(nn);
            const float L = sqrtf(L2h);
            const float s = num / (xi * (L + xi));
            const float as = fabsf(s);
            bool brk;
            if (as > s0_lo && as < s0_hi) {
                // guard band: decide with the FP64 stretch of the FP64 path
                const double2 pi = d.p[i], pj = d.p[j];
                double ddx = pj.x - pi.x, ddy = pj.y - pi.y;
                double L64 = sqrt(ddx * ddx + ddy * ddy);
                double xi64 = d.xi[b];
                double s64 = (L64 - xi64) / xi64;
                brk = fabs(s64) > d.g_s0[gi];
            } else {
                brk = as > s0;
            }
            if (brk) {
                word |= 1u << (kk & 31);
                dirty = true;
                continue;
            }
            const float cws = (k.micro ? cw * (1.0f - xi / eps) : cw) * s;
            const float qf = cws * VV / L;
            Fbx += qf * (dxh + dxl);
            Fby += qf * (dyh + dyl);
        }
        if (dirty) bw[wk] = word;
    }

    // ---- contact candidates S^nbr, ascending node index
    int cand[kMaxCand];
    int nc = 0;
    {
        const double2 pi = d.p[i];
        const int cx = cell_coord(pi.x, k.ox, k.cell), cy = cell_coord(pi.y, k.oy, k.cell);
        unsigned seen[9];
        int ns = 0;
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                unsigned bkt = cell_bucket(cx + ox, cy + oy, k.T);
                bool dup = false;
                for (int q = 0; q < ns; ++q) dup |= seen[q] == bkt;
                if (dup) continue;
                seen[ns++] = bkt;
                const int t0 = d.start[bkt], t1 = d.start[bkt + 1];
                for (int t = t0; t < t1; ++t) {
                    const int j = d.sorted[t];
                    if (j == i) continue;
                    const float2 phj = d.ph[j], plj = d.pl[j];
                    float L2h, L2l;
                    len2_ff(__fsub_rn(phj.x, phi.x), plj.x - pli.x, __fsub_rn(phj.y, phi.y), plj.y - pli.y, L2h,
                            L2l);
                    if (ff_diff(k.rc2_hi, k.rc2_lo, L2h, L2l) > 0.f) {
                        if (nc < kMaxCand) {
                            int w = nc++;
                            while (w > 0 && cand[w - 1] > j) {
                                cand[w] = cand[w - 1];
                                --w;
                            }
                            cand[w] = j;
                        } else {
                            atomicAdd(&d.status[PD_STATUS_OVERFLOW], 1);
                        }
                    }
                }
            }
    }

    const double2 vi = vI[i];
    const float rd = (float)k.rd, rho = (float)k.rho, dt = (float)k.dt, mu = (float)k.mu;
    float Fsx = 0.f, Fsy = 0.f, Fnx = 0.f, Fny = 0.f;
    for (int q = 0; q < nc; ++q) {
        const int j = cand[q];
        const float2 phj = d.ph[j], plj = d.pl[j];
        const float dxh = __fsub_rn(phj.x, phi.x), dxl = plj.x - pli.x;
        const float dyh = __fsub_rn(phj.y, phi.y), dyl = plj.y - pli.y;
        float L2h, L2l;
        len2_ff(dxh, dxl, dyh, dyl, L2h, L2l);
        const float dd = sqrtf(L2h);
        if (dd == 0.f) {
            atomicAdd(&d.status[PD_STATUS_COINCIDENT], 1);
            continue;
        }
        const float ex = (dxh + dxl) / dd, ey = (dyh + dyl) / dd;
        const float overlap = ff_diff(k.rc2_hi, k.rc2_lo, L2h, L2l) / (Rc + dd);   // R_c - |d|
        const int gj = d.grain[j];
        const float Vj = d.gq[gj].w;
        const double2 vj = vI[j];
        const float vrx = (float)(vi.x - vj.x), vry = (float)(vi.y - vj.y);
        if (gj == gi) {
            int lo = r0, hi = r1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (d.col[mid] < j) lo = mid + 1; else hi = mid;
            }
            if (lo < r1 && d.col[lo] == j) {
                int kk = lo - r0;
                if (!((bw[kk >> 5] >> (kk & 31)) & 1u)) continue;
            }
            const int2 lj = d.lat[j];
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
            damping_friction32(rd, Kn, rho, dt, mu, ex, ey, vrx, vry, -f, Vi, Vj, gx, gy);
            Fsx += gx;
            Fsy += gy;
        } else {
            const float Fr = Kn * overlap * Vi * Vj;
            float gx = -Fr * ex, gy = -Fr * ey;
            damping_friction32(rd, Kn, rho, dt, mu, ex, ey, vrx, vry, Fr, Vi, Vj, gx, gy);
            Fnx += gx;
            Fny += gy;
        }
    }

    // ---- walls (FP64; only nodes within R_c of a wall do work)
    const double2 pi64 = d.p[i];
    const double Vi64 = d.V[i];
    double Fwx, Fwy;
    wall_force64(k, d.walls_now, pi64.x, pi64.y, vi.x, vi.y, Vi64, Fwx, Fwy, d.status);

    const double Fx = (double)((Fbx + Fsx) + Fnx) + Fwx;
    const double Fy = (double)((Fby + Fsy) + Fny) + Fwy;

    const double m = k.rho * Vi64;
    const double ax = Fx / m + k.gx, ay = Fy / m + k.gy;
    if (update_v) {
        const double2 ao = d.a[i];
        double2 vn;
        vn.x = vi.x + k.half_dt * (ao.x + ax);
        vn.y = vi.y + k.half_dt * (ao.y + ay);
        d.v[vin ^ 1][i] = vn;
    }
    d.a[i] = make_double2(ax, ay);
    if (!isfinite(ax) || !isfinite(ay)) atomicAdd(&d.status[PD_STATUS_NONFINITE], 1);
    if (k.store) {
        d.F[i] = make_double2(Fx, Fy);
        d.parts[i] = make_double2(Fbx, Fby);
        d.parts[k.N + i] = make_double2(Fsx, Fsy);
        d.parts[2 * (size_t)k.N + i] = make_double2(Fnx, Fny);
        d.parts[3 * (size_t)k.N + i] = make_double2(Fwx, Fwy);
    }
}

cudaError_t launch_force_fp32(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s) {
    k_force32<<<(k.N + kBlock - 1) / kBlock, kBlock, 0, s>>>(d, k, vin, update_v);
    return cudaGetLastError();
}

}  // namespace pd
