// pd_force_fp64.cu -- the plain FP64 force + update kernel of one time step.
//
// One thread per node x evaluates, in this order (eq:full, Algorithm 1):
//   f^peri : bond forces over the CSR row of x with irreversible breaking
//            (eq:peri, eq:pmb; Sec. 3.1 |s| > s0 breaks the bond for good),
//   S^nbr  : every node y with |p(y) - p(x)| < R_c from the 3x3 hash-grid
//            cells around p(x), visited in ascending node index,
//   f^self : same-grain y without an intact bond (Sec. 4.4),
//   f^nbr  : other-grain y: repulsion, damping, friction (Secs. 4.1-4.3),
//   f^wall : analytic wall contact (Sec. 4.5),
// then a = F / (rho V) + b / rho and v <- v + dt/2 (a_old + a).
// Damping and friction read the start-of-step velocities v_in; the new
// velocities go to the other buffer so no thread reads a value written in the
// same step.  The file is compiled without FMA contraction: each expression
// rounds as written, in the same order as the textbook evaluation.
#include "pd_device.cuh"

namespace pd {

__global__ void __launch_bounds__(kBlock) k_force64(DevPtrs d, KParams k, int vin, int update_v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.N) return;
    const double2 *__restrict__ vI = d.v[vin];
    const double2 pi = d.p[i];
    const double2 Xi = d.X[i];
    const double Vi = d.V[i];
    const int gi = d.grain[i];
    const double cw = d.g_cw[gi], s0 = d.g_s0[gi], eps = d.g_eps[gi];
    const int r0 = d.row_ptr[i], r1 = d.row_ptr[i + 1];
    uint32_t *bw = d.bits + (size_t)i * k.wpn;

    // ---- peridynamic bonds with breaking
    double Fbx = 0.0, Fby = 0.0;
    {
        int wk = -1;
        uint32_t word = 0;
        bool dirty = false;
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
            const double xi = d.xi[b];
            const double2 pj = d.p[j];
            double dx = pj.x - pi.x, dy = pj.y - pi.y;
            double L = sqrt(dx * dx + dy * dy);
            double s = (L - xi) / xi;
            if (fabs(s) > s0) {
                word |= 1u << (kk & 31);
                dirty = true;
                continue;
            }
            double cws = (k.micro ? cw * (1.0 - xi / eps) : cw) * s;
            double q = cws * Vi * d.V[j] / L;
            Fbx += q * dx;
            Fby += q * dy;
        }
        if (dirty) bw[wk] = word;
    }

    // ---- contact candidates S^nbr, ascending node index
    int cand[kMaxCand];
    int nc = 0;
    {
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
                    const double2 pj = d.p[j];
                    double dx = pj.x - pi.x, dy = pj.y - pi.y;
                    double dd = sqrt(dx * dx + dy * dy);
                    if (dd < k.Rc) {
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

    // ---- self-contact and inter-grain contact
    const double2 vi = vI[i];
    double Fsx = 0.0, Fsy = 0.0, Fnx = 0.0, Fny = 0.0;
    for (int q = 0; q < nc; ++q) {
        const int j = cand[q];
        const double2 pj = d.p[j];
        double dx = pj.x - pi.x, dy = pj.y - pi.y;
        double dd = sqrt(dx * dx + dy * dy);
        if (dd == 0.0) {
            atomicAdd(&d.status[PD_STATUS_COINCIDENT], 1);
            continue;
        }
        double ex = dx / dd, ey = dy / dd;
        const double Vj = d.V[j];
        const double2 vj = vI[j];
        double vrx = vi.x - vj.x, vry = vi.y - vj.y;
        if (d.grain[j] == gi) {
            // intact bond to j?  (row columns ascending: binary search)
            int lo = r0, hi = r1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (d.col[mid] < j) lo = mid + 1; else hi = mid;
            }
            if (lo < r1 && d.col[lo] == j) {
                int kk = lo - r0;
                if (!((bw[kk >> 5] >> (kk & 31)) & 1u)) continue;
            }
            const double2 Xj = d.X[j];
            double xix = Xj.x - Xi.x, xiy = Xj.y - Xi.y;
            double xi = sqrt(xix * xix + xiy * xiy);
            double m;
            if (xi < k.Rc)
                m = (dd < xi) ? cw * (dd - xi) / xi : 0.0;
            else
                m = cw * (dd - k.Rc) / k.Rc;
            if (m == 0.0) continue;
            double f = m * Vi * Vj;
            double gx = f * ex, gy = f * ey;
            damping_friction64(k, ex, ey, vrx, vry, -f, Vi, Vj, gx, gy);
            Fsx += gx;
            Fsy += gy;
        } else {
            double Fr = k.Kn * (k.Rc - dd) * Vi * Vj;
            double gx = -Fr * ex, gy = -Fr * ey;
            damping_friction64(k, ex, ey, vrx, vry, Fr, Vi, Vj, gx, gy);
            Fnx += gx;
            Fny += gy;
        }
    }

    // ---- walls
    double Fwx, Fwy;
    wall_force64(k, d.walls_now, pi.x, pi.y, vi.x, vi.y, Vi, Fwx, Fwy, d.status);

    const double Fx = ((Fbx + Fsx) + Fnx) + Fwx;
    const double Fy = ((Fby + Fsy) + Fny) + Fwy;

    // ---- acceleration and velocity update (Algorithm 1)
    const double m = k.rho * Vi;
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

cudaError_t launch_force_fp64(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s) {
    k_force64<<<(k.N + kBlock - 1) / kBlock, kBlock, 0, s>>>(d, k, vin, update_v);
    return cudaGetLastError();
}

}  // namespace pd
