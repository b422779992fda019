/*
 * peridem_oracle.c -- plain, slow, FP64 CPU oracle of the PeriDEM force loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the GPU library: it has its own mesher, its own bond builder (the exact
 * segment-in-domain definition of the non-convex horizon, not the paper's
 * extended-boundary construction), its own contact search and its own time
 * loop.  Every function follows the paper's notation and cites the passage it
 * implements.
 *
 * Paper: Bhattacharya & Lipton, "Simulating grain shape effects and damage in
 * granular media using PeriDEM" (arXiv 2108.07212).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - horizon membership is the strict |xi| < eps of Algorithm 1, evaluated on
 *     the integer lattice offsets (di^2 + dj^2 < (eps/h)^2);
 *   - each pair law (bond, contact, self-contact, wall) is evaluated as the
 *     force on node x; rho V_x u'' = sum of those forces + rho V_x b;
 *   - normal damping is the Kelvin-Voigt form -beta_d V_x V_y (v(x,y).e) e with
 *     e pointing from x to y (dissipative sign, Sec. 4.3 energy identity);
 *   - friction opposes the tangential relative velocity v_perp(x,y); slip when
 *     |v_perp| > v_thr, otherwise the sticking force -(rho V_x / dt) v_perp;
 *   - damping and friction use the velocity at the start of the step;
 *   - a bond whose |s| exceeds s0 breaks at that evaluation and carries no force
 *     from then on; self-contact acts between same-grain nodes with no intact
 *     bond; self-contact damping/friction use the contact beta_d and |F_r^self|
 *     and act only while the self repulsion is active;
 *   - wall contact uses the literal R_c - |c_l - p| of Eq. (wall-repulsive); a
 *     node past a wall is treated as touching it (d clamped to 0, counted);
 *     only adjacent (perpendicular) walls form corners.
 *
 * multi-grain trajectories are pinned by their invariants only (linear and
 * angular momentum to rounding, energy to the velocity-Verlet error); parity
 * unpinned beyond them (only the GPU comparison checks the exact trajectory;
 * the paper gives no trajectory data).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* geometry helpers                                                          */

static double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

/* distance from point (px,py) to the closed segment (ax,ay)-(bx,by) */
static double point_segment_distance(double px, double py, double ax, double ay, double bx, double by)
{
    double ex = bx - ax, ey = by - ay;
    double len2 = ex * ex + ey * ey;
    double t = 0.0;
    if (len2 > 0.0) {
        t = ((px - ax) * ex + (py - ay) * ey) / len2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double qx = ax + t * ex - px, qy = ay + t * ey - py;
    return sqrt(qx * qx + qy * qy);
}

/* even-odd point-in-region test over all loops (outer + holes) */
static int point_in_loops(double px, double py, const double *xy, const int *loop_start, int n_loops, double scale)
{
    int inside = 0;
    for (int l = 0; l < n_loops; ++l) {
        int a = loop_start[l], n = loop_start[l + 1] - a;
        for (int k = 0; k < n; ++k) {
            int k1 = (k + 1) % n;
            double x0 = scale * xy[2 * (a + k)], y0 = scale * xy[2 * (a + k) + 1];
            double x1 = scale * xy[2 * (a + k1)], y1 = scale * xy[2 * (a + k1) + 1];
            if ((y0 > py) != (y1 > py)) {
                double xc = x0 + (py - y0) * (x1 - x0) / (y1 - y0);
                if (px < xc) inside = !inside;
            }
        }
    }
    return inside;
}

static double distance_to_loops(double px, double py, const double *xy, const int *loop_start, int n_loops, double scale)
{
    double best = 1e300;
    for (int l = 0; l < n_loops; ++l) {
        int a = loop_start[l], n = loop_start[l + 1] - a;
        for (int k = 0; k < n; ++k) {
            int k1 = (k + 1) % n;
            double d = point_segment_distance(px, py, scale * xy[2 * (a + k)], scale * xy[2 * (a + k) + 1],
                                              scale * xy[2 * (a + k1)], scale * xy[2 * (a + k1) + 1]);
            if (d < best) best = d;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Mesh: uniform lattice of spacing h (Sec. 5 intro: nodes inside the grain,  */
/* V = h^2 per node in 2D).  Lattice points (i h, j h) of the grain frame that */
/* lie strictly inside the grain (even-odd over all loops) and at least        */
/* clear*h away from its boundary are kept, ordered by j then i, then rotated  */
/* by theta and translated to (cx, cy).                                       */
/* Returns the node count; writes at most max_nodes nodes.                    */
int or_mesh_grain(const double *xy, const int *loop_start, int n_loops, double R, double h,
                  double cx, double cy, double theta, double clear, int max_nodes,
                  double *X, int *lat)
{
    int m = (int)ceil(R / h) + 1;
    double c = cos(theta), s = sin(theta);
    int n = 0;
    for (int j = -m; j <= m; ++j) {
        for (int i = -m; i <= m; ++i) {
            double lx = (double)i * h, ly = (double)j * h;
            if (!point_in_loops(lx, ly, xy, loop_start, n_loops, R)) continue;
            if (distance_to_loops(lx, ly, xy, loop_start, n_loops, R) < clear * h) continue;
            if (n < max_nodes) {
                X[2 * n] = cx + (c * lx - s * ly);
                X[2 * n + 1] = cy + (s * lx + c * ly);
                lat[2 * n] = i;
                lat[2 * n + 1] = j;
            }
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Non-convex horizon, Sec. 4 "Peridynamic bonds in nonconvex domains":      */
/* y is removed from the horizon of x when the straight segment x->y leaves   */
/* the (closed) grain D.  This is the definition of the set C_x itself,       */
/* evaluated directly: the segment is cut at every crossing or touching with  */
/* a boundary edge and the midpoint of every piece must lie in closed D       */
/* (inside, or within tol of the boundary).                                   */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int or_segment_in_domain(double ax, double ay, double bx, double by, const double *xy,
                         const int *loop_start, int n_loops, double scale, double tol)
{
    int n_edges = loop_start[n_loops];
    double *ts = (double *)malloc(sizeof(double) * (size_t)(2 * n_edges + 2));
    int nt = 0;
    ts[nt++] = 0.0;
    ts[nt++] = 1.0;
    double rx = bx - ax, ry = by - ay;
    double rlen2 = rx * rx + ry * ry;
    for (int l = 0; l < n_loops; ++l) {
        int a = loop_start[l], n = loop_start[l + 1] - a;
        for (int k = 0; k < n; ++k) {
            int k1 = (k + 1) % n;
            double cxv = scale * xy[2 * (a + k)], cyv = scale * xy[2 * (a + k) + 1];
            double dxv = scale * xy[2 * (a + k1)], dyv = scale * xy[2 * (a + k1) + 1];
            double sx = dxv - cxv, sy = dyv - cyv;
            double den = cross2(rx, ry, sx, sy);
            double qx = cxv - ax, qy = cyv - ay;
            if (fabs(den) > 1e-14 * sqrt(rlen2 * (sx * sx + sy * sy))) {
                double t = cross2(qx, qy, sx, sy) / den;
                double u = cross2(qx, qy, rx, ry) / den;
                if (t >= 0.0 && t <= 1.0 && u >= -1e-12 && u <= 1.0 + 1e-12) ts[nt++] = t;
            } else if (fabs(cross2(qx, qy, rx, ry)) <= 1e-14 * rlen2) {
                /* collinear: the edge end points split the segment */
                double t0 = (qx * rx + qy * ry) / rlen2;
                double t1 = ((dxv - ax) * rx + (dyv - ay) * ry) / rlen2;
                if (t0 > 0.0 && t0 < 1.0) ts[nt++] = t0;
                if (t1 > 0.0 && t1 < 1.0) ts[nt++] = t1;
            }
        }
    }
    qsort(ts, (size_t)nt, sizeof(double), cmp_double);
    int ok = 1;
    for (int k = 0; k + 1 < nt && ok; ++k) {
        if (ts[k + 1] - ts[k] <= 1e-15) continue;
        double tm = 0.5 * (ts[k] + ts[k + 1]);
        double mx = ax + tm * rx, my = ay + tm * ry;
        if (!point_in_loops(mx, my, xy, loop_start, n_loops, scale) &&
            distance_to_loops(mx, my, xy, loop_start, n_loops, scale) > tol)
            ok = 0;
    }
    free(ts);
    return ok;
}

/* Reference neighbour list S^ref(x) of Algorithm 1 for one grain, in local   */
/* node indices: every node y != x of the same grain whose lattice offset     */
/* satisfies di^2 + dj^2 < (eps/h)^2 and whose segment stays inside the grain. */
/* Columns are ascending.  row_ptr has n+1 entries.  Returns the bond count    */
/* (writes at most max_bonds columns).                                        */
int or_grain_bonds(const double *xy, const int *loop_start, int n_loops, double R, double h,
                   double horizon_ratio, double tol_frac, int n, const int *lat,
                   int *row_ptr, int *col, int max_bonds)
{
    if (n <= 0) {
        row_ptr[0] = 0;
        return 0;
    }
    int imin = 1 << 30, imax = -(1 << 30), jmin = 1 << 30, jmax = -(1 << 30);
    for (int k = 0; k < n; ++k) {
        if (lat[2 * k] < imin) imin = lat[2 * k];
        if (lat[2 * k] > imax) imax = lat[2 * k];
        if (lat[2 * k + 1] < jmin) jmin = lat[2 * k + 1];
        if (lat[2 * k + 1] > jmax) jmax = lat[2 * k + 1];
    }
    int W = imax - imin + 1, H = jmax - jmin + 1;
    int *map = (int *)malloc(sizeof(int) * (size_t)W * (size_t)H);
    for (int k = 0; k < W * H; ++k) map[k] = -1;
    for (int k = 0; k < n; ++k) map[(lat[2 * k + 1] - jmin) * W + (lat[2 * k] - imin)] = k;
    int r = (int)ceil(horizon_ratio);
    double r2 = horizon_ratio * horizon_ratio;
    int nb = 0;
    int cand[1024];
    for (int x = 0; x < n; ++x) {
        row_ptr[x] = nb;
        int nc = 0;
        int ix = lat[2 * x], jx = lat[2 * x + 1];
        for (int dj = -r; dj <= r; ++dj) {
            for (int di = -r; di <= r; ++di) {
                if (di == 0 && dj == 0) continue;
                if ((double)(di * di + dj * dj) >= r2) continue;
                int iy = ix + di, jy = jx + dj;
                if (iy < imin || iy > imax || jy < jmin || jy > jmax) continue;
                int y = map[(jy - jmin) * W + (iy - imin)];
                if (y < 0) continue;
                if (!or_segment_in_domain((double)ix * h, (double)jx * h, (double)iy * h, (double)jy * h,
                                          xy, loop_start, n_loops, R, tol_frac * h))
                    continue;
                if (nc < 1024) cand[nc++] = y;
            }
        }
        /* ascending column order (insertion sort) */
        for (int a = 1; a < nc; ++a) {
            int v = cand[a], b = a - 1;
            while (b >= 0 && cand[b] > v) { cand[b + 1] = cand[b]; --b; }
            cand[b + 1] = v;
        }
        for (int a = 0; a < nc; ++a) {
            if (nb < max_bonds) col[nb] = cand[a];
            ++nb;
        }
    }
    row_ptr[n] = nb;
    free(map);
    return nb;
}

/* ------------------------------------------------------------------------ */
/* Material constants, Table 1 (tab:2d-peri).                                 */
/* micromodulus 0: constant w = 1,  c_w = 6E/(pi eps^3 (1-nu)),               */
/*                 s0 = sqrt(4 pi Gc / (9 E eps))                             */
/* micromodulus 1: conic w = 1-|xi|/eps, c_w = 24E/(pi eps^3 (1-nu)),          */
/*                 s0 = sqrt(5 pi Gc / (9 E eps))                             */
void or_bond_constants(double E, double nu, double Gc, double eps, int micromodulus, double *cw, double *s0)
{
    if (micromodulus == 0) {
        *cw = 6.0 * E / (OR_PI * eps * eps * eps * (1.0 - nu));
        *s0 = sqrt(4.0 * OR_PI * Gc / (9.0 * E * eps));
    } else {
        *cw = 24.0 * E / (OR_PI * eps * eps * eps * (1.0 - nu));
        *s0 = sqrt(5.0 * OR_PI * Gc / (9.0 * E * eps));
    }
}

/* Normal contact stiffness K_n = 18 k / (pi eps^5), Sec. 4.1. */
double or_contact_stiffness(double k_bulk, double eps)
{
    return 18.0 * k_bulk / (OR_PI * eps * eps * eps * eps * eps);
}

/* Single-wall contact region S_l, Sec. 4.5: the circular segment of B_{R_c}(p)
 * beyond a line at distance d.  The paper's closed forms
 *   |S_l| = pi R^2/2 - R^2 asin(d/R) - sqrt(R^2 - d^2) d,
 *   |c_l - p| = 2/3 (R^2 - d^2)^{3/2} / |S_l|
 * cancel catastrophically as d -> R (the segment vanishes), so they are
 * evaluated through the half-angle theta = acos(d/R) = atan2(sqrt(R^2-d^2), d):
 *   |S_l| = R^2 h1(theta),  h1 = theta - sin(theta) cos(theta),
 *   R - |c_l - p| = R g(theta) / h1(theta),  g = h1 - 2/3 sin^3(theta),
 * with the Taylor series of h1 and g (g starts at 0.2 theta^5) for small theta.
 * gap returns R_c - |c_l - p|, the factor of eq. (wall-repulsive). */
static void segment_shape(double th, double *h1, double *g)
{
    if (th < 0.3) {
        double t2 = th * th;
        /* h1 = sum_{k>=1} (-1)^{k+1} 4^k th^{2k+1} / (2k+1)! */
        double term = 4.0 * th * t2 / 6.0, sum = 0.0;
        for (int k = 1; k <= 12; ++k) {
            sum += term;
            term *= -4.0 * t2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
        *h1 = sum;
        /* g = sum_{k>=2} (-1)^k (3^{2k+1}/6 - 4^k - 1/2) th^{2k+1} / (2k+1)! */
        double t5 = t2 * t2 * th;
        double a = 243.0 / 6.0 * t5 / 120.0, b = 16.0 * t5 / 120.0, e = 0.5 * t5 / 120.0;
        double gs = 0.0;
        for (int k = 2; k <= 14; ++k) {
            gs += a - b - e;
            double den = (2.0 * k + 2.0) * (2.0 * k + 3.0);
            a *= -9.0 * t2 / den;
            b *= -4.0 * t2 / den;
            e *= -t2 / den;
        }
        *g = gs;
    } else {
        double sn = sin(th), cs = cos(th);
        *h1 = th - sn * cs;
        *g = *h1 - (2.0 / 3.0) * sn * sn * sn;
    }
}

void or_wall_segment_gap(double d, double Rc, double *area, double *gap)
{
    double q = (Rc - d) * (Rc + d);
    double th = atan2(sqrt(q), d);
    double h1, g;
    segment_shape(th, &h1, &g);
    *area = Rc * Rc * h1;
    *gap = Rc * g / h1;
}

void or_wall_segment(double d, double Rc, double *area, double *cdist)
{
    double gap;
    or_wall_segment_gap(d, Rc, area, &gap);
    *cdist = Rc - gap;
}

/* Corner region S_li cap S_lj, Sec. 4.5.  Local frame: x towards l_i (at
 * distance d_i), y towards l_j (distance d_j), p at the origin; the region is
 * {x >= d_i, y >= d_j, |.| <= R}.  The paper's polar integrals for the area
 * and the moments I_x, I_y cancel as the corner point approaches the circle,
 * so the same region is split into the triangle Q P1 P2 (Q = (d_i, d_j),
 * P1 = (b, d_j), P2 = (d_i, c) on the circle) and the circular segment cut by
 * the chord P1 P2 (angle dth); both parts have positive area.  Returns the
 * area and the first moments I_x, I_y (centroid = (I_x, I_y) / area). */
void or_corner_region(double di, double dj, double Rc, double *area, double *Ix, double *Iy)
{
    double b = sqrt((Rc - dj) * (Rc + dj)), c = sqrt((Rc - di) * (Rc + di));
    double w = (Rc - di) * (Rc + di) - dj * dj;          /* R^2 - di^2 - dj^2 >= 0 */
    double bmi = w / (b + di), cmj = w / (c + dj);        /* b - di, c - dj */
    double T = 0.5 * bmi * cmj;
    double cr = b * cmj + dj * bmi;                       /* P1 x P2 = b c - di dj */
    double dt = b * di + dj * c;                          /* P1 . P2 */
    double dth = atan2(cr, dt);
    double f;                                             /* dth - sin(dth) */
    if (dth < 0.5) {
        double t2 = dth * dth, term = dth * t2 / 6.0;
        f = 0.0;
        for (int k = 1; k <= 12; ++k) {
            f += term;
            term *= -t2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
        }
    } else {
        f = dth - sin(dth);
    }
    double Sg = 0.5 * Rc * Rc * f;
    /* segment centroid: on the chord bisector, at 4 R sin^3(dth/2) / (3 (dth - sin dth)) */
    double mx = b + di, my = dj + c, ml = sqrt(mx * mx + my * my);
    double s2 = sin(0.5 * dth);
    double sd;
    if (dth < 0.5) {
        /* 4 sin^3(x/2) / (3 (x - sin x)) -> 1 as x -> 0: evaluate as ratio of series-safe parts */
        sd = (dth > 0.0) ? Rc * (4.0 * s2 * s2 * s2) / (3.0 * f) : Rc;
    } else {
        sd = Rc * (4.0 * s2 * s2 * s2) / (3.0 * f);
    }
    double sgx = sd * mx / ml, sgy = sd * my / ml;
    double tx = (di + b + di) / 3.0, ty = (dj + dj + c) / 3.0;
    *area = Sg + T;
    *Ix = Sg * sgx + T * tx;
    *Iy = Sg * sgy + T * ty;
}

/* ------------------------------------------------------------------------ */
/* The time loop.                                                             */

/* parameter vector layout */
enum {
    P_RHO = 0, P_KN, P_RC, P_RD, P_MU, P_GX, P_GY, P_DT,
    P_WX0, P_WX1, P_WY0, P_WY1,          /* wall positions at t = 0: x_lo, x_hi, y_lo, y_hi */
    P_VX0, P_VX1, P_VY0, P_VY1,          /* wall normal velocities                           */
    P_MICRO, P_SEARCH,
    P_PE5,                               /* pi eps_c^5 of K_n = 18 k / (pi eps_c^5) (materials) */
    P_NPARAM
};

/* status word layout */
enum { ST_PENETRATION = 0, ST_COINCIDENT, ST_NONFINITE, ST_NSTATUS };

typedef struct {
    const double *prm;
    int N;
    const double *X;
    const double *u, *v;
    const double *V;
    const int *grain;
    const double *g_cw, *g_s0, *g_eps;
    const double *g_mat; /* nullable: per grain (rho, k_bulk); NULL = prm's rho and K_n */
    const int *row_ptr, *col;
    unsigned char *broken;
    double t;            /* time at which the walls are evaluated */
    double *p;           /* scratch: current positions */
    int *cand;           /* scratch: contact candidates */
    int max_cand;
    /* contact grid */
    int use_grid;
    double gx0, gy0, cell;
    int ncx, ncy;
    int *head, *next;
    int *status;
} or_sys;

/* Materials (Sec. 4.1 and the material table of Sec. 5): each grain has its */
/* own density and bulk modulus.  Contact between grains of bulk moduli k1   */
/* and k2 uses K_n = 18 k / (pi eps_c^5) with the harmonic mean              */
/* k = 2 k1 k2 / (k1 + k2) (equal moduli: k itself); a wall uses the grain's  */
/* own k; damping uses the harmonic mean of the two densities (equal: rho),  */
/* friction and mass the node's own density.                                  */
static double harmonic(double a, double b) { return a == b ? a : 2.0 * a * b / (a + b); }

static double rho_of(const or_sys *S, int g) { return S->g_mat ? S->g_mat[2 * g] : S->prm[P_RHO]; }

static double kn_pair(const or_sys *S, int g, int h)
{
    if (!S->g_mat) return S->prm[P_KN];
    return 18.0 * harmonic(S->g_mat[2 * g + 1], S->g_mat[2 * h + 1]) / S->prm[P_PE5];
}

/* cell index along one axis, clamped to the grid (non-finite -> 0) */
static int grid_index(double x, double x0, double cell, int n)
{
    double f = floor((x - x0) / cell);
    if (!(f >= 0.0)) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int)f;
}

/* S^nbr of Algorithm 1: indices y != x with |p(y) - p(x)| < R_c, ascending.  */
static int contact_candidates(const or_sys *S, int x, int *out)
{
    double Rc = S->prm[P_RC];
    double px = S->p[2 * x], py = S->p[2 * x + 1];
    int n = 0;
    if (!(Rc > 0.0)) return 0;
    if (!S->use_grid) {
        for (int y = 0; y < S->N; ++y) {
            if (y == x) continue;
            double dx = S->p[2 * y] - px, dy = S->p[2 * y + 1] - py;
            double d = sqrt(dx * dx + dy * dy);
            if (d < Rc && n < S->max_cand) out[n++] = y;
        }
        return n;
    }
    int ci = grid_index(px, S->gx0, S->cell, S->ncx), cj = grid_index(py, S->gy0, S->cell, S->ncy);
    for (int dj = -1; dj <= 1; ++dj) {
        for (int di = -1; di <= 1; ++di) {
            int a = ci + di, b = cj + dj;
            if (a < 0 || b < 0 || a >= S->ncx || b >= S->ncy) continue;
            for (int y = S->head[b * S->ncx + a]; y >= 0; y = S->next[y]) {
                if (y == x) continue;
                double dx = S->p[2 * y] - px, dy = S->p[2 * y + 1] - py;
                double d = sqrt(dx * dx + dy * dy);
                if (d < Rc && n < S->max_cand) out[n++] = y;
            }
        }
    }
    for (int a = 1; a < n; ++a) {
        int v = out[a], b = a - 1;
        while (b >= 0 && out[b] > v) { out[b + 1] = out[b]; --b; }
        out[b + 1] = v;
    }
    return n;
}

static void build_grid(or_sys *S)
{
    double Rc = S->prm[P_RC];
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int k = 0; k < S->N; ++k) {
        double x = S->p[2 * k], y = S->p[2 * k + 1];
        if (!isfinite(x) || !isfinite(y)) continue;
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    S->cell = Rc;
    S->gx0 = xmin - Rc;
    S->gy0 = ymin - Rc;
    if (!(xmax >= xmin)) { xmin = xmax = 0.0; ymin = ymax = 0.0; S->gx0 = -Rc; S->gy0 = -Rc; }
    S->ncx = (int)((xmax - S->gx0) / Rc) + 3;
    S->ncy = (int)((ymax - S->gy0) / Rc) + 3;
    size_t nc = (size_t)S->ncx * (size_t)S->ncy;
    S->head = (int *)malloc(sizeof(int) * nc);
    S->next = (int *)malloc(sizeof(int) * (size_t)(S->N > 0 ? S->N : 1));
    for (size_t k = 0; k < nc; ++k) S->head[k] = -1;
    for (int k = S->N - 1; k >= 0; --k) {
        int ci = grid_index(S->p[2 * k], S->gx0, Rc, S->ncx), cj = grid_index(S->p[2 * k + 1], S->gy0, Rc, S->ncy);
        int c = cj * S->ncx + ci;
        S->next[k] = S->head[c];
        S->head[c] = k;
    }
}

static void free_grid(or_sys *S)
{
    free(S->head);
    free(S->next);
    S->head = S->next = NULL;
}

/* Damping + friction of a pair, Sec. 4.2-4.3, with e pointing from x to y,   */
/* relative velocity vr = v(x) - v(y), repulsion magnitude Fr (>= 0) and the   */
/* partner volume Vy used in beta_d.  Adds to (fx, fy).                        */
static void damping_friction(const double *prm, double Kn, double rho_d, double rho, double ex, double ey,
                             double vrx, double vry, double Fr, double Vx, double Vy, double *fx, double *fy)
{
    double dt = prm[P_DT], mu = prm[P_MU];
    /* normal damping (eq:normal-damp), Kelvin-Voigt reading; rho_d the pair's */
    /* density, rho the density of x (friction's eps_f = dt / (rho V_x))       */
    double beta = 2.0 * prm[P_RD] * sqrt(Kn * rho_d / Vy);
    double vn = vrx * ex + vry * ey;
    double cd = beta * Vx * Vy * vn;
    double Fdx = -cd * ex, Fdy = -cd * ey;
    /* friction (eq:friction) with threshold v_thr = mu |F_r| dt / (rho V_x) */
    double vtx = vrx - vn * ex, vty = vry - vn * ey;
    double vt = sqrt(vtx * vtx + vty * vty);
    double vthr = mu * Fr * dt / (rho * Vx);
    double Ffx, Ffy;
    if (vt > vthr) {
        double c = mu * Fr / vt;
        Ffx = -c * vtx;
        Ffy = -c * vty;
    } else {
        double c = rho * Vx / dt;
        Ffx = -c * vtx;
        Ffy = -c * vty;
    }
    *fx += Fdx + Ffx;
    *fy += Fdy + Ffy;
}

/* Wall terms on one node, Sec. 4.5 (eq:wall-repulsive, eq:wall-total), with   */
/* friction and damping obtained by the substitution e -> e^l, V_y -> |S_l|,   */
/* p(y) -> c_l: single[l] is the force of wall l (x_lo, x_hi, y_lo, y_hi) by   */
/* its own segment, corner[k] the term of the corner region S_i cap S_j that   */
/* eq:wall-total subtracts (k: (x_lo,y_lo), (x_lo,y_hi), (x_hi,y_lo),          */
/* (x_hi,y_hi)).  The node's wall force is sum single - sum corner.            */
static void wall_terms(const or_sys *S, int x, double single[4][2], double corner[4][2])
{
    const double *prm = S->prm;
    /* a rigid wall: K_n and densities of the node's own material */
    int g = S->grain ? S->grain[x] : 0;
    double Rc = prm[P_RC], Kn = S->grain ? kn_pair(S, g, g) : prm[P_KN];
    double rho = S->grain ? rho_of(S, g) : prm[P_RHO];
    double px = S->p[2 * x], py = S->p[2 * x + 1];
    double vx = S->v[2 * x], vy = S->v[2 * x + 1];
    double Vx = S->V[x];
    double t = S->t;
    double wpos[4], wvel[4], d[4], ex[4], ey[4];
    for (int l = 0; l < 4; ++l) {
        wvel[l] = prm[P_VX0 + l];
        wpos[l] = prm[P_WX0 + l] + wvel[l] * t;
    }
    d[0] = px - wpos[0]; ex[0] = -1.0; ey[0] = 0.0;
    d[1] = wpos[1] - px; ex[1] = 1.0;  ey[1] = 0.0;
    d[2] = py - wpos[2]; ex[2] = 0.0;  ey[2] = -1.0;
    d[3] = wpos[3] - py; ex[3] = 0.0;  ey[3] = 1.0;
    for (int l = 0; l < 4; ++l) {
        if (d[l] < 0.0) {
#pragma omp atomic
            S->status[ST_PENETRATION]++;
            d[l] = 0.0;
        }
    }
    for (int l = 0; l < 4; ++l) {
        single[l][0] = single[l][1] = 0.0;
        corner[l][0] = corner[l][1] = 0.0;
    }
    for (int l = 0; l < 4; ++l) {
        if (!(d[l] < Rc)) continue;
        double A, gap;
        or_wall_segment_gap(d[l], Rc, &A, &gap);
        /* a vanished region (no positive area) exerts no force */
        if (!(A > 0.0) || !(gap > 0.0)) continue;
        double Fr = Kn * gap * Vx * A;
        double wvx = (l < 2) ? wvel[l] : 0.0, wvy = (l < 2) ? 0.0 : wvel[l];
        double gx = -Fr * ex[l], gy = -Fr * ey[l];
        damping_friction(prm, Kn, rho, rho, ex[l], ey[l], vx - wvx, vy - wvy, Fr, Vx, A, &gx, &gy);
        single[l][0] = gx;
        single[l][1] = gy;
    }
    static const int ci[4] = {0, 0, 1, 1}, cj[4] = {2, 3, 2, 3};
    for (int k = 0; k < 4; ++k) {
        int i = ci[k], j = cj[k];
        if (!(sqrt(d[i] * d[i] + d[j] * d[j]) < Rc)) continue;
        double A, Ix, Iy;
        or_corner_region(d[i], d[j], Rc, &A, &Ix, &Iy);
        if (!(A > 0.0)) continue;
        double cx = (Ix * ex[i] + Iy * ex[j]) / A, cy = (Ix * ey[i] + Iy * ey[j]) / A;
        double cd = sqrt(cx * cx + cy * cy);
        if (!(cd < Rc) || !(cd > 0.0)) continue;
        double ux = cx / cd, uy = cy / cd;
        double Fr = Kn * (Rc - cd) * Vx * A;
        double wvx = wvel[i], wvy = wvel[j];
        double gx = -Fr * ux, gy = -Fr * uy;
        damping_friction(prm, Kn, rho, rho, ux, uy, vx - wvx, vy - wvy, Fr, Vx, A, &gx, &gy);
        corner[k][0] = gx;
        corner[k][1] = gy;
    }
}

/* Wall force on one node: eq:wall-total, walls in order then corners. */
static void wall_force(const or_sys *S, int x, double *fx, double *fy)
{
    double single[4][2], corner[4][2];
    wall_terms(S, x, single, corner);
    double Fx = 0.0, Fy = 0.0;
    for (int l = 0; l < 4; ++l) {
        Fx += single[l][0];
        Fy += single[l][1];
    }
    for (int k = 0; k < 4; ++k) {
        Fx -= corner[k][0];
        Fy -= corner[k][1];
    }
    *fx = Fx;
    *fy = Fy;
}

/* Force on node x from all its interactions (eq:full, Algorithm 1 lines for  */
/* f^peri, f^self, f^nbr, f^wall).  parts (nullable) receives the four parts.  */
static void node_force(or_sys *S, int x, int *cand, double *Fx_out, double *Fy_out, double *parts)
{
    const double *prm = S->prm;
    double Rc = prm[P_RC];
    int micro = (int)prm[P_MICRO];
    int g = S->grain[x];
    double rho_x = rho_of(S, g);
    double cw = S->g_cw[g], s0 = S->g_s0[g], eps = S->g_eps[g];
    double px = S->p[2 * x], py = S->p[2 * x + 1];
    double Xx = S->X[2 * x], Xy = S->X[2 * x + 1];
    double Vx = S->V[x];

    /* peridynamic bond force with irreversible breaking (eq:peri, pmb, Sec. 3.1) */
    double Fbx = 0.0, Fby = 0.0;
    for (int b = S->row_ptr[x]; b < S->row_ptr[x + 1]; ++b) {
        if (S->broken[b]) continue;
        int y = S->col[b];
        double xix = S->X[2 * y] - Xx, xiy = S->X[2 * y + 1] - Xy;
        double xi = sqrt(xix * xix + xiy * xiy);
        double dx = S->p[2 * y] - px, dy = S->p[2 * y + 1] - py;
        double L = sqrt(dx * dx + dy * dy);
        double s = (L - xi) / xi;
        if (fabs(s) > s0) {
            S->broken[b] = 1;
            continue;
        }
        double cws = (micro ? cw * (1.0 - xi / eps) : cw) * s;
        double q = cws * Vx * S->V[y] / L;
        Fbx += q * dx;
        Fby += q * dy;
    }

    /* contact candidates S^nbr (all grains, ascending index) */
    int nc = contact_candidates(S, x, cand);
    double Fsx = 0.0, Fsy = 0.0, Fnx = 0.0, Fny = 0.0;
    for (int k = 0; k < nc; ++k) {
        int y = cand[k];
        double dx = S->p[2 * y] - px, dy = S->p[2 * y + 1] - py;
        double d = sqrt(dx * dx + dy * dy);
        if (d == 0.0) {
#pragma omp atomic
            S->status[ST_COINCIDENT]++;
            continue;
        }
        double ex = dx / d, ey = dy / d;
        double Vy = S->V[y];
        double vrx = S->v[2 * x] - S->v[2 * y], vry = S->v[2 * x + 1] - S->v[2 * y + 1];
        if (S->grain[y] == g) {
            /* self-contact (Sec. 4.4) between nodes with no intact bond */
            int bonded = 0;
            for (int b = S->row_ptr[x]; b < S->row_ptr[x + 1]; ++b)
                if (S->col[b] == y && !S->broken[b]) bonded = 1;
            if (bonded) continue;
            double xix = S->X[2 * y] - Xx, xiy = S->X[2 * y + 1] - Xy;
            double xi = sqrt(xix * xix + xiy * xiy);
            double m;
            if (xi < Rc)
                m = (d < xi) ? cw * (d - xi) / xi : 0.0;
            else
                m = cw * (d - Rc) / Rc;
            if (m == 0.0) continue;
            double f = m * Vx * Vy;          /* negative: pushes x away from y */
            double gx = f * ex, gy = f * ey;
            damping_friction(prm, kn_pair(S, g, g), rho_x, rho_x, ex, ey, vrx, vry, -f, Vx, Vy, &gx, &gy);
            Fsx += gx;
            Fsy += gy;
        } else {
            /* inter-grain contact: repulsion (eq:law-repulsive), damping, friction */
            int gy_ = S->grain[y];
            double Kn = kn_pair(S, g, gy_);
            double Fr = Kn * (Rc - d) * Vx * Vy;
            double gx = -Fr * ex, gy = -Fr * ey;
            damping_friction(prm, Kn, harmonic(rho_x, rho_of(S, gy_)), rho_x, ex, ey, vrx, vry, Fr, Vx, Vy, &gx,
                             &gy);
            Fnx += gx;
            Fny += gy;
        }
    }

    double Fwx, Fwy;
    wall_force(S, x, &Fwx, &Fwy);

    *Fx_out = ((Fbx + Fsx) + Fnx) + Fwx;
    *Fy_out = ((Fby + Fsy) + Fny) + Fwy;
    if (parts) {
        parts[2 * x] = Fbx;                 parts[2 * x + 1] = Fby;
        parts[2 * S->N + 2 * x] = Fsx;      parts[2 * S->N + 2 * x + 1] = Fsy;
        parts[4 * S->N + 2 * x] = Fnx;      parts[4 * S->N + 2 * x + 1] = Fny;
        parts[6 * S->N + 2 * x] = Fwx;      parts[6 * S->N + 2 * x + 1] = Fwy;
    }
}

static void sys_init(or_sys *S, const double *prm, int N, const double *X, const double *u, const double *v,
                     const double *V, const int *grain, const double *g_cw, const double *g_s0,
                     const double *g_eps, const double *g_mat, const int *row_ptr, const int *col,
                     unsigned char *broken, int *status)
{
    memset(S, 0, sizeof(*S));
    S->prm = prm; S->N = N; S->X = X; S->u = u; S->v = v; S->V = V; S->grain = grain;
    S->g_cw = g_cw; S->g_s0 = g_s0; S->g_eps = g_eps; S->g_mat = g_mat; S->row_ptr = row_ptr; S->col = col;
    S->broken = broken; S->status = status;
    S->p = (double *)malloc(sizeof(double) * (size_t)(2 * (N > 0 ? N : 1)));
    S->max_cand = 4096;
    S->cand = (int *)malloc(sizeof(int) * (size_t)S->max_cand);
    S->use_grid = ((int)prm[P_SEARCH]) != 0;
}

static void sys_free(or_sys *S)
{
    free(S->p);
    free(S->cand);
}

static void all_forces(or_sys *S, double *F, double *parts)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < 2 * S->N; ++k) S->p[k] = S->X[k] + S->u[k];
    int grid = S->use_grid && S->prm[P_RC] > 0.0 && S->N > 0;
    if (grid) build_grid(S);
    /* Nodes are independent: each writes only its own force and the broken  */
    /* flags of its own bonds.  The all-core build (-fopenmp) splits them     */
    /* over threads, each with its own candidate scratch; the arithmetic of   */
    /* every node is the same as in the single-threaded build.                */
#pragma omp parallel
    {
        int *cand = (int *)malloc(sizeof(int) * (size_t)S->max_cand);
#pragma omp for schedule(static)
        for (int x = 0; x < S->N; ++x) node_force(S, x, cand, &F[2 * x], &F[2 * x + 1], parts);
        free(cand);
    }
    if (grid) free_grid(S);
}

/* One force evaluation at the current (u, v) with walls at time t.  Breaks  */
/* bonds as a side effect (pass a copy of `broken` to keep it).  F: 2N total  */
/* force; parts (nullable): 8N = bond | self | neighbour | wall.              */
void or_forces(const double *prm, double t, int N, const double *X, const double *u, const double *v,
               const double *V, const int *grain, const double *g_cw, const double *g_s0,
               const double *g_eps, const double *g_mat, const int *row_ptr, const int *col,
               unsigned char *broken, double *F, double *parts, int *status)
{
    or_sys S;
    sys_init(&S, prm, N, X, u, v, V, grain, g_cw, g_s0, g_eps, g_mat, row_ptr, col, broken, status);
    S.t = t;
    all_forces(&S, F, parts);
    sys_free(&S);
}

/* Sums over all nodes of the wall terms at the current state (walls at time */
/* t): out[2 l + c] for wall l's own segment, out[8 + 2 k + c] for corner k   */
/* (the orders of wall_terms).  Used for the force the aggregate exerts on a  */
/* wall (Sec. 6, compaction: force on the top wall).                          */
void or_wall_sums(const double *prm, double t, int N, const double *X, const double *u, const double *v,
                  const double *V, const int *grain, const double *g_mat, double *out)
{
    or_sys S;
    sys_init(&S, prm, N, X, u, v, V, grain, NULL, NULL, NULL, g_mat, NULL, NULL, NULL, NULL);
    S.t = t;
    int status[8] = {0};
    S.status = status;
    for (int q = 0; q < 16; ++q) out[q] = 0.0;
    for (int k = 0; k < 2 * N; ++k) S.p[k] = X[k] + u[k];
    for (int x = 0; x < N; ++x) {
        double single[4][2], corner[4][2];
        wall_terms(&S, x, single, corner);
        for (int l = 0; l < 4; ++l) {
            out[2 * l] += single[l][0];
            out[2 * l + 1] += single[l][1];
            out[8 + 2 * l] += corner[l][0];
            out[8 + 2 * l + 1] += corner[l][1];
        }
    }
    sys_free(&S);
}

/* Algorithm 1: n_steps velocity-Verlet steps starting at step index step0   */
/* (time t = step0 * dt).  On entry `a` holds the acceleration of the current */
/* state.  F_last/parts_last (nullable) receive the forces of the last step.  */
void or_run(const double *prm, long step0, int n_steps, int N, const double *X, double *u, double *v,
            double *a, const double *V, const int *grain, const double *g_cw, const double *g_s0,
            const double *g_eps, const double *g_mat, const int *row_ptr, const int *col,
            unsigned char *broken, double *F_last, double *parts_last, int *status)
{
    double dt = prm[P_DT], gx = prm[P_GX], gy = prm[P_GY];
    double half_dt = 0.5 * dt, half_dt2 = 0.5 * dt * dt;
    double *F = (double *)malloc(sizeof(double) * (size_t)(2 * (N > 0 ? N : 1)));
    or_sys S;
    sys_init(&S, prm, N, X, u, v, V, grain, g_cw, g_s0, g_eps, g_mat, row_ptr, col, broken, status);
    for (int n = 0; n < n_steps; ++n) {
        long step = step0 + n;
        /* displacement update, current position (Algorithm 1) */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < 2 * N; ++k) u[k] = (u[k] + dt * v[k]) + half_dt2 * a[k];
        S.t = (double)(step + 1) * dt;
        all_forces(&S, F, (n == n_steps - 1) ? parts_last : NULL);
        /* acceleration and velocity update (Algorithm 1) */
#pragma omp parallel for schedule(static)
        for (int x = 0; x < N; ++x) {
            double m = rho_of(&S, grain[x]) * V[x];
            double ax = F[2 * x] / m + gx, ay = F[2 * x + 1] / m + gy;
            v[2 * x] = v[2 * x] + half_dt * (a[2 * x] + ax);
            v[2 * x + 1] = v[2 * x + 1] + half_dt * (a[2 * x + 1] + ay);
            a[2 * x] = ax;
            a[2 * x + 1] = ay;
            if (!isfinite(ax) || !isfinite(ay)) {
#pragma omp atomic
                status[ST_NONFINITE]++;
            }
        }
    }
    if (F_last) memcpy(F_last, F, sizeof(double) * (size_t)(2 * N));
    sys_free(&S);
    free(F);
}

/* Initial acceleration a^0 = F(u^0, v^0) / (rho V) + b / rho at t = t0        */
/* (first line of Algorithm 1).                                               */
void or_init_accel(const double *prm, double t0, int N, const double *X, const double *u, const double *v,
                   double *a, const double *V, const int *grain, const double *g_cw, const double *g_s0,
                   const double *g_eps, const double *g_mat, const int *row_ptr, const int *col,
                   unsigned char *broken, int *status)
{
    double gx = prm[P_GX], gy = prm[P_GY];
    double *F = (double *)malloc(sizeof(double) * (size_t)(2 * (N > 0 ? N : 1)));
    or_forces(prm, t0, N, X, u, v, V, grain, g_cw, g_s0, g_eps, g_mat, row_ptr, col, broken, F, NULL, status);
    for (int x = 0; x < N; ++x) {
        double m = (g_mat ? g_mat[2 * grain[x]] : prm[P_RHO]) * V[x];
        a[2 * x] = F[2 * x] / m + gx;
        a[2 * x + 1] = F[2 * x + 1] / m + gy;
    }
    free(F);
}

/* Diagnostics: kinetic energy, bond (micro-potential) energy, node-node     */
/* contact potential, linear and angular momentum.  out[0..6] =               */
/* KE, E_bond, E_contact, Px, Py, Lz, n_broken (directed bonds).             */
void or_diagnostics(const double *prm, int N, const double *X, const double *u, const double *v,
                    const double *V, const int *grain, const double *g_cw, const double *g_eps,
                    const double *g_mat, const int *row_ptr, const int *col, const unsigned char *broken,
                    double *out)
{
    double Rc = prm[P_RC];
    int micro = (int)prm[P_MICRO];
    double KE = 0, Eb = 0, Ec = 0, Px = 0, Py = 0, Lz = 0, nbk = 0;
    or_sys S;
    memset(&S, 0, sizeof(S));
    S.prm = prm;
    S.g_mat = g_mat;
    for (int x = 0; x < N; ++x) {
        double m = rho_of(&S, grain[x]) * V[x];
        double vx = v[2 * x], vy = v[2 * x + 1];
        double px = X[2 * x] + u[2 * x], py = X[2 * x + 1] + u[2 * x + 1];
        KE += 0.5 * m * (vx * vx + vy * vy);
        Px += m * vx;
        Py += m * vy;
        Lz += m * (px * vy - py * vx);
        int g = grain[x];
        for (int b = row_ptr[x]; b < row_ptr[x + 1]; ++b) {
            if (broken[b]) { nbk += 1; continue; }
            int y = col[b];
            double xix = X[2 * y] - X[2 * x], xiy = X[2 * y + 1] - X[2 * x + 1];
            double xi = sqrt(xix * xix + xiy * xiy);
            double dx = (X[2 * y] + u[2 * y]) - px, dy = (X[2 * y + 1] + u[2 * y + 1]) - py;
            double L = sqrt(dx * dx + dy * dy);
            double s = (L - xi) / xi;
            double c = micro ? g_cw[g] * (1.0 - xi / g_eps[g]) : g_cw[g];
            /* pair potential 1/2 c s^2 |xi| per unit volume^2, each bond seen twice */
            Eb += 0.25 * c * s * s * xi * V[x] * V[y];
        }
        for (int y = x + 1; y < N; ++y) {
            if (grain[y] == grain[x]) continue;
            double dx = (X[2 * y] + u[2 * y]) - px, dy = (X[2 * y + 1] + u[2 * y + 1]) - py;
            double d = sqrt(dx * dx + dy * dy);
            if (d < Rc) Ec += 0.5 * kn_pair(&S, grain[x], grain[y]) * V[x] * V[y] * (Rc - d) * (Rc - d);
        }
    }
    out[0] = KE; out[1] = Eb; out[2] = Ec; out[3] = Px; out[4] = Py; out[5] = Lz; out[6] = nbk;
}

/* Single-wall contact potential, Sec. 4.5: the energy whose negative        */
/* derivative along the wall normal is the repulsion of eq. (wall-repulsive),*/
/*   W(d) = int_d^{R_c} K_n V_x |S_l(s)| (R_c - |c_l(s) - p|) ds.            */
/* With s = R cos(t), |S_l| (R - |c_l - p|) = R^3 g(t) (segment_shape), so    */
/* W = K_n V_x R^4 J(theta) with J(theta) = int_0^theta g(t) sin(t) dt        */
/*   = sin th - th cos th - sin^3 th / 3 - th / 4 + sin(2 th)/6 - sin(4 th)/48 */
/* (int t sin t, int sin^2 t cos t and int sin^4 t written out).  J starts at */
/* th^7 / 35, so below th = 1 the terms of that closed form cancel; there the */
/* sum of its Taylor series is used: expanding every term in odd powers,      */
/*   J = sum_{m>=3} (-1)^m c_m th^(2m+1) / (2m+1)!,                           */
/*   c_m = 1 - (2m+1) - (3 - 3^(2m+1)) / 12 + 2^(2m+1) / 6 - 4^(2m+1) / 48    */
/* (the m = 0, 1, 2 coefficients vanish).  Returns R^4 J; the energy is that */
/* times K_n V_x.  A node past the wall (d < 0) is taken at d = 0, as its     */
/* force is.                                                                  */
double or_wall_segment_energy(double d, double Rc)
{
    if (!(d < Rc)) return 0.0;
    if (d < 0.0) d = 0.0;
    double th = atan2(sqrt((Rc - d) * (Rc + d)), d);
    double J;
    if (th < 1.0) {
        double t2 = th * th;
        double pw = th * t2 * t2 * t2;                    /* th^7      */
        double fact = 5040.0;                             /* 7!        */
        double p2 = 128.0, p3 = 2187.0, p4 = 16384.0;     /* 2^7, 3^7, 4^7 */
        double sign = -1.0;
        J = 0.0;
        for (int m = 3; m <= 22; ++m) {
            double c = 1.0 - (2.0 * m + 1.0) - (3.0 - p3) / 12.0 + p2 / 6.0 - p4 / 48.0;
            J += sign * c * pw / fact;
            pw *= t2;
            fact *= (2.0 * m + 2.0) * (2.0 * m + 3.0);
            p2 *= 4.0;
            p3 *= 9.0;
            p4 *= 16.0;
            sign = -sign;
        }
    } else {
        double sn = sin(th), cs = cos(th);
        J = sn - th * cs - sn * sn * sn / 3.0 - th / 4.0 + sin(2.0 * th) / 6.0 - sin(4.0 * th) / 48.0;
    }
    double R2 = Rc * Rc;
    return R2 * R2 * J;
}

/* Potential energies of the contact laws at the current state, walls at    */
/* time t.  out[0] E_contact: inter-grain pairs within R_c, the energy       */
/* 1/2 K_n V_x V_y (R_c - d)^2 of eq. (law-repulsive); out[1] E_self: pairs   */
/* of one grain with no intact bond (Sec. 4.4), 1/2 (c_w / R_c) V_x V_y       */
/* (R_c - d)^2 when |xi| >= R_c and 1/2 (c_w / |xi|) V_x V_y (|xi| - d)^2     */
/* while d < |xi| < R_c -- the energies of the two self-contact branches;    */
/* out[2] E_wall: the single-wall potentials K_n V_x W(d_l) of every node and */
/* wall (corner regions excluded: the corner term of eq. (wall-total) is not  */
/* the gradient of a potential).  Pairs come from S^nbr (grid search).       */
void or_energies(const double *prm, double t, int N, const double *X, const double *u, const double *V,
                 const int *grain, const double *g_cw, const double *g_mat, const int *row_ptr, const int *col,
                 const unsigned char *broken, double *out)
{
    or_sys S;
    sys_init(&S, prm, N, X, u, NULL, V, grain, g_cw, NULL, NULL, g_mat, row_ptr, col, NULL, NULL);
    S.t = t;
    S.use_grid = 1;
    double Rc = prm[P_RC];
    double Ec = 0.0, Es = 0.0, Ew = 0.0;
    for (int k = 0; k < 2 * N; ++k) S.p[k] = X[k] + u[k];
    int grid = Rc > 0.0 && N > 0;
    if (grid) build_grid(&S);
    for (int x = 0; x < N; ++x) {
        double px = S.p[2 * x], py = S.p[2 * x + 1];
        int g = grain[x];
        int nc = grid ? contact_candidates(&S, x, S.cand) : 0;
        for (int k = 0; k < nc; ++k) {
            int y = S.cand[k];
            if (y < x) continue;
            double dx = S.p[2 * y] - px, dy = S.p[2 * y + 1] - py;
            double d = sqrt(dx * dx + dy * dy);
            if (grain[y] != g) {
                Ec += 0.5 * kn_pair(&S, g, grain[y]) * V[x] * V[y] * (Rc - d) * (Rc - d);
                continue;
            }
            int bonded = 0;
            for (int b = row_ptr[x]; b < row_ptr[x + 1]; ++b)
                if (col[b] == y && !broken[b]) bonded = 1;
            if (bonded) continue;
            double xix = X[2 * y] - X[2 * x], xiy = X[2 * y + 1] - X[2 * x + 1];
            double xi = sqrt(xix * xix + xiy * xiy);
            if (xi < Rc) {
                if (d < xi) Es += 0.5 * (g_cw[g] / xi) * V[x] * V[y] * (xi - d) * (xi - d);
            } else {
                Es += 0.5 * (g_cw[g] / Rc) * V[x] * V[y] * (Rc - d) * (Rc - d);
            }
        }
        /* walls at time t: x_lo, x_hi, y_lo, y_hi */
        double w[4];
        for (int l = 0; l < 4; ++l) w[l] = prm[P_WX0 + l] + prm[P_VX0 + l] * t;
        double dl[4] = {px - w[0], w[1] - px, py - w[2], w[3] - py};
        double Kn = kn_pair(&S, g, g);
        for (int l = 0; l < 4; ++l) Ew += Kn * V[x] * or_wall_segment_energy(dl[l], Rc);
    }
    if (grid) free_grid(&S);
    sys_free(&S);
    out[0] = Ec;
    out[1] = Es;
    out[2] = Ew;
}
