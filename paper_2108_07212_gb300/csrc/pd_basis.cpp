// pd_basis.cpp -- modal basis of the learned surrogate (host).
//
// Per bond-network template (grains of one shape meshed at the same h/R share
// one lattice and one bond network) the basis is made of the softest non-rigid
// eigenvectors of the template's linearised bond operator.  Linearising the
// bond force of eq:pmb about the reference lattice, a bond of lattice offset d
// (length |d| h, unit e) with micromodulus c_w w contributes the stiffness
// c_w w V_x V_y / |xi| e e^T between its two nodes; in units of E h, with
// displacements in units of h, that is k = c_w w V^2 / (E h |d|) e e^T
// (V = h^2), so F / (E h) = -(K / E) u / h with
//   (K / E)[a, a] += k,  (K / E)[a, b] -= k      for every directed bond a -> b.
// c_w and w are the library's own (Table 1, per grain), so the basis and the
// force kernels share one source for the bond constants.
//
// The 2 n x 2 n operator is sparse (25 2 x 2 blocks per interior node) and
// positive semi-definite with three zero modes (two translations, one
// rotation).  Its lowest eigenpairs are found by Chebyshev-filtered subspace
// iteration (Zhou & Saad, J. Comput. Phys. 219, 2006): a block of p vectors is
// multiplied by a Chebyshev polynomial of K that is small on [theta_p, lambda_max]
// (theta_p the block's largest Ritz value, lambda_max a Gershgorin bound) and
// large below it, orthonormalised, and rotated to the Ritz vectors of K in its
// span (Rayleigh-Ritz, dense Jacobi eigen-decomposition) until the wanted
// residuals are small.  Templates of at most kDenseDofs unknowns are solved
// densely by the cyclic Jacobi method.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "peridem.h"

namespace pd {
int set_error(int code, const char *msg);
}

namespace {

constexpr int kDenseDofs = 400;      // dense Jacobi up to this many unknowns
constexpr int kChebDegree = 24;      // degree of the filter polynomial
constexpr int kMaxIter = 400;        // filter applications at most
constexpr double kResTol = 1e-10;    // residual norms below this times lambda_max

struct Csr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

// Y = K X for p vectors stored row-major (x[i p + k]).
void spmm(const Csr &K, const double *x, double *y, int p) {
    for (int i = 0; i < K.n; ++i) {
        double *yi = y + (size_t)i * p;
        std::fill(yi, yi + p, 0.0);
        for (int q = K.rp[i]; q < K.rp[i + 1]; ++q) {
            const double a = K.v[q];
            const double *xj = x + (size_t)K.ci[q] * p;
            for (int k = 0; k < p; ++k) yi[k] += a * xj[k];
        }
    }
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row-major,
// destroyed): eigenvalues w ascending, eigenvectors as the columns of V.
void jacobi_eigen(std::vector<double> &A, int n, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) (i == j ? diag : off) += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                // rotation angle that zeroes A[p][q]: tan(2 phi) = 2 a_pq / (a_qq - a_pp)
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    w.resize(n);
    std::vector<double> Vs((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        w[k] = A[(size_t)order[k] * n + order[k]];
        for (int i = 0; i < n; ++i) Vs[(size_t)i * n + k] = V[(size_t)i * n + order[k]];
    }
    V.swap(Vs);
}

// Orthonormalise the p columns of X (N x p, row-major) by modified Gram-Schmidt,
// twice (columns that vanish are replaced by the next unit vector).
void orthonormalise(std::vector<double> &X, int N, int p) {
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < p; ++k) {
            for (int j = 0; j < k; ++j) {
                double d = 0.0;
                for (int i = 0; i < N; ++i) d += X[(size_t)i * p + j] * X[(size_t)i * p + k];
                for (int i = 0; i < N; ++i) X[(size_t)i * p + k] -= d * X[(size_t)i * p + j];
            }
            double nrm = 0.0;
            for (int i = 0; i < N; ++i) nrm += X[(size_t)i * p + k] * X[(size_t)i * p + k];
            nrm = std::sqrt(nrm);
            if (nrm < 1e-300) {
                for (int i = 0; i < N; ++i) X[(size_t)i * p + k] = (i == k % N) ? 1.0 : 0.0;
                --k;            // orthogonalise the replacement again
                continue;
            }
            for (int i = 0; i < N; ++i) X[(size_t)i * p + k] /= nrm;
        }
}

// Lowest k eigenpairs of K (ascending): values w[k], vectors as columns of
// Z (N x k, row-major).  Returns false when the iteration did not converge.
bool lowest_eigenpairs(const Csr &K, int k, std::vector<double> &w, std::vector<double> &Z) {
    const int N = K.n;
    if (N <= kDenseDofs) {
        std::vector<double> A((size_t)N * N, 0.0), V, ww;
        for (int i = 0; i < N; ++i)
            for (int q = K.rp[i]; q < K.rp[i + 1]; ++q) A[(size_t)i * N + K.ci[q]] += K.v[q];
        jacobi_eigen(A, N, ww, V);
        w.assign(ww.begin(), ww.begin() + k);
        Z.assign((size_t)N * k, 0.0);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < k; ++j) Z[(size_t)i * k + j] = V[(size_t)i * N + j];
        return true;
    }
    const int p = std::min(N, k + std::max(8, k / 3));
    // Gershgorin bound of the largest eigenvalue
    double lmax = 0.0;
    for (int i = 0; i < N; ++i) {
        double r = 0.0;
        for (int q = K.rp[i]; q < K.rp[i + 1]; ++q) r += std::fabs(K.v[q]);
        lmax = std::max(lmax, r);
    }
    // seeded start block (a 64-bit linear congruential generator, Knuth's MMIX constants)
    std::vector<double> X((size_t)N * p), Y((size_t)N * p), KY((size_t)N * p), T0((size_t)N * p);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (auto &x : X) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    orthonormalise(X, N, p);
    std::vector<double> H((size_t)p * p), V, theta;
    double cut = lmax * 1e-2;          // first damping threshold, then the block's top Ritz value
    for (int it = 0; it < kMaxIter; ++it) {
        // Chebyshev filter on [cut, lmax]: Y_{j+1} = 2 (K - c) Y_j / e - Y_{j-1}
        const double e = 0.5 * (lmax - cut), c = 0.5 * (lmax + cut);
        spmm(K, X.data(), KY.data(), p);
        for (size_t q = 0; q < Y.size(); ++q) Y[q] = (KY[q] - c * X[q]) / e;
        T0 = X;
        for (int j = 1; j < kChebDegree; ++j) {
            spmm(K, Y.data(), KY.data(), p);
            for (size_t q = 0; q < Y.size(); ++q) {
                const double nxt = 2.0 * (KY[q] - c * Y[q]) / e - T0[q];
                T0[q] = Y[q];
                Y[q] = nxt;
            }
        }
        orthonormalise(Y, N, p);
        // Rayleigh-Ritz: H = Y^T K Y, X = Y V
        spmm(K, Y.data(), KY.data(), p);
        std::fill(H.begin(), H.end(), 0.0);
        for (int i = 0; i < N; ++i) {
            const double *yi = &Y[(size_t)i * p], *ki = &KY[(size_t)i * p];
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) H[(size_t)a * p + b] += yi[a] * ki[b];
        }
        for (int a = 0; a < p; ++a)
            for (int b = a + 1; b < p; ++b) H[(size_t)a * p + b] = H[(size_t)b * p + a] =
                                                0.5 * (H[(size_t)a * p + b] + H[(size_t)b * p + a]);
        jacobi_eigen(H, p, theta, V);
        std::fill(X.begin(), X.end(), 0.0);
        std::fill(T0.begin(), T0.end(), 0.0);   // K X = (K Y) V
        for (int i = 0; i < N; ++i)
            for (int b = 0; b < p; ++b) {
                const double yb = Y[(size_t)i * p + b], kb = KY[(size_t)i * p + b];
                for (int a = 0; a < p; ++a) {
                    X[(size_t)i * p + a] += yb * V[(size_t)b * p + a];
                    T0[(size_t)i * p + a] += kb * V[(size_t)b * p + a];
                }
            }
        // residuals of the wanted pairs
        double worst = 0.0;
        for (int a = 0; a < k; ++a) {
            double r2 = 0.0;
            for (int i = 0; i < N; ++i) {
                const double r = T0[(size_t)i * p + a] - theta[a] * X[(size_t)i * p + a];
                r2 += r * r;
            }
            worst = std::max(worst, std::sqrt(r2));
        }
        cut = std::max(theta[p - 1], 1e-6 * lmax);
        if (worst <= kResTol * lmax) {
            w.assign(theta.begin(), theta.begin() + k);
            Z.assign((size_t)N * k, 0.0);
            for (int i = 0; i < N; ++i)
                for (int a = 0; a < k; ++a) Z[(size_t)i * k + a] = X[(size_t)i * p + a];
            return true;
        }
    }
    return false;
}

}  // namespace

// Host-side template data of a bonded context (defined in pd_host.cpp).
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
int template_view(pd_ctx *c, TemplateView *out);
}  // namespace pd

extern "C" int pd_surrogate_basis(pd_ctx *ctx, int n_modes, float *basis, size_t *basis_len, float *lambda,
                                  double *rigid) {
    pd::TemplateView tv{};
    if (int r = pd::template_view(ctx, &tv)) return r;
    if (n_modes < 1 || !basis_len) return pd::set_error(PD_EINVAL, "pd_surrogate_basis: n_modes >= 1, basis_len required");
    size_t need = 0;
    for (int t = 0; t < tv.n_tmpl; ++t) need += (size_t)2 * tv.tmpl_nodes[t] * n_modes;
    if (!basis) {
        *basis_len = need;
        return PD_OK;
    }
    if (*basis_len != need || !lambda)
        return pd::set_error(PD_EINVAL, "pd_surrogate_basis: basis_len must equal sum over templates of 2 n_t n_modes"
                                        " (call with basis = NULL to query it) and lambda must be non-null");
    size_t out = 0;
    for (int t = 0; t < tv.n_tmpl; ++t) {
        const int g = tv.tmpl_first[t];
        const int64_t a0 = tv.g_start[g];
        const int n = tv.tmpl_nodes[t], N = 2 * n, k = n_modes + 3;
        if (N < k) return pd::set_error(PD_EINVAL, "pd_surrogate_basis: a template has fewer unknowns than n_modes + 3");
        // c_w V^2 / (E h) = c_w h^3 / E of the template's grain (V = h^2)
        const double h = tv.g_h[g];
        const double cdim = tv.g_cw[g] * h * h * h / tv.E;
        const double r = tv.g_eps[g] / h;        // horizon / h
        // assemble K / E as 2 x 2 blocks: diagonal blocks summed, one off-diagonal block per bond
        Csr K;
        K.n = N;
        K.rp.assign(N + 1, 0);
        std::vector<double> diag((size_t)4 * n, 0.0);
        for (int a = 0; a < n; ++a) {
            const int deg = tv.row_ptr[a0 + a + 1] - tv.row_ptr[a0 + a];
            K.rp[2 * a + 1] = 2 * (deg + 1);
            K.rp[2 * a + 2] = 2 * (deg + 1);
        }
        for (int i = 0; i < N; ++i) K.rp[i + 1] += K.rp[i];
        K.ci.resize(K.rp[N]);
        K.v.resize(K.rp[N]);
        for (int a = 0; a < n; ++a) {
            const int b0 = tv.row_ptr[a0 + a], b1 = tv.row_ptr[a0 + a + 1];
            int pos[2] = {K.rp[2 * a], K.rp[2 * a + 1]};
            double dsum[4] = {0.0, 0.0, 0.0, 0.0};
            // off-diagonal blocks after the diagonal one
            for (int comp = 0; comp < 2; ++comp) pos[comp] += 2;
            for (int q = b0; q < b1; ++q) {
                const int b = (int)(tv.col[q] - a0);
                const double dx = (double)(tv.lat[2 * (a0 + b)] - tv.lat[2 * (a0 + a)]);
                const double dy = (double)(tv.lat[2 * (a0 + b) + 1] - tv.lat[2 * (a0 + a) + 1]);
                const double L = std::sqrt(dx * dx + dy * dy);
                const double wgt = tv.micromodulus == PD_MICRO_CONIC ? 1.0 - L / r : 1.0;
                const double kk = cdim * wgt / L;
                const double ex = dx / L, ey = dy / L;
                const double blk[4] = {kk * ex * ex, kk * ex * ey, kk * ey * ex, kk * ey * ey};
                for (int m = 0; m < 4; ++m) dsum[m] += blk[m];
                for (int comp = 0; comp < 2; ++comp) {
                    K.ci[pos[comp]] = 2 * b;
                    K.v[pos[comp]] = -blk[2 * comp];
                    K.ci[pos[comp] + 1] = 2 * b + 1;
                    K.v[pos[comp] + 1] = -blk[2 * comp + 1];
                    pos[comp] += 2;
                }
            }
            for (int comp = 0; comp < 2; ++comp) {
                const int p0 = K.rp[2 * a + comp];
                K.ci[p0] = 2 * a;
                K.v[p0] = dsum[2 * comp];
                K.ci[p0 + 1] = 2 * a + 1;
                K.v[p0 + 1] = dsum[2 * comp + 1];
            }
        }
        std::vector<double> w, Z;
        if (!lowest_eigenpairs(K, k, w, Z))
            return pd::set_error(PD_ENUMERIC, "pd_surrogate_basis: the eigen-iteration did not converge");
        // modes 3 .. 3 + n_modes - 1 (the first three are the rigid motions)
        for (int l = 0; l < n; ++l)
            for (int comp = 0; comp < 2; ++comp)
                for (int m = 0; m < n_modes; ++m) basis[out++] = (float)Z[(size_t)(2 * l + comp) * k + 3 + m];
        for (int m = 0; m < n_modes; ++m) lambda[(size_t)t * n_modes + m] = (float)w[3 + m];
        if (rigid)
            for (int m = 0; m < 3; ++m) rigid[3 * t + m] = w[m];
    }
    return PD_OK;
}
