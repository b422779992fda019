"""The modal basis of the learned surrogate built by the library
(pd_surrogate_basis, host only): against an independent assembly of the
linearised bond operator of eq:pmb (written out here from Table 1's c_w) and
LAPACK's symmetric eigensolver.  Eigenvalues must agree to 1e-9 of the largest
wanted one; the eigenvectors must span the same invariant subspaces (repeated
eigenvalues make single vectors arbitrary), so the check is on the projector."""
import math

import numpy as np
import pytest

from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I
from paper_2108_07212_gb300 import surrogate as SU

scipy_linalg = pytest.importorskip("scipy.linalg")


def _operator(lat, row_ptr, col, params):
    """K/E of one template: a bond of lattice offset d (|d| in units of h) with
    micromodulus c_w w adds c_w w V^2 / (E h |d|) e e^T; with c_w = 6 E / (pi eps^3
    (1 - nu)) (constant) or 24 E / (...) (conic, w = 1 - |d| h / eps), V = h^2 and
    eps = r h that is (6 or 24) / (pi r^3 (1 - nu)) w / |d| e e^T."""
    n = lat.shape[0]
    r = params["horizon_ratio"]
    conic = int(params["micromodulus"]) == 1
    c = (24.0 if conic else 6.0) / (math.pi * r ** 3 * (1.0 - params["nu"]))
    K = np.zeros((2 * n, 2 * n))
    for a in range(n):
        for b in col[row_ptr[a]:row_ptr[a + 1]]:
            d = (lat[b] - lat[a]).astype(np.float64)
            L = math.hypot(d[0], d[1])
            e = d / L
            k = c * ((1.0 - L / r) if conic else 1.0) / L * np.outer(e, e)
            K[2 * a:2 * a + 2, 2 * a:2 * a + 2] += k
            K[2 * a:2 * a + 2, 2 * b:2 * b + 2] -= k
    return K


@pytest.mark.parametrize("shape,h_ratio,micro", [("hexagon", 6, 0), ("disk", 10, 0), ("plus", 10, 1),
                                                 ("annulus", 12, 0)])
def test_library_basis_matches_lapack_on_the_assembled_operator(shape, h_ratio, micro):
    w = I.free_grains(shapes=(shape,), n_per_shape=2, h_ratio=h_ratio)
    w.params["micromodulus"] = micro
    S = B.Simulation(w)                          # host only: mesh and bonds
    cfg = SU.build_basis(S, n_modes=16)
    lat, row, col = S.get("LATTICE"), S.get("ROW_PTR"), S.get("COL")
    grain = S.get("GRAIN")
    n = int(np.sum(grain == 0))
    K = _operator(lat[:n], row[:n + 1], col[:row[n]], w.params)
    vals, vecs = scipy_linalg.eigh(K)
    M = 16
    lam = cfg["lambda_"][:M].astype(np.float64)
    scale = vals[3 + M - 1]
    assert np.abs(lam - vals[3:3 + M]).max() <= 1e-6 * scale      # FP32 output: 2^-24 relative
    assert np.all(np.abs(np.array(cfg["templates"][0]["rigid"])) <= 1e-9 * scale)
    Phi = cfg["basis"][:2 * n * M].astype(np.float64).reshape(n, 2, M).reshape(2 * n, M)
    assert np.abs(Phi.T @ Phi - np.eye(M)).max() <= 1e-5
    # same invariant subspace: group the eigenvalues into clusters, compare projectors
    lo = 3
    while lo < 3 + M:
        hi = lo + 1
        while hi < len(vals) and vals[hi] - vals[hi - 1] <= 1e-7 * scale:
            hi += 1
        if hi <= 3 + M:
            P_ref = vecs[:, lo:hi] @ vecs[:, lo:hi].T
            P_lib = Phi[:, lo - 3:hi - 3] @ Phi[:, lo - 3:hi - 3].T
            assert np.abs(P_ref - P_lib).max() <= 1e-5, (lo, hi)
        lo = hi


def test_library_basis_of_the_largest_settling_template_is_fast_and_converged():
    """The 2000-grain surrogate settling's largest template (about 1650 nodes,
    3300 unknowns): the sparse iteration converges to the dense eigenvalues."""
    import time
    w = I.surrogate_settling(n_grains=40, seed=5)
    S = B.Simulation(w)
    t0 = time.perf_counter()
    cfg = SU.build_basis(S)
    dt = time.perf_counter() - t0
    big = int(np.argmax([d["nodes"] for d in cfg["templates"]]))
    n = cfg["templates"][big]["nodes"]
    tmpl = cfg["template_of_grain"]
    g = int(np.argmax(tmpl == big))
    grain = S.get("GRAIN")
    s0 = int(np.argmax(grain == g))
    lat, row, col = S.get("LATTICE"), S.get("ROW_PTR"), S.get("COL")
    K = _operator(lat[s0:s0 + n], row[s0:s0 + n + 1] - row[s0], col[row[s0]:row[s0 + n]] - s0, w.params)
    vals = scipy_linalg.eigh(K, eigvals_only=True, subset_by_index=[0, 34])
    lam = cfg["lambda_"].reshape(-1, 32)[big].astype(np.float64)
    assert n > 1000
    assert np.abs(lam - vals[3:]).max() <= 1e-6 * vals[-1]
    assert dt < 120.0, dt
