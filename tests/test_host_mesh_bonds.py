"""Host part of the boundary: the library's lattice mesher and its bond builder
(the paper's extended-boundary + cusp-bisector construction, Sec. 4) against
the oracle (exact segment-in-domain definition).  Bit-exact: node positions,
lattice indices, grain ids and every CSR row."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I


def _one(shape_loops, ratio, theta=0.37):
    R = 1e-3
    return I.Workload(shapes=[shape_loops], grain_shape=np.array([0], np.int32),
                      grain_geom=np.array([[2e-3, 3e-3, R, theta, 0, 0, R / ratio]]),
                      params=I.default_params(), n_steps=1, name="one")


CASES = {
    "two_disks": lambda: I.two_disks(),
    "settling_seed1": lambda: I.settling(),
    "settling_seed2": lambda: I.settling(seed=2),
    "settling_h12": lambda: I.settling(seed=4, h_ratio=12),
    "perturbed": lambda: I.perturbed_disks(24, h_ratio=15),
    "plus8": lambda: _one(I.plus_shape(), 8),
    "plus15": lambda: _one(I.plus_shape(), 15),
    "plus_thin": lambda: _one(I.plus_shape(0.12), 20),
    "annulus12": lambda: _one(I.annulus_shape(), 12),
    "annulus_thin": lambda: _one(I.annulus_shape(0.8), 20),
    "square": lambda: _one(I.square_shape(), 10),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_mesh_and_bonds_match_oracle(case):
    w = CASES[case]()
    S = B.Simulation(w)
    P = O.OracleProblem.from_workload(w)
    assert S.N == P.N
    assert np.array_equal(S.get("X"), P.X)
    assert np.array_equal(S.get("LATTICE"), P.lat)
    assert np.array_equal(S.get("GRAIN"), P.grain)
    assert np.array_equal(S.get("VOLUME"), P.V)
    assert np.array_equal(S.get("ROW_PTR"), P.row_ptr)
    assert np.array_equal(S.get("COL"), P.col)
    info = S.info()
    assert info["Rc"] == P.prm[O.P_RC]
    assert info["Kn"] == P.prm[O.P_KN]


def test_non_convex_grains_lose_bonds():
    """The construction really removes bonds across re-entrant corners / holes."""
    full = B.Simulation(_one(I.disk_shape(), 12))
    plus = B.Simulation(_one(I.plus_shape(), 8))
    rp = plus.get("ROW_PTR")
    lat = plus.get("LATTICE")
    # lattice neighbours within the horizon present as nodes but not bonded
    index = {tuple(l): k for k, l in enumerate(lat)}
    col = plus.get("COL")
    missing = 0
    for i, (a, b) in enumerate(lat):
        have = set(col[rp[i]:rp[i + 1]])
        for dj in range(-3, 4):
            for di in range(-3, 4):
                if (di, dj) != (0, 0) and di * di + dj * dj < 9:
                    j = index.get((a + di, b + dj))
                    if j is not None and j not in have:
                        missing += 1
    assert missing > 0
    assert full.n_bonds > 0


def test_notched_square_has_no_bond_across_the_notch():
    """No bond of the notched square crosses the notch (the segment of every
    bond of A stays on one side of the slit where both ends lie left of the tip)."""
    w = I.three_particles()
    S = B.Simulation(w)
    X, row, col, grain = S.get("X"), S.get("ROW_PTR"), S.get("COL"), S.get("GRAIN")
    h = 0.5e-3 / 10
    y_notch = 0.5 * h
    crossing = 0
    for x in np.nonzero(grain == 0)[0]:
        for y in col[row[x]:row[x + 1]]:
            a, b = X[x], X[y]
            if (a[1] - y_notch) * (b[1] - y_notch) < 0:
                t = (y_notch - a[1]) / (b[1] - a[1])
                crossing += a[0] + t * (b[0] - a[0]) < 0.0          # crosses the slit, left of the tip
    assert crossing == 0
    assert S.n_bonds > 0
