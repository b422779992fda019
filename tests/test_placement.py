"""Shape-agnostic jammed placement of Sec. 6.1 (host set-up): inscribed
circles, nodal circles, the R_c / 2 shrink and the grains placed in the disks."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import placement as PL


def _seg_dist(p, a, b):
    t = np.clip(np.dot(p - a, b - a) / np.dot(b - a, b - a), 0.0, 1.0)
    return float(np.linalg.norm(p - (a + t * (b - a))))


def test_incircle_touches_the_three_sides():
    """Step 2: the centre (v1 l1 + v2 l2 + v3 l3) / (l1 + l2 + l3) is at the
    distance r = 2 |T| / (l1 + l2 + l3) from each side, inside the triangle."""
    rng = np.random.Generator(np.random.PCG64(3))
    nodes = rng.uniform(-1, 1, (30, 2))
    tris = np.array([rng.choice(30, 3, replace=False) for _ in range(40)])
    c, r = PL.incircles(nodes, tris)
    for t in range(len(tris)):
        a, b, e = nodes[tris[t]]
        for p, q in ((a, b), (b, e), (e, a)):
            assert _seg_dist(c[t], p, q) == pytest.approx(r[t], rel=1e-10, abs=1e-14)


def _disks(box=(8e-3, 8e-3), spacing=2.5e-3, seed=2):
    nodes, tris, _ = PL.structured_mesh((0.0, 0.0), box, spacing, 0.2, seed)
    cT, rT = PL.incircles(nodes, tris)
    cN, rN = PL.nodal_circles(nodes, tris, cT, rT, (0.0, 0.0), box)
    return nodes, tris, cT, rT, cN, rN


def test_jammed_disks_are_disjoint_and_inside_the_box():
    box = (8e-3, 8e-3)
    nodes, tris, cT, rT, cN, rN = _disks(box)
    c = np.vstack([cT, cN])
    r = np.concatenate([rT, rN])
    gap = np.linalg.norm(c[:, None] - c[None], axis=2) - r[:, None] - r[None]
    np.fill_diagonal(gap, 1.0)
    assert gap.min() >= -1e-12 * box[0]
    assert np.all(c[:, 0] - r >= -1e-12) and np.all(c[:, 0] + r <= box[0] + 1e-12)
    assert np.all(c[:, 1] - r >= -1e-12) and np.all(c[:, 1] + r <= box[1] + 1e-12)
    # the nodal circles add to the inscribed circles' packing (Fig. myfig: 0.69 -> 0.80)
    area = box[0] * box[1]
    p_in = np.sum(math.pi * rT ** 2) / area
    p_all = np.sum(math.pi * r ** 2) / area
    assert p_all > p_in + 0.05 and 0.6 < p_all < 0.9


def test_nodal_circles_are_locally_maximal():
    """Step 4: moving a nodal circle's centre in any direction does not let it
    grow by more than a sliver of the move (the maximum of a minimum of
    distances lies on a ridge, which a pattern search climbs to within its
    final step)."""
    box = (8e-3, 8e-3)
    nodes, tris, cT, rT, cN, rN = _disks(box)
    star = [[] for _ in range(len(nodes))]
    nbr = [set() for _ in range(len(nodes))]
    for t, (a, b, e) in enumerate(tris):
        for p, q, s in ((a, b, e), (b, e, a), (e, a, b)):
            star[p].append(t)
            nbr[p].update((q, s))
    for v in range(len(nodes)):
        ts = np.array(star[v])
        ws = [nodes[w] for w in sorted(nbr[v])]
        f = lambda c: PL._clearance(c, cT[ts], rT[ts], (0.0, 0.0), box, nodes[v], ws)
        assert f(cN[v]) == pytest.approx(rN[v], abs=1e-15)
        d = 1e-3 * rN[v]
        for ang in np.linspace(0, 2 * math.pi, 16, endpoint=False):
            assert f(cN[v] + d * np.array([math.cos(ang), math.sin(ang)])) <= rN[v] + 1e-3 * d


def test_grains_start_without_contact():
    """Steps 5-6: grains fill their shrunk disks (radius = disk radius) and start
    at least R_c apart and R_c from the walls: no contact or wall force at t = 0."""
    w = PL.jammed_settling(box=(8e-3, 8e-3), spacing=2.5e-3, h_ratio=8, gy=0.0)
    assert w.n_grains > 5
    r = w.grain_geom[:, 2]
    c = w.grain_geom[:, :2]
    gap = np.linalg.norm(c[:, None] - c[None], axis=2) - r[:, None] - r[None]
    np.fill_diagonal(gap, 1.0)
    P = O.OracleProblem.from_workload(w)
    assert gap.min() >= P.prm[O.P_RC] * (1 - 1e-9)
    # every node of a grain lies inside its disk
    for g in range(w.n_grains):
        x = P.X[P.grain == g]
        assert np.linalg.norm(x - c[g], axis=1).max() <= r[g]
    F, parts = P.forces()
    assert np.abs(parts[1]).max() == 0 and np.abs(parts[2]).max() == 0 and np.abs(parts[3]).max() == 0
