"""Parity against the FP64 oracle at the full sizes of the benchmark workloads.

At these sizes the kernels take paths the small parity cases never reach: the
split force phase of the kernel graph (lane sums through device memory, then the
per-node epilogue), hash grids of 2^20 to 2^24 buckets with the two-level
scan, the aliased buckets of 64 aggregates sharing one grid, and the learned
surrogate on 2000 grains.  The oracle (all-core build) advances each workload
from its initial state to a loaded one (collisions, wall contact, fracture);
the GPU trajectory from the same initial state is compared with it, and the
oracle's state is pushed into the GPU contexts for one force evaluation
compared element by element (Algorithm 1; eq:full): plain FP64 path within
1e-12 of the largest force, FP32-split path within 1e-5, with identical
broken-bond sets.  Each force part (bond, self-contact, contact, wall) is also
compared at the scale of its own largest value.  No oracle input comes from
the GPU: the GPU runs only choose which aggregates of the ensemble the oracle
advances.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _state(S):
    return {f: S.get(f) for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP")}


def _push_gpu(S, st):
    for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP"):
        S.set(f, st[f])


def _oracle_state(P):
    """The oracle's state, in the layout of the GPU state fields."""
    return {"DISP": P.u.copy(), "VEL": P.v.copy(), "ACC": P.a.copy(),
            "BROKEN": P.broken[: len(P.col)].copy(), "STEP": np.array([P.step], np.int64)}


def _l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _eval(S):
    S.eval_forces()
    return S.get("FORCE"), S.get("FORCE_PARTS"), S.get("BROKEN")


def _compare(F, parts, broken, F_or, parts_or, broken_or, tol, label, floor=0.0):
    """Element-wise: every component within tol of the largest oracle force of
    the evaluation (of its part, for each part), that scale floored at `floor`."""
    def err(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), floor, 1e-300))
    assert err(F, F_or) <= tol, (label, "total", err(F, F_or))
    for k, name in enumerate(("bond", "self", "contact", "wall")):
        if np.abs(parts_or[k]).max() > 0:
            assert err(parts[k], parts_or[k]) <= tol, (label, name, err(parts[k], parts_or[k]))
        else:
            assert np.abs(parts[k]).max() <= tol * floor, (label, name)
    assert np.array_equal(broken, broken_or), (label, int(np.sum(broken != broken_or)))


def test_compaction_521k_nodes_one_force_evaluation_against_oracle():
    """The 500-grain compaction (521,454 nodes, 11.4M directed bonds) with every
    grain thrown at 5 m/s: after 500 steps grains collide and break bonds.  The
    GPU's FP64 trajectory follows the oracle's (1e-9 relative L2, identical
    breaks); at the oracle's state both GPU paths match its forces."""
    w = I.compaction(agitation=5.0)
    P = O.OracleProblem.from_workload(w)
    P.omp = True
    P.init_accel()
    P.run(500)
    st = _oracle_state(P)
    F_or, parts_or = P.forces(keep_broken=False)
    assert st["BROKEN"].sum() > 0 and np.abs(parts_or[2]).max() > 0
    A = B.Simulation(w, precision=B.PD_FP64, store_parts=True, device="cuda:0")
    info = A.info()
    assert A.N > 500_000 and info["buckets"] >= 2 ** 20 and int(info["mode"]) == 2
    A.step(500)
    assert _l2(A.get("DISP"), st["DISP"]) <= 1e-9
    assert np.array_equal(A.get("BROKEN"), st["BROKEN"])
    _push_gpu(A, st)
    F64, parts64, br64 = _eval(A)
    _compare(F64, parts64, br64, F_or, parts_or, P.broken[: len(P.col)], FP64_TOL, "fp64")
    del A
    C = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0")
    _push_gpu(C, st)
    F32, parts32, br32 = _eval(C)
    _compare(F32, parts32, br32, F_or, parts_or, P.broken[: len(P.col)], FP32_TOL, "fp32")


def test_ensemble_of_64_aggregates_against_oracle_per_aggregate():
    """The batched ensemble (64 aggregates, 6.69M nodes, one shared hash grid
    whose buckets alias across aggregates) with every grain thrown at 5 m/s.
    The batched FP64 context runs 600 steps; on four of its aggregates (the
    largest, the smallest and the two with the largest contact forces) the
    oracle, run on the single aggregate (its own walls, R_c and K_n), gives the
    same trajectory; at the oracle's states the batched FP64 and FP32-split
    contexts match its forces."""
    w = I.ensemble()
    ang = np.random.Generator(np.random.PCG64(4242)).uniform(0.0, 2 * math.pi, w.n_grains)
    w.grain_geom[:, 4] = 5.0 * np.cos(ang)
    w.grain_geom[:, 5] = 5.0 * np.sin(ang)
    # the same initial velocities in the single-aggregate workloads the oracle runs
    g0 = 0
    for part in w.parts:
        part.grain_geom = part.grain_geom.copy()
        part.grain_geom[:, 4:6] = w.grain_geom[g0:g0 + part.n_grains, 4:6]
        g0 += part.n_grains
    assert g0 == w.n_grains
    n_steps = 600
    A = B.Simulation(w, precision=B.PD_FP64, store_parts=True, device="cuda:0")
    assert A.N > 6_000_000 and int(A.info()["n_agg"]) == 64
    A.step(n_steps)
    st = _state(A)
    _, parts_gpu, _ = _eval(A)
    row = A.get("ROW_PTR")
    agg_of_node = w.grain_agg[A.get("GRAIN")]
    # the largest and the smallest aggregate and the two with the largest contact forces
    counts = np.bincount(w.grain_agg)
    cmax = np.zeros(64)
    np.maximum.at(cmax, agg_of_node, np.abs(parts_gpu[2]).max(axis=1))
    pick = {int(np.argmax(counts)), int(np.argmin(counts))} | {int(a) for a in np.argsort(-cmax)[:2]}
    del parts_gpu
    # the oracle on each picked aggregate; its states replace the GPU's there
    ref = {}
    for a in sorted(pick):
        nodes = np.flatnonzero(agg_of_node == a)
        n0, n1 = int(nodes[0]), int(nodes[-1]) + 1
        assert n1 - n0 == nodes.size
        b0, b1 = int(row[n0]), int(row[n1])
        P = O.OracleProblem.from_workload(w.parts[a])
        P.omp = True
        assert P.N == n1 - n0 and len(P.col) == b1 - b0
        P.init_accel()
        P.run(n_steps)
        so = _oracle_state(P)
        assert _l2(st["DISP"][n0:n1], so["DISP"]) <= 1e-9, a
        assert np.array_equal(st["BROKEN"][b0:b1], so["BROKEN"]), a
        for f in ("DISP", "VEL", "ACC"):
            st[f][n0:n1] = so[f]
        st["BROKEN"][b0:b1] = so["BROKEN"]
        F_or, parts_or = P.forces(keep_broken=False)
        ref[a] = (n0, n1, b0, b1, F_or, parts_or, P.broken[: b1 - b0].copy())
    _push_gpu(A, st)
    F64, parts64, br64 = _eval(A)
    del A
    C = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0")
    _push_gpu(C, st)
    F32, parts32, br32 = _eval(C)
    del C
    # a node's weight: the scale below which a force is round-off of the float path
    weight = w.params["rho"] * (w.grain_geom[:, 6].min() ** 2) * abs(w.params["gy"])
    contact_seen = 0
    for a, (n0, n1, b0, b1, F_or, parts_or, br_or) in sorted(ref.items()):
        contact_seen += int(np.abs(parts_or[2]).max() > 0)
        _compare(F64[n0:n1], parts64[:, n0:n1], br64[b0:b1], F_or, parts_or, br_or, FP64_TOL,
                 f"fp64 aggregate {a}")
        _compare(F32[n0:n1], parts32[:, n0:n1], br32[b0:b1], F_or, parts_or, br_or, FP32_TOL,
                 f"fp32 aggregate {a}", floor=weight)
    assert contact_seen >= 2


def test_surrogate_2000_grains_against_oracle_bond_force():
    """The 2000-grain surrogate settling (2.03M nodes, six templates) lowered
    to R_c above the floor, every grain moving down at 2 m/s, with the linear
    modal model (networks with a zero last layer) and the full bond kernel as
    judge every 50 steps.  The lowest grains land on the floor and deform; the
    judge takes off the surrogate every grain whose surrogate bond force is off
    by more than 1e-3 (nodal error over the grain, floored at its weight).  The
    oracle advances the full model over the same 1201 steps; at its state every
    grain still on the surrogate must meet that criterion against the oracle's
    bond force, and at a judge step the full FP32 bond force the judge uses is
    within the FP32-split tolerance of the oracle's, as are the contact and
    wall parts."""
    from paper_2108_07212_gb300 import surrogate as SU

    w = I.surrogate_settling()
    X = B.Simulation(w).get("X")                # meshing only (host)
    rc = w.params["rc_ratio"] * w.grain_geom[:, 6].min()
    w.grain_geom[:, 1] -= X[:, 1].min() - 1.02 * rc   # lowest nodes 1.02 R_c above the floor
    w.grain_geom[:, 5] = -2.0
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0",
                     surrogate=lambda s: SU.build_basis(s))
    cfg = S.surrogate_basis
    counts = np.bincount(cfg["template_of_grain"])
    nets = [B.MLP(max_batch=int(c), params=SU.init_params(t)) for t, c in enumerate(counts)]
    for t, net in enumerate(nets):
        S.surrogate_set_mlp(t, net)
    S.surrogate_enable(True)
    S.step(1201)
    # the oracle's full model over the same 1201 steps; its state goes into the
    # surrogate context (the grains the judge kept on the surrogate stay on it)
    P = O.OracleProblem.from_workload(w)
    P.omp = True
    P.init_accel()
    P.run(1201)
    st = _oracle_state(P)
    F_or, parts_or = P.forces(keep_broken=False)
    _push_gpu(S, st)
    S.surrogate_inspect()                       # force evaluation with the surrogate (not a judge step)
    parts = S.get("FORCE_PARTS")
    active, err, merr, maxs = S.surrogate_stats()
    grain = S.get("GRAIN")
    V = S.get("VOLUME")
    for k in (1, 2, 3):
        if np.abs(parts_or[k]).max() > 0:
            assert _rel(parts[k], parts_or[k]) <= FP32_TOL, k
    assert np.abs(parts_or[3]).max() > 0                  # grains on the floor
    assert 1000 <= active.sum() < w.n_grains              # the judge took the landed grains off
    rho, g = w.params["rho"], max(abs(w.params["gy"]), 100.0)
    bounds = np.r_[0, np.cumsum(np.bincount(grain, minlength=w.n_grains))]
    worst = 0.0
    for gi in np.flatnonzero(active):
        m = slice(bounds[gi], bounds[gi + 1])
        ref = parts_or[0][m]
        floor_ = np.sqrt(np.sum((rho * V[m] * g) ** 2))
        e = np.sqrt(np.sum((parts[0][m] - ref) ** 2)) / max(np.sqrt(np.sum(ref ** 2)), floor_)
        worst = max(worst, e)
    assert worst <= cfg["err_tol"], worst
    # a judge step: the full FP32 bond kernel runs for surrogate grains too
    S.set("STEP", np.array([1250], np.int64))
    S.surrogate_inspect()
    full = S.get("FORCE_PARTS")[0]
    assert np.abs(full - parts_or[0]).max() <= FP32_TOL * np.abs(parts_or[0]).max()
