"""Batched ensembles, the persistent cooperative step kernel and the autotuner.

A batched run must advance every aggregate exactly as a run of that aggregate
alone; the persistent kernel must reproduce the graph of separate kernels; the
autotuner must not move the simulation."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _parts():
    a = I.settling(n_grains=6, box=(9e-3, 12e-3), seed=21)
    b = I.settling(n_grains=10, box=(11e-3, 14e-3), seed=22, h_ratio=12)
    c = I.settling(n_grains=3, box=(7e-3, 9e-3), seed=23)
    for w in (a, b, c):                      # lowest grains on the floor quickly
        w.grain_geom[:, 5] = -3.0
    return [a, b, c]


def _sim(w, prec, **kw):
    return B.Simulation(w, precision=prec, device="cuda:0", **kw)


@pytest.mark.parametrize("prec", [B.PD_FP64, B.PD_FP32_SPLIT])
def test_batched_run_equals_separate_runs(prec):
    parts = _parts()
    merged = I.merge_aggregates(parts)
    S = _sim(merged, prec)
    S.step(400)
    u = S.get("DISP")
    br = S.get("BROKEN")
    off, boff = 0, 0
    for w in parts:
        A = _sim(w, prec)
        A.step(400)
        ua = A.get("DISP")
        n = ua.shape[0]
        # the hash grid of the batched context aliases other cells, which moves
        # candidates between lanes: only the order of the contact sums differs
        tol = 1e-10 if prec == B.PD_FP64 else 1e-8
        assert np.linalg.norm(u[off:off + n] - ua) <= tol * np.linalg.norm(ua)
        assert np.array_equal(br[boff:boff + A.n_bonds], A.get("BROKEN"))
        off += n
        boff += A.n_bonds
    assert off == S.N
    rc, st = S.status()
    assert rc == B.PD_OK


def test_batched_aggregate_matches_oracle():
    parts = _parts()
    S = _sim(I.merge_aggregates(parts), B.PD_FP64)
    S.step(300)
    u = S.get("DISP")
    n0 = 0
    for w in parts[:2]:
        P = O.OracleProblem.from_workload(w).init_accel()
        P.run(300)
        n = P.N
        assert np.linalg.norm(u[n0:n0 + n] - P.u) <= 1e-9 * np.linalg.norm(P.u)
        n0 += n


@pytest.mark.parametrize("prec", [B.PD_FP64, B.PD_FP32_SPLIT])
@pytest.mark.parametrize("lanes,block,modes", [(8, 128, (0, 1)), (4, 256, (0, 1)), (1, 128, (0, 1)),
                                               (8, 128, (0, 2)), (4, 128, (2, 3)), (8, 256, (0, 3)),
                                               (4, 128, (0, 4)), (1, 128, (2, 6))])
def test_persistent_kernel_reproduces_kernel_graph(prec, lanes, block, modes):
    """Graph of kernels vs persistent kernel, fused vs split force phase, the
    candidate-list rebuild behind a conditional node vs launched every step."""
    w = I.merge_aggregates(_parts())
    a = _sim(w, prec)
    b = _sim(w, prec)
    a.set_path(modes[0], lanes, 128)
    b.set_path(modes[1], lanes, block)
    assert b.info()["mode"] == modes[1]
    for k in (1, 16, 37):                    # single steps and whole chunks
        a.step(k)
        b.step(k)
    ua, ub = a.get("DISP"), b.get("DISP")
    if prec == B.PD_FP64:
        assert np.array_equal(ua, ub)
        assert np.array_equal(a.get("VEL"), b.get("VEL"))
    else:
        assert np.linalg.norm(ua - ub) <= 1e-9 * np.linalg.norm(ua)
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))
    assert int(b.get("STEP")[0]) == 54
    rc, st = b.status()
    assert rc == B.PD_OK and st[4] == 0
    if prec == B.PD_FP64:                    # same trajectory: same rebuild steps
        assert st[B.STATUS_REBUILDS] == a.status()[1][B.STATUS_REBUILDS]


@pytest.mark.parametrize("field", ["DISP", "VEL", "ACC"])
def test_state_written_between_persistent_launches_replaces_the_prediction(field):
    """The FP32-split persistent kernel forms the next step's displacement and
    positions in its velocity update, and the next launch starts from them.  A
    state written between two launches must replace that prediction: the run
    then equals a kernel-graph run given the same writes (a stale prediction
    would differ by the size of the change)."""
    w = I.merge_aggregates(_parts())
    a = _sim(w, B.PD_FP32_SPLIT)
    b = _sim(w, B.PD_FP32_SPLIT)
    a.set_path(2, 1, 128)
    b.set_path(1, 1, 256)
    for k in (1, 16, 5):                     # single steps and a chunk: odd parity at the write
        a.step(k)
        b.step(k)
    val = a.get(field)
    assert np.linalg.norm(val - b.get(field)) <= 1e-9 * np.linalg.norm(val)
    changed = val + 1e-3 * np.abs(val).max() * np.sin(np.arange(val.size)).reshape(val.shape)
    for sim in (a, b):
        sim.set(field, changed)
    for k in (1, 16, 3):
        a.step(k)
        b.step(k)
    ua, ub = a.get("DISP"), b.get("DISP")
    assert np.linalg.norm(ua - ub) <= 1e-9 * np.linalg.norm(ua)
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))
    assert int(b.get("STEP")[0]) == 42
    rc, st = b.status()
    assert rc == B.PD_OK and st[4] == 0


def test_switching_between_persistent_kernel_and_graph_mid_run():
    """The persistent kernel leaves the next step's displacement predicted
    (FP32 split); a kernel-graph step recomputes it, and a later persistent
    launch must not take a prediction the graph steps made stale.  One context
    switching paths between calls follows one that stays on the graph."""
    w = I.merge_aggregates(_parts())
    a = _sim(w, B.PD_FP32_SPLIT)
    b = _sim(w, B.PD_FP32_SPLIT)
    a.set_path(2, 1, 128)
    for k, path in ((3, (1, 1, 256)), (16, (2, 1, 128)), (5, (1, 1, 128)), (16, (0, 1, 128)),
                    (7, (3, 1, 256)), (1, (2, 1, 128)), (9, (1, 1, 256))):
        b.set_path(*path)
        a.step(k)
        b.step(k)
    ua, ub = a.get("DISP"), b.get("DISP")
    assert np.linalg.norm(ua - ub) <= 1e-9 * np.linalg.norm(ua)
    va, vb = a.get("VEL"), b.get("VEL")
    assert np.linalg.norm(va - vb) <= 1e-9 * np.linalg.norm(va)
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))
    assert int(b.get("STEP")[0]) == 57
    rc, st = b.status()
    assert rc == B.PD_OK and st[4] == 0


def _colliding_disks():
    """Two disks in oblique contact (damping and friction act every step)."""
    w = I.two_disks(Gc=0.5)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + rc * 0.25
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -6.0
    return w


@pytest.mark.parametrize("prec", [B.PD_FP64, B.PD_FP32_SPLIT])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_split_force_phase_equals_fused_under_contact(prec, lanes):
    """The split force phase hands the same lane sums to the same epilogue:
    identical states on a fracturing impact with velocity-dependent contact."""
    w = _colliding_disks()
    a = _sim(w, prec)
    b = _sim(w, prec)
    a.set_path(0, max(lanes, 4), 128)
    b.set_path(2, max(lanes, 4), 128)
    for k in (1, 16, 33, 250):
        a.step(k)
        b.step(k)
    assert a.get("BROKEN").sum() > 0
    if prec == B.PD_FP64:
        assert np.array_equal(a.get("DISP"), b.get("DISP"))
        assert np.array_equal(a.get("VEL"), b.get("VEL"))
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))
    c = _sim(w, prec)
    c.set_path(2, lanes, 128)
    c.step(300)
    ua, uc = a.get("DISP"), c.get("DISP")
    # another summation order; the fracturing impact amplifies the round-off
    tol = 1e-9 if prec == B.PD_FP64 else 1e-4
    assert np.linalg.norm(uc - ua) <= tol * np.linalg.norm(ua)


def test_autotune_keeps_the_state_and_the_results():
    w = I.merge_aggregates(_parts())
    a = _sim(w, B.PD_FP64)
    b = _sim(w, B.PD_FP64)
    a.step(50)
    b.step(50)
    before = {f: b.get(f) for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP")}
    rep = b.autotune()
    assert rep["mode"] in (0, 1, 2, 3, 4, 6) and rep["lanes"] in (1, 2, 4, 8) and rep["ms_per_step"] > 0
    for f, v in before.items():
        assert np.array_equal(b.get(f), v), f
    a.step(100)
    b.step(100)
    ua, ub = a.get("DISP"), b.get("DISP")
    assert np.linalg.norm(ua - ub) <= 1e-12 * np.linalg.norm(ua)
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))
