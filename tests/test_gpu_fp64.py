"""GPU parity of the plain FP64 path against the FP64 CPU oracle.

Tolerances (per-step force 1e-12 relative, displacement 1e-9 relative L2 after
1000 steps, identical broken-bond sets) are the targets for the FP64 path.
The kernels evaluate every expression as the oracle does, without FMA
contraction; the default force kernel splits each node over 8 threads, so only
the order of the force sums (and the library's atan2/sin) differ from the
oracle, at round-off level.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-12
DISP_RTOL = 1e-9


def _contact_disks(**over):
    """Two disks already close: the upper one moves down at 1 m/s onto the lower
    one, which sits R_c/4 above the floor -- contact within a few dozen steps."""
    w = I.two_disks(**over)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + rc * 0.25 + 0.0 * h
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    return w


def _gpu(w, store=True, lanes=0):
    return B.Simulation(w, precision=B.PD_FP64, store_parts=store, device="cuda:0", lanes=lanes)


def _push_state(S, P):
    S.set("DISP", P.u)
    S.set("VEL", P.v)
    S.set("ACC", P.a)
    S.set("BROKEN", P.broken[: S.n_bonds])
    S.set("STEP", np.array([P.step], np.int64))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_initial_acceleration_matches_oracle():
    w = _contact_disks()
    S = _gpu(w)
    P = O.OracleProblem.from_workload(w).init_accel()
    assert _rel(S.get("ACC"), P.a) <= FORCE_RTOL


@pytest.mark.parametrize("steps", [60, 200, 400])
def test_force_evaluation_matches_oracle_in_contact(steps):
    w = _contact_disks()
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(steps)
    S = _gpu(w)
    _push_state(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    F = S.get("FORCE")
    parts = S.get("FORCE_PARTS")
    assert np.abs(parts_o[2]).max() > 0 or np.abs(parts_o[3]).max() > 0   # contact or wall active
    scale = np.abs(Fo).max()
    assert np.abs(F - Fo).max() <= FORCE_RTOL * scale
    for k in range(4):
        assert np.abs(parts[k] - parts_o[k]).max() <= FORCE_RTOL * scale, k
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])


def _run_both(w, n, chunks=1):
    S = _gpu(w)
    P = O.OracleProblem.from_workload(w).init_accel()
    for _ in range(chunks):
        S.step(n // chunks)
        F_last, parts_last = P.run(n // chunks, want_parts=True)
    return S, P, F_last, parts_last


def test_candidate_lists_rebuilt_only_after_motion():
    """Contact neighbourhoods come from per-node lists of radius R_c + skin
    (skin = 0.1 R_c), rebuilt only in steps where a node has moved 0.45 skin
    since the last rebuild.  The upper disk moves at about 1 m/s (1e-7 m per
    step) against a trigger of 0.45 * 0.1 * 0.95 h = 5.3e-6 m: about one
    rebuild in 53 steps over 400 steps (plus the one at binding), and the
    trajectory through the impact still matches the oracle's full search."""
    w = _contact_disks()
    S, P, F_last, _ = _run_both(w, 400)
    _, st = S.status()
    assert 3 <= st[B.STATUS_REBUILDS] <= 25, st
    _assert_parity(S, P, F_last)


def _assert_parity(S, P, F_last):
    """Trajectory: displacement within 1e-9 relative L2 and identical broken
    bonds; then the per-step force error from the SAME state (the oracle's state
    loaded into the GPU) within 1e-12 of the largest nodal force."""
    u = S.get("DISP")
    assert np.linalg.norm(u - P.u) <= DISP_RTOL * np.linalg.norm(P.u)
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])
    rc, st = S.status()
    assert rc == B.PD_OK, st
    assert int(S.get("STEP")[0]) == P.step
    _push_state(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    assert np.abs(S.get("FORCE") - Fo).max() <= FORCE_RTOL * np.abs(Fo).max()


def test_two_disks_1000_steps_match_oracle():
    w = _contact_disks()
    S, P, F_last, _ = _run_both(w, 1000, chunks=4)
    assert np.abs(P.v).max() > 0.1
    _assert_parity(S, P, F_last)


def test_settling_50_grains_1000_steps_match_oracle():
    """The 50-grain settling workload (h = R/15, dt = 5e-8) at full size."""
    w = I.settling()
    S, P, F_last, _ = _run_both(w, 1000)
    assert S.N == P.N
    _assert_parity(S, P, F_last)


def test_fracturing_impact_breaks_identical_bonds():
    w = _contact_disks(Gc=0.5)
    w.grain_geom[1, 5] = -6.0
    S, P, F_last, _ = _run_both(w, 300, chunks=3)
    assert P.broken.sum() > 0
    _assert_parity(S, P, F_last)
    dmg = S.get("DAMAGE")
    assert np.allclose(dmg, P.damage(), rtol=0, atol=0)


def _corner_workload():
    """A disk thrown into the lower-left corner while the left and bottom walls
    move inwards and the right/top walls move down/left: single walls, corners,
    wall friction and damping with moving walls."""
    R = 1e-3
    h = R / 8
    p = I.default_params(k_bulk=1.0e6, wall_lo=(0.0, 0.0), wall_hi=(3.2e-3, 3.2e-3), wall_vel_lo=(0.5, 0.3),
                         wall_vel_hi=(-0.4, -0.6), gy=-5000.0)
    rc = p["rc_ratio"] * h
    # an axis-aligned square grain (corner node at (-5h, -5h) from its centre)
    # next to the lower-left corner, and a disk against the right wall
    geom = [(5 * h + 1.1 * rc, 5 * h + 1.2 * rc, R, 0.0, -0.5, -0.4, h),
            (3.2e-3 - 7 * h - 1.05 * rc, 2.0e-3, R * 0.999, 0.2, 0.6, 0.1, h)]
    return I.Workload(shapes=[I.square_shape(), I.disk_shape()], grain_shape=np.array([0, 1], np.int32),
                      grain_geom=np.array(geom), params=p, n_steps=600, name="corner")


def test_moving_walls_and_corners_match_oracle():
    w = _corner_workload()
    S, P, F_last, parts = _run_both(w, 400, chunks=4)
    assert np.abs(parts[3]).max() > 0
    _assert_parity(S, P, F_last)


def test_wall_and_corner_forces_on_a_grid_of_positions():
    """Nodes placed (through the displacement field) on a grid covering the
    single-wall bands and all four corner zones, with random velocities: the
    wall part of the force (segments, corners, damping, friction) matches."""
    w = _corner_workload()
    P = O.OracleProblem.from_workload(w).init_accel()
    S = _gpu(w)
    rc = P.prm[O.P_RC]
    lo, hi = np.array(w.params["wall_lo"]), np.array(w.params["wall_hi"])
    rng = np.random.default_rng(3)
    targets = []
    g = np.linspace(0.02, 1.3, 9) * rc
    for cx, sx in ((lo[0], 1), (hi[0], -1)):
        for cy, sy in ((lo[1], 1), (hi[1], -1)):
            for a in g:
                for b in g:
                    targets.append((cx + sx * a, cy + sy * b))
    targets = np.array(targets)[: P.N]
    n = len(targets)
    P.u[:n] = targets - P.X[:n]
    P.v[:] = rng.normal(scale=0.3, size=P.v.shape)
    P.broken[:] = 1                      # isolate the wall terms: no bond forces
    _push_state(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    parts = S.get("FORCE_PARTS")
    assert np.count_nonzero(parts_o[3][:n, 0]) > 200
    scale = np.abs(parts_o[3]).max()
    assert np.abs(parts[3] - parts_o[3]).max() <= FORCE_RTOL * scale


def test_conic_micromodulus_matches_oracle():
    w = _contact_disks(micromodulus=1)
    S, P, F_last, _ = _run_both(w, 300)
    _assert_parity(S, P, F_last)


def test_diagnostics_match_oracle():
    w = _contact_disks()
    S, P, F_last, _ = _run_both(w, 200)
    d = S.diagnostics()
    o = P.diagnostics()
    for k in ("KE", "E_bond"):
        assert d[k] == pytest.approx(o[k], rel=1e-9), k
    e = P.energies()
    assert e["E_contact"] > 0
    assert d["E_contact"] == pytest.approx(e["E_contact"] + e["E_self"], rel=1e-9)
    assert d["E_wall"] == pytest.approx(e["E_wall"], rel=1e-9, abs=1e-30)
    m = P.prm[O.P_RHO] * P.V
    pscale = np.sum(m * np.abs(P.v).sum(axis=1))
    lscale = pscale * np.abs(P.positions).max()
    for k, sc in (("Px", pscale), ("Py", pscale), ("Lz", lscale)):
        assert abs(d[k] - o[k]) <= 1e-12 * sc, k
    assert d["n_broken"] == o["n_broken"]


def test_checkpoint_resume_is_bitwise():
    w = _contact_disks()
    A = _gpu(w)
    A.step(100)
    ck = {f: A.get(f) for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP")}
    A.step(100)
    B2 = _gpu(w)
    for f, v in ck.items():
        B2.set(f, v)
    B2.step(100)
    for f in ("DISP", "VEL", "ACC", "BROKEN"):
        assert np.array_equal(A.get(f), B2.get(f)), f


def test_page_locked_async_copies_match_synchronous_ones():
    """PD_MEM_HOST_ASYNC: copies enqueued on the stream from and to page-locked
    host memory give the same state as the synchronous copies."""
    import torch

    w = _contact_disks()
    A = _gpu(w)
    A.step(60)
    ck = {f: A.get(f) for f in ("DISP", "VEL", "ACC")}
    B2 = _gpu(w)
    B2.set("STEP", A.get("STEP"))
    B2.set("BROKEN", A.get("BROKEN"))
    for f, v in ck.items():
        t = torch.from_numpy(v.copy()).pin_memory()
        B2.set(f, t)                                    # enqueued, no wait
    A.step(40)
    B2.step(40)
    out = torch.empty((B2.N, 2), dtype=torch.float64).pin_memory()
    lib = B.load()
    B._check(lib.pd_get_state(B2._ctx, B.FIELDS["DISP"], B._ptr(out.numpy()), out.numel() * 8,
                              B.PD_MEM_HOST_ASYNC))
    B2._stream.synchronize()
    assert np.array_equal(out.numpy(), A.get("DISP"))
    assert np.array_equal(B2.get("VEL"), A.get("VEL"))


def test_runs_are_deterministic():
    w = I.settling(n_grains=12, seed=9)
    a = _gpu(w, store=False)
    b = _gpu(w, store=False)
    a.step(150)
    b.step(150)
    assert np.array_equal(a.get("DISP"), b.get("DISP"))
    assert np.array_equal(a.get("VEL"), b.get("VEL"))


def test_nonfinite_state_is_reported_not_faulted():
    w = _contact_disks()
    S = _gpu(w)
    u = S.get("DISP")
    u[3] = np.nan
    S.set("DISP", u)
    S.step(2)
    rc, st = S.status()
    assert rc == B.PD_ENUMERIC
    assert st[2] > 0


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_lane_split_matches_textbook_order(lanes):
    """lanes = 1 sums every force in the oracle's order; 2, 4 and 8 only
    reorder the sums: same broken bonds, displacements within the trajectory
    tolerance (a fracturing impact amplifies round-off)."""
    w = _contact_disks(Gc=0.5)
    w.grain_geom[1, 5] = -6.0
    a = _gpu(w, store=False, lanes=lanes)
    b = _gpu(w, store=False, lanes=8)
    a.step(300)
    b.step(300)
    ua, ub = a.get("DISP"), b.get("DISP")
    assert np.linalg.norm(ua - ub) <= DISP_RTOL * np.linalg.norm(ua)
    assert np.array_equal(a.get("BROKEN"), b.get("BROKEN"))


def test_textbook_order_kernel_matches_oracle():
    w = _contact_disks()
    S = _gpu(w, lanes=1)
    P = O.OracleProblem.from_workload(w).init_accel()
    S.step(400)
    F_last, _ = P.run(400)
    _assert_parity(S, P, F_last)


def test_single_steps_and_chunks_agree():
    """pd_step(1) x 20 and pd_step(20) run the same captured kernels."""
    w = _contact_disks()
    a = _gpu(w, store=False)
    b = _gpu(w, store=False)
    for _ in range(20):
        a.step(1)
    b.step(20)
    assert np.array_equal(a.get("DISP"), b.get("DISP"))
    assert np.array_equal(a.get("VEL"), b.get("VEL"))


def test_integer_square_root_is_the_ieee_square_root():
    """The FP64 bond loop's correctly rounded square root from integer and FP32
    arithmetic equals the hardware's IEEE square root on 2^27 random inputs
    (uniform significands over 100 binades, and exact squares)."""
    for seed in (1, 2):
        mism, first = B.check_sqrt(1 << 27, seed)
        assert mism == 0, (mism, first)
