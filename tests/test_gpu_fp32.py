"""FP32-split path: per-step force error against the FP64 oracle (<= 1e-5 of the
largest nodal force, from the same state), break decisions equal to the FP64
path's, and trajectories that stay close to the FP64 ones."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE_RTOL_FP32 = 1e-5


def _contact_disks(**over):
    w = I.two_disks(**over)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + rc * 0.25
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    return w


def _sim(w, prec, store=True):
    return B.Simulation(w, precision=prec, store_parts=store, device="cuda:0")


def _push(S, P):
    S.set("DISP", P.u)
    S.set("VEL", P.v)
    S.set("ACC", P.a)
    S.set("BROKEN", P.broken[: S.n_bonds])
    S.set("STEP", np.array([P.step], np.int64))


def _thrown_settling():
    """The 50-grain settling aggregate thrown at the floor (vy = -5 m/s), so that
    wall and grain contacts are loaded within a few hundred steps."""
    w = I.settling()
    P = O.OracleProblem.from_workload(w)
    w.grain_geom[:, 1] -= P.X[:, 1].min() - 1.2 * P.prm[O.P_RC]     # lowest node just above the floor
    w.grain_geom[:, 5] = -5.0
    return w


@pytest.mark.parametrize("case,steps", [("disks", 100), ("disks", 400), ("settling", 300)])
def test_fp32_force_error_against_oracle(case, steps):
    """Per-step force error from the same (loaded) state: the FP32-split forces
    against the FP64 oracle, relative to the largest nodal force."""
    w = _contact_disks() if case == "disks" else _thrown_settling()
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(steps)
    S = _sim(w, B.PD_FP32_SPLIT)
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    F = S.get("FORCE")
    assert np.abs(parts_o[2]).max() > 0 or np.abs(parts_o[3]).max() > 0
    err = np.abs(F - Fo).max() / np.abs(Fo).max()
    assert err <= FORCE_RTOL_FP32, err
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])


def test_fp32_bond_force_error_far_from_origin():
    """Large rigid motion (grain translated by 3 mm): the float-float relative
    displacement keeps the bond forces accurate."""
    w = _contact_disks()
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(150)
    P.u[:, 0] += 3e-3
    P.u[:, 1] += 2e-3
    S = _sim(w, B.PD_FP32_SPLIT)
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    parts = S.get("FORCE_PARTS")
    err = np.abs(parts[0] - parts_o[0]).max() / np.abs(parts_o[0]).max()
    assert err <= FORCE_RTOL_FP32, err


def test_fp32_breaks_same_bonds_as_fp64_in_fracturing_impact():
    w = _contact_disks(Gc=0.5)
    w.grain_geom[1, 5] = -6.0
    a = _sim(w, B.PD_FP64, store=False)
    b = _sim(w, B.PD_FP32_SPLIT, store=False)
    for _ in range(6):
        a.step(50)
        b.step(50)
    ba, bb = a.get("BROKEN"), b.get("BROKEN")
    assert ba.sum() > 0
    assert int(np.sum(ba != bb)) == 0
    assert np.array_equal(a.get("DAMAGE"), b.get("DAMAGE"))


def test_fp32_trajectory_tracks_fp64():
    w = I.settling()
    a = _sim(w, B.PD_FP64, store=False)
    b = _sim(w, B.PD_FP32_SPLIT, store=False)
    a.step(1000)
    b.step(1000)
    ua, ub = a.get("DISP"), b.get("DISP")
    assert np.linalg.norm(ub - ua) <= 1e-5 * np.linalg.norm(ua)
    rc, st = b.status()
    assert rc == B.PD_OK


def _corner_workload():
    """A square grain in the lower-left corner and a disk at the right wall, all
    four walls moving (single walls, corners, wall damping and friction)."""
    R = 1e-3
    h = R / 8
    p = I.default_params(k_bulk=1.0e6, wall_lo=(0.0, 0.0), wall_hi=(3.2e-3, 3.2e-3), wall_vel_lo=(0.5, 0.3),
                         wall_vel_hi=(-0.4, -0.6), gy=-5000.0)
    rc = p["rc_ratio"] * h
    geom = [(5 * h + 1.1 * rc, 5 * h + 1.2 * rc, R, 0.0, -0.5, -0.4, h),
            (3.2e-3 - 7 * h - 1.05 * rc, 2.0e-3, R * 0.999, 0.2, 0.6, 0.1, h)]
    return I.Workload(shapes=[I.square_shape(), I.disk_shape()], grain_shape=np.array([0, 1], np.int32),
                      grain_geom=np.array(geom), params=p, n_steps=600, name="corner")


def test_fp32_wall_and_corner_forces_on_a_grid_of_positions():
    """The FP32-split wall terms (float single-wall segments, FP64 corner zones)
    against the oracle for nodes on a grid over the single-wall bands and the
    four corner zones, with random velocities: per node within 1e-5 of the
    largest wall force."""
    w = _corner_workload()
    P = O.OracleProblem.from_workload(w).init_accel()
    S = _sim(w, B.PD_FP32_SPLIT)
    rc = P.prm[O.P_RC]
    lo, hi = np.array(w.params["wall_lo"]), np.array(w.params["wall_hi"])
    rng = np.random.default_rng(4)
    g = np.linspace(0.02, 1.3, 9) * rc
    targets = [(cx + sx * a, cy + sy * b) for cx, sx in ((lo[0], 1), (hi[0], -1)) for cy, sy in ((lo[1], 1), (hi[1], -1))
               for a in g for b in g]
    targets = np.array(targets)[: P.N]
    n = len(targets)
    P.u[:n] = targets - P.X[:n]
    P.v[:] = rng.normal(scale=0.3, size=P.v.shape)
    P.broken[:] = 1                      # no bond forces
    _push(S, P)
    S.eval_forces()
    _, parts_o = P.forces()
    parts = S.get("FORCE_PARTS")
    single = np.array([(min(a, b) < rc) and np.hypot(a, b) >= rc for a in g for b in g] * 4)[:n]
    assert single.sum() > 50             # nodes on the float single-wall path
    assert np.count_nonzero(parts_o[3][:n, 0]) > 200
    scale = np.abs(parts_o[3]).max()
    assert np.abs(parts[3] - parts_o[3]).max() <= FORCE_RTOL_FP32 * scale


def test_fp32_stiff_material_contact_and_walls_stay_finite():
    """A GPa-range bulk modulus (K_n ~ 1e28 in float) in grain and wall contact:
    the FP32-split damping must not overflow; the force matches the oracle."""
    w = _contact_disks(k_bulk=2.0e9)
    rc = w.params["rc_ratio"] * 1e-3 / 8
    w.grain_geom[1, 1] -= 0.5 * rc        # the disks overlap: node-node contact from the start
    X = O.OracleProblem.from_workload(w).X
    w.grain_geom[:, 1] -= X[:, 1].min() - 0.5 * rc     # lowest node R_c / 2 above the floor
    P = O.OracleProblem.from_workload(w).init_accel()
    S = _sim(w, B.PD_FP32_SPLIT)
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    F = S.get("FORCE")
    assert np.abs(parts_o[2]).max() > 0 and np.abs(parts_o[3]).max() > 0
    assert np.all(np.isfinite(F))
    assert np.abs(F - Fo).max() <= FORCE_RTOL_FP32 * np.abs(Fo).max()


def test_fp32_acceleration_field_is_kept_in_float():
    """The FP32-split context keeps the acceleration in FP32: ACC set from
    doubles reads back as the float-rounded values, through host and device
    buffers alike, and the next step starts from them."""
    import torch
    w = _contact_disks()
    S = _sim(w, B.PD_FP32_SPLIT, store=False)
    rng = np.random.default_rng(7)
    a = rng.normal(scale=3.0e3, size=(S.N, 2))
    S.set("ACC", a)
    af = a.astype(np.float32).astype(np.float64)
    assert np.array_equal(S.get("ACC"), af)
    dev = torch.empty((S.N, 2), dtype=torch.float64, device="cuda:0")
    S.get_device("ACC", dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), af)
    S.set("ACC", a[::-1].copy())
    assert np.array_equal(S.get("ACC"), a[::-1].astype(np.float32).astype(np.float64))
