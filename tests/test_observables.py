"""Observables of the settling and compaction sections (Sec. 6): volume
fraction, particle / bulk damage and the force the aggregate exerts on a wall.

CPU: the oracle's observables against what mechanics and geometry fix.  GPU:
pd_observables against the oracle at the same state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I


def _resting_disk():
    w = I.two_disks()
    w.grain_geom = w.grain_geom[:1].copy()
    w.grain_shape = w.grain_shape[:1].copy()
    w.grain_geom[0, 1] = 1e-3 + 0.3 * 0.95e-3 / 8        # 0.3 R_c above the floor
    return w


def test_floor_carries_the_weight_at_rest():
    """Newton: once the damped bounce has died out, the time-averaged force on
    the floor is the grain's weight (pointing down)."""
    P = O.OracleProblem.from_workload(_resting_disk()).init_accel()
    weight = P.prm[O.P_RHO] * P.V.sum() * -P.prm[O.P_GY]
    P.run(50_000)
    f = []
    for _ in range(40):
        P.run(250)
        f.append(P.wall_reaction(2))
    f = np.array(f)
    assert abs(f[:, 1].mean() / -weight - 1.0) < 5e-3
    assert abs(f[:, 0].mean()) < 1e-3 * weight           # no tangential load on a level floor
    side = np.array([P.wall_reaction(l) for l in (0, 1, 3)])
    assert np.all(side == 0.0)                            # walls out of reach feel nothing


def test_wall_shares_add_up_to_the_total_wall_force():
    """Each corner term is split between its two walls: the four wall forces add
    up to minus the summed wall force on the nodes (eq:wall-total)."""
    R, h = 1e-3, 1e-3 / 10
    rc = 0.95 * h
    half = R / np.sqrt(2.0)                               # axis-aligned square of side sqrt(2) R
    params = I.default_params(k_bulk=1e6, gx=-5000.0, gy=-5000.0, wall_lo=(0.0, 0.0), wall_hi=(5e-3, 5e-3))
    w = I.Workload(shapes=[I.square_shape()], grain_shape=np.array([0], np.int32),
                   grain_geom=np.array([[half + 0.2 * rc, half + 0.2 * rc, R, 0.0, -0.2, -0.2, h]]),
                   params=params, n_steps=1)
    P = O.OracleProblem.from_workload(w)                  # corner node 0.27 R_c from both walls
    _, parts = P.forces()
    total = parts[3].sum(axis=0)
    walls = sum(P.wall_reaction(l) for l in range(4))
    single, corner = P.wall_sums()
    assert np.abs(corner).max() > 0 and np.abs(single[0]).max() > 0 and np.abs(single[2]).max() > 0
    assert np.allclose(walls, -total, rtol=1e-12, atol=1e-12 * np.abs(total).max())


def test_bulk_damage_is_the_mean_over_particles():
    """Bulk damage averages particle damage over particles, not over nodes: a
    fully broken small grain and an intact large one give 1/2."""
    w = I.two_disks()
    w.grain_geom[1, 2] = 0.5e-3                           # second disk: half the radius, same h
    w.grain_geom[1, 1] += 2e-3
    P = O.OracleProblem.from_workload(w)
    first = P.grain == 1
    rows = np.repeat(np.arange(P.N), np.diff(P.row_ptr))
    P.broken[: len(P.col)] = first[rows].astype(np.uint8)
    assert np.allclose(P.particle_damage(), [0.0, 1.0])
    assert P.bulk_damage() == 0.5
    assert P.damage().mean() < 0.5                        # the node average is not the bulk damage


def test_volume_fraction_follows_the_moving_lid():
    """phi(t) = sum V / (l (H - v t)): the ratio to phi(0) is H / (H - v t)."""
    w = I.compaction(n_grains=6, width=8e-3, seed=4, wall_speed=0.5)
    P = O.OracleProblem.from_workload(w)
    lo, hi = w.params["wall_lo"], w.params["wall_hi"]
    H = hi[1] - lo[1]
    t = 2e-3
    assert P.volume_fraction(t) / P.volume_fraction(0.0) == pytest.approx(H / (H - 0.5 * t), rel=1e-14)


def _lid_and_floor(n_grains=8, seed=4, lid_speed=3.0):
    """Floor and lid moved to within R_c / 2 of the lowest and highest node, the
    lid moving down: both walls carry load from the first steps on."""
    w = I.settling(n_grains=n_grains, box=(12e-3, 12e-3), seed=seed)
    X = B.Simulation(w).get("X")
    rc = w.params["rc_ratio"] * float(w.grain_geom[:, 6].min())
    w.params["wall_lo"] = (w.params["wall_lo"][0], float(X[:, 1].min()) - 0.5 * rc)
    w.params["wall_hi"] = (w.params["wall_hi"][0], float(X[:, 1].max()) + 0.5 * rc)
    w.params["wall_vel_hi"] = (0.0, -lid_speed)
    return w


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [B.PD_FP64, B.PD_FP32_SPLIT])
def test_gpu_observables_match_the_oracle(prec):
    w = _lid_and_floor()
    # the oracle advances 300 steps; its state goes into the GPU context
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(300)
    S = B.Simulation(w, precision=prec, device="cuda:0")
    for f, val in (("DISP", P.u), ("VEL", P.v), ("ACC", P.a), ("BROKEN", P.broken[: S.n_bonds]),
                   ("STEP", np.array([P.step], np.int64))):
        S.set(f, val)
    obs = S.observables()
    assert obs.shape == (1, 4)
    assert obs[0, 0] == pytest.approx(P.volume_fraction(), rel=1e-14)
    assert obs[0, 1] == pytest.approx(P.bulk_damage(), rel=1e-12, abs=1e-15)
    top, bottom = P.wall_reaction(3)[1], P.wall_reaction(2)[1]
    scale = max(abs(top), abs(bottom), 1e-30)
    assert abs(obs[0, 2] - top) <= 1e-10 * scale
    assert abs(obs[0, 3] - bottom) <= 1e-10 * scale
    assert abs(top) + abs(bottom) > 0


@pytest.mark.gpu
def test_gpu_observables_per_aggregate():
    parts = [_lid_and_floor(n_grains=6, seed=5 + a, lid_speed=2.0 + a) for a in range(3)]
    merged = I.merge_aggregates(parts)
    S = B.Simulation(merged, precision=B.PD_FP64, device="cuda:0")
    S.step(300)
    obs = S.observables()
    assert obs.shape == (3, 4)
    for a, w in enumerate(parts):
        A = B.Simulation(w, precision=B.PD_FP64, device="cuda:0")
        A.step(300)
        oa = A.observables()[0]
        assert obs[a, 0] == pytest.approx(oa[0], rel=1e-14)
        assert obs[a, 1] == pytest.approx(oa[1], rel=1e-9, abs=1e-12)
        assert np.allclose(obs[a, 2:], oa[2:], rtol=1e-6, atol=1e-9 * max(1.0, np.abs(oa[2:]).max()))
