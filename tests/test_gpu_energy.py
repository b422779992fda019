"""Energy balance of Sec. 4.3 on the GPU path: with normal damping, friction
and breaking switched off, kinetic + bond + contact + wall energy minus the
work of gravity is conserved up to the O(dt^2) error of velocity Verlet.  The
GPU diagnostics (contact and single-wall potentials included) are checked
against the oracle's energies at the same state, and the balance is followed
through an impact of two disks and a disk bouncing on the floor."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _colliding_disks():
    w = I.two_disks(gap=0.02e-3, gy=0.0, friction=0.0, damping_ratio=0.0, Gc=1e9,
                    wall_lo=(-1.0, -1.0), wall_hi=(1.0, 1.0), dt=2e-8)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[1, 0] = 0.3e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    return w


def _bouncing_disk():
    w = I.two_disks(gy=-5000.0, friction=0.0, damping_ratio=0.0, Gc=1e9, dt=2e-8)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_shape = w.grain_shape[:1]
    w.grain_geom = w.grain_geom[:1].copy()
    low = O.OracleProblem.from_workload(w).positions[:, 1].min()
    w.grain_geom[0, 1] += 1.02 * rc - low
    w.grain_geom[0, 5] = -1.0
    return w


def _total(S, w):
    d = S.diagnostics()
    m = w.params["rho"] * S.get("VOLUME")
    p = S.get("POS")
    grav = -np.sum(m * (w.params["gx"] * p[:, 0] + w.params["gy"] * p[:, 1]))
    return d["KE"] + d["E_bond"] + d["E_contact"] + d["E_wall"] + grav, d


@pytest.mark.parametrize("precision,tol", [(B.PD_FP64, 1e-4), (B.PD_FP32_SPLIT, 1e-3)])
@pytest.mark.parametrize("case", ["impact", "floor"])
def test_energy_balance_on_the_gpu(precision, tol, case):
    w = _colliding_disks() if case == "impact" else _bouncing_disk()
    S = B.Simulation(w, precision=precision, device="cuda:0")
    E0, d0 = _total(S, w)
    ke0 = d0["KE"]
    worst, peak = 0.0, 0.0
    key = "E_contact" if case == "impact" else "E_wall"
    for _ in range(40 if case == "floor" else 60):
        S.step(100 if case == "floor" else 50)
        Et, d = _total(S, w)
        peak = max(peak, d[key])
        worst = max(worst, abs(Et - E0) / ke0)
    assert peak > 1e-3 * ke0, peak
    assert worst < tol, worst


@pytest.mark.parametrize("case", ["impact", "floor"])
def test_energies_match_oracle_mid_contact(case):
    """GPU contact and wall potentials against the oracle's at one state in
    contact (the oracle advanced alone, its state pushed into the GPU context)."""
    w = _colliding_disks() if case == "impact" else _bouncing_disk()
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(2050 if case == "impact" else 900)
    S = B.Simulation(w, precision=B.PD_FP64, device="cuda:0")
    S.set("DISP", P.u)
    S.set("VEL", P.v)
    S.set("ACC", P.a)
    S.set("BROKEN", P.broken[: S.n_bonds])
    S.set("STEP", np.array([P.step], np.int64))
    d = S.diagnostics()
    o = P.diagnostics()
    e = P.energies()
    if case == "impact":
        assert e["E_contact"] > 0
    else:
        assert e["E_wall"] > 0
    assert d["E_contact"] == pytest.approx(e["E_contact"] + e["E_self"], rel=1e-9, abs=1e-30)
    assert d["E_wall"] == pytest.approx(e["E_wall"], rel=1e-9, abs=1e-30)
    assert d["KE"] == pytest.approx(o["KE"], rel=1e-12)
    assert d["E_bond"] == pytest.approx(o["E_bond"], rel=1e-9)
