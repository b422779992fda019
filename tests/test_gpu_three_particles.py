"""The symmetric-impact test of Sec. 5.3 (a notched square hit from below and
above by two rectangles): fracture, child particles and self-contact across
the closing notch, GPU against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _push(S, P):
    S.set("DISP", P.u)
    S.set("VEL", P.v)
    S.set("ACC", P.a)
    S.set("BROKEN", P.broken[: S.n_bonds])
    S.set("STEP", np.array([P.step], np.int64))


@pytest.mark.parametrize("prec,tol", [(B.PD_FP64, 1e-12), (B.PD_FP32_SPLIT, 1e-5)])
def test_shattered_state_forces_match_oracle(prec, tol):
    """Per-step force from the oracle's state after 250 steps of the soft case
    (G_c = 13.5 J/m^2: particle A shattered, self-contact between its pieces)."""
    w = I.three_particles(gc_a=13.5)
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(250)
    S = B.Simulation(w, precision=prec, store_parts=True, device="cuda:0")
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    assert np.abs(parts_o[1]).max() > 0                     # self-contact is active
    scale = np.abs(Fo).max()
    assert np.abs(S.get("FORCE") - Fo).max() <= tol * scale
    parts = S.get("FORCE_PARTS")
    for k in range(4):
        assert np.abs(parts[k] - parts_o[k]).max() <= tol * scale, k
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])


def test_fp64_trajectory_with_fracture_matches_oracle():
    w = I.three_particles(gc_a=135.0)
    S = B.Simulation(w, precision=B.PD_FP64, device="cuda:0")
    P = O.OracleProblem.from_workload(w).init_accel()
    S.step(500)
    P.run(500)
    assert int(P.broken.sum()) > 0
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])
    assert np.linalg.norm(S.get("DISP") - P.u) <= 1e-9 * np.linalg.norm(P.u)
    rc, st = S.status()
    assert rc == B.PD_OK


def test_lower_fracture_energy_breaks_more_of_particle_a():
    """Sec. 5.3: with G_c = 13.5 J/m^2 particle A fractures far more than with
    135 J/m^2 (FP32-split path, 1500 steps = 30 us)."""
    broken = {}
    for gc in (135.0, 13.5):
        w = I.three_particles(gc_a=gc)
        S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device="cuda:0")
        S.step(1500)
        g = S.get("GRAIN")
        row = S.get("ROW_PTR")
        owner = np.repeat(g, np.diff(row))
        broken[gc] = int(S.get("BROKEN")[owner == 0].sum())
        assert S.status()[0] == B.PD_OK
    assert broken[135.0] > 0
    assert broken[13.5] > 5 * broken[135.0]
