"""Materials on the GPU (Sec. 4.1 harmonic-mean bulk modulus in K_n, per-grain
density and bond constants) against the FP64 oracle: the FP64 path to 1e-12
per-step force and 1e-9 relative L2 displacement, the FP32-split path to 1e-5
per-step force, identical broken bonds; a one-material table reproduces the
single-material run bit for bit."""
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


def test_two_materials_fp64_trajectory_and_forces_match_oracle():
    w = I.two_material_disks()
    S = B.Simulation(w, precision=B.PD_FP64, store_parts=True, device="cuda:0")
    P = O.OracleProblem.from_workload(w).init_accel()
    assert np.abs(S.get("ACC") - P.a).max() <= 1e-12 * np.abs(P.a).max()
    S.step(600)
    P.run(600)
    u = S.get("DISP")
    assert np.linalg.norm(u - P.u) <= 1e-9 * np.linalg.norm(P.u)
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    parts = S.get("FORCE_PARTS")
    assert np.abs(parts_o[2]).max() > 0                     # the two materials are in contact
    scale = np.abs(Fo).max()
    assert np.abs(S.get("FORCE") - Fo).max() <= 1e-12 * scale
    for k in range(4):
        assert np.abs(parts[k] - parts_o[k]).max() <= 1e-12 * scale, k
    rc, st = S.status()
    assert rc == B.PD_OK


def test_two_materials_fp32_force_error_against_oracle():
    w = I.two_material_disks()
    P = O.OracleProblem.from_workload(w).init_accel()
    P.run(500)
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0")
    _push(S, P)
    S.eval_forces()
    Fo, parts_o = P.forces()
    assert np.abs(parts_o[2]).max() > 0
    assert np.abs(S.get("FORCE") - Fo).max() <= 1e-5 * np.abs(Fo).max()
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])


@pytest.mark.parametrize("prec", [B.PD_FP64, B.PD_FP32_SPLIT])
def test_one_material_table_is_bitwise_single_material(prec):
    w = I.two_material_disks()
    p = w.params
    w1 = I.two_material_disks()
    w1.materials = (np.array([[p["E"], p["k_bulk"], p["rho"], p["Gc"]]]), np.zeros(2, dtype=np.int32))
    w.materials = None
    a = B.Simulation(w, precision=prec, device="cuda:0")
    b = B.Simulation(w1, precision=prec, device="cuda:0")
    a.step(300)
    b.step(300)
    assert np.array_equal(a.get("DISP"), b.get("DISP"))
    assert np.array_equal(a.get("VEL"), b.get("VEL"))
