"""The shape-agnostic jammed placement of Sec. 6.1 run on the GPU: every
security disk of the 20 x 30 mm box holds a grain, grains start R_c apart, and
with a seeded 1 m/s kick they reach their neighbours and the walls.  The oracle
runs the first 4000 steps (grains meet, small grains break on the walls); from
that state the FP64 path's force is within 1e-12 of the oracle's and the
FP32-split path's within 1e-5, and 300 further steps of the FP64 path follow
the oracle (displacements within 1e-9 relative L2, identical broken bonds)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import placement as PL

pytestmark = pytest.mark.gpu


def _push(S, P):
    S.set("DISP", P.u)
    S.set("VEL", P.v)
    S.set("ACC", P.a)
    S.set("BROKEN", P.broken[: S.n_bonds])
    S.set("STEP", np.array([P.step], np.int64))


def test_jammed_placement_forces_and_trajectory_match_oracle():
    w = PL.jammed_settling()
    ang = np.random.Generator(np.random.PCG64(77)).uniform(0.0, 2 * math.pi, w.n_grains)
    w.grain_geom[:, 4] = np.cos(ang)
    w.grain_geom[:, 5] = np.sin(ang)
    P = O.OracleProblem.from_workload(w)
    P.omp = True
    P.init_accel()
    P.run(4000)
    S = B.Simulation(w, precision=B.PD_FP64, store_parts=True, device="cuda:0")
    assert S.N == P.N and S.n_bonds == len(P.col)
    _push(S, P)
    S.eval_forces()
    F_or, parts_or = P.forces()
    assert np.abs(parts_or[2]).max() > 0 and np.abs(parts_or[3]).max() > 0 and P.broken.sum() > 0
    scale = np.abs(F_or).max()
    assert np.abs(S.get("FORCE") - F_or).max() <= 1e-12 * scale
    C = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0")
    _push(C, P)
    C.eval_forces()
    assert np.abs(C.get("FORCE") - F_or).max() <= 1e-5 * scale
    # trajectory from the pushed state
    _push(S, P)
    S.step(300)
    P.run(300)
    u = S.get("DISP")
    assert np.linalg.norm(u - P.u) <= 1e-9 * np.linalg.norm(P.u)
    assert np.array_equal(S.get("BROKEN"), P.broken[: S.n_bonds])
