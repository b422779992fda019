"""Bounded waits of the persistent step kernel.

One block withholds its arrival at the first grid barrier (pd_set_wait_test),
so the other blocks' barrier waits run out: the launch must return by itself
with status[PD_STATUS_TIMEOUT] set and pd_status reporting PD_ETIMEOUT, with
no device fault.  After the state is restored and the status cleared
(pd_clear_status) the same context must step on exactly as one that never
timed out (the FP64 path also agrees with the FP64 oracle).  The FP32-split
case also covers the persistent kernel's prediction of the next step, which a
timed-out launch leaves half written.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATUS_TIMEOUT = 4


def _contact_disks():
    """Two disks 1.05 R_c apart, the upper one moving down at 1 m/s: contact
    (and a candidate-list rebuild) within the first steps."""
    w = I.two_disks()
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + rc * 0.25
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    return w


def _state(S):
    return {f: S.get(f) for f in ("DISP", "VEL", "ACC", "BROKEN", "STEP")}


def _restore(S, st):
    for f, val in st.items():
        S.set(f, val)


@pytest.mark.parametrize("withhold,prec,lanes,block", [(0, B.PD_FP64, 8, 128), (3, B.PD_FP64, 8, 128),
                                                      (1, B.PD_FP32_SPLIT, 1, 256)])
def test_barrier_timeout_is_reported_and_the_context_recovers(withhold, prec, lanes, block):
    w = _contact_disks()
    S = B.Simulation(w, precision=prec, device="cuda:0")
    S.set_path(1, lanes, block)
    s0 = _state(S)

    # a withheld block: the others give up after 20000 polls (a few ms)
    S.set_wait_test(withhold_block=withhold, max_spins=20_000)
    t0 = time.perf_counter()
    S.step(1)
    rc, st = S.status()
    elapsed = time.perf_counter() - t0
    assert rc == B.PD_ETIMEOUT
    assert st[STATUS_TIMEOUT] == 1
    assert elapsed < 30.0

    # back to the default waits; restore the state, clear the status, step on
    S.set_wait_test()
    _restore(S, s0)
    S.clear_status()
    rc, st = S.status()
    assert rc == B.PD_OK and not st.any()
    n = 120
    S.step(n)
    rc, st = S.status()
    assert rc == B.PD_OK and st[STATUS_TIMEOUT] == 0
    u_rec = S.get("DISP")

    # a context that never timed out, from the same state
    R = B.Simulation(w, precision=prec, device="cuda:0")
    R.set_path(1, lanes, block)
    R.clear_status()
    R.step(n)
    u_ref = R.get("DISP")
    scale = np.abs(u_ref).max()
    assert scale > 0
    assert np.abs(u_rec - u_ref).max() <= 1e-12 * scale
    assert np.array_equal(S.get("BROKEN"), R.get("BROKEN"))

    # and the oracle (the FP32 split's own oracle parity is tested elsewhere)
    if prec == B.PD_FP64:
        P = O.OracleProblem.from_workload(w).init_accel()
        P.run(n)
        assert np.abs(u_rec - P.u).max() <= 1e-9 * np.abs(P.u).max()


def test_wait_test_arguments_are_checked():
    S = B.Simulation(_contact_disks(), precision=B.PD_FP64, device="cuda:0")
    with pytest.raises(B.PeridemError):
        S.set_wait_test(withhold_block=-2)
    with pytest.raises(B.PeridemError):
        S.set_wait_test(withhold_block=0, max_spins=-1)
