"""pd_diagnostics_noalloc: the diagnostics reduction for callers that cannot
allocate device memory (their device memory comes from a fixed budget or
another runtime).  It must give the same sums as pd_diagnostics, call after
call, from state arrays the caller owns.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _workload():
    w = I.two_disks(Gc=0.5)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + 0.25 * rc
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -6.0                 # fracturing impact: broken bonds appear
    return w


def test_noalloc_diagnostics_match_pd_diagnostics_on_two_calls():
    torch = pytest.importorskip("torch")
    w = _workload()
    S = B.Simulation(w, precision=B.PD_FP64, device="cuda:0")
    P = O.OracleProblem.from_workload(w)
    L = B.load()
    vp = ctypes.c_void_p
    L.pd_diagnostics_noalloc.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                         ctypes.c_int, vp, vp]
    L.pd_diagnostics_noalloc.restype = ctypes.c_int
    dev = torch.device("cuda:0")
    N = S.N

    def dev_field(name, shape, dtype):
        t = torch.empty(shape, dtype=dtype, device=dev)
        return S.get_device(name, t)

    g_cw = torch.tensor(P.g_cw, dtype=torch.float64, device=dev)
    g_eps = torch.tensor(P.g_eps, dtype=torch.float64, device=dev)
    X = dev_field("X", (N, 2), torch.float64)
    Vd = dev_field("VOLUME", (N,), torch.float64)
    grain = dev_field("GRAIN", (N,), torch.int32)
    row = dev_field("ROW_PTR", (N + 1,), torch.int32)
    col = dev_field("COL", (S.n_bonds,), torch.int32)
    stream = torch.cuda.current_stream(dev).cuda_stream
    saw_broken = False
    for call in range(2):
        S.step(150)
        ref = S.diagnostics()
        u = dev_field("DISP", (N, 2), torch.float64)
        v = dev_field("VEL", (N, 2), torch.float64)
        broken = torch.from_numpy(S.get("BROKEN")).to(dev)
        out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
        rc = L.pd_diagnostics_noalloc(N, X.data_ptr(), u.data_ptr(), v.data_ptr(), Vd.data_ptr(), grain.data_ptr(),
                                      row.data_ptr(), col.data_ptr(), broken.data_ptr(), g_cw.data_ptr(),
                                      g_eps.data_ptr(), w.params["rho"], int(w.params["micromodulus"]),
                                      out.data_ptr(), vp(stream))
        assert rc == B.PD_OK, L.pd_last_error()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ref["KE"], rel=1e-12)
        assert got[1] == pytest.approx(ref["E_bond"], rel=1e-12)
        m = w.params["rho"] * S.get("VOLUME")
        vh = S.get("VEL")
        pscale = float(np.sum(m * np.abs(vh).sum(axis=1)))
        assert abs(got[2] - ref["Px"]) <= 1e-12 * pscale
        assert abs(got[3] - ref["Py"]) <= 1e-12 * pscale
        assert abs(got[4] - ref["Lz"]) <= 1e-12 * pscale * float(np.abs(S.get("POS")).max())
        assert int(got[5]) == ref["n_broken"]
        saw_broken |= ref["n_broken"] > 0
    assert saw_broken


def test_noalloc_diagnostics_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = B.load()
    vp = ctypes.c_void_p
    L.pd_diagnostics_noalloc.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                         ctypes.c_int, vp, vp]
    L.pd_diagnostics_noalloc.restype = ctypes.c_int
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    rc = L.pd_diagnostics_noalloc(2097152 + 1, *([None] * 10), 1200.0, 0, out.data_ptr(), None)
    assert rc == B.PD_EINVAL
    assert b"PD_NOALLOC_MAX_NODES" in L.pd_last_error()
