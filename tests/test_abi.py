"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/peridem.h declares; host-only calls validate arguments."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "peridem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_binding_symbols():
    assert set(B.SYMBOLS) <= set(_declared())


def test_library_exports_every_declared_symbol():
    L = B.load()
    for name in _declared():
        assert hasattr(L, name), name


def test_invalid_arguments_are_rejected():
    L = B.load()
    ctx = ctypes.c_void_p()
    assert L.pd_create(None, None, None) == B.PD_EINVAL
    p = B.make_params(I.default_params())
    p.dt = 0.0
    assert L.pd_create(ctypes.byref(ctx), ctypes.byref(p), None) == B.PD_EINVAL
    assert b"dt" in L.pd_last_error()
    p = B.make_params(I.default_params())
    assert L.pd_create(ctypes.byref(ctx), ctypes.byref(p), None) == B.PD_OK
    # out of order: bonds before mesh, step before bind
    assert L.pd_build_bonds(ctx, None) == B.PD_ESTATE
    assert L.pd_step(ctx, 1) == B.PD_ESTATE
    # a loop with two vertices is rejected
    sls = np.array([0, 1], np.int32)
    lvs = np.array([0, 2], np.int32)
    vtx = np.array([0, 0, 1, 0], np.float64)
    gs = np.array([0], np.int32)
    gg = np.array([0, 0, 1e-3, 0, 0, 0, 1e-4], np.float64)
    n = ctypes.c_int64()
    rc = L.pd_mesh_grains(ctx, 1, B._ptr(sls), B._ptr(lvs), B._ptr(vtx), 1, B._ptr(gs), B._ptr(gg), ctypes.byref(n))
    assert rc == B.PD_EINVAL
    assert L.pd_destroy(ctx) == B.PD_OK
    assert L.pd_destroy(None) == B.PD_OK


def test_unbound_context_reports_state_errors():
    S = B.Simulation(I.two_disks())
    with pytest.raises(B.PeridemError) as e:
        S.step(1)
    assert e.value.code == B.PD_ESTATE
    with pytest.raises(B.PeridemError) as e:
        S.get("DISP")
    assert e.value.code == B.PD_ESTATE
    with pytest.raises(B.PeridemError) as e:
        S.set("DISP", np.zeros((S.N, 2)))
    assert e.value.code == B.PD_ESTATE
    info = S.info()
    assert info["N"] == S.N and info["max_row"] == 24
