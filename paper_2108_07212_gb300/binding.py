"""Thin Python binding of libperidem.so (the C ABI of include/peridem.h).

Argument marshalling only: every step of the time loop runs in the library's
CUDA kernels.  PyTorch supplies the device arena and the CUDA stream.  There
is no fallback: if the library cannot be loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

c_double, c_int32, c_int64, c_size_t, c_void_p = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                                   ctypes.c_size_t, ctypes.c_void_p)

PD_OK, PD_EINVAL, PD_ESTATE, PD_ECUDA, PD_ENUMERIC, PD_EOVERFLOW, PD_ENOMEM, PD_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
PD_FP64, PD_FP32_SPLIT = 0, 1
PD_MEM_HOST, PD_MEM_DEVICE, PD_MEM_HOST_ASYNC = 0, 1, 2     # buffer kinds of pd_get_state / pd_set_state
FIELDS = dict(X=0, DISP=1, VEL=2, ACC=3, POS=4, FORCE=5, FORCE_PARTS=6, BROKEN=7, DAMAGE=8, GRAIN=9,
              VOLUME=10, ROW_PTR=11, COL=12, LATTICE=13, STEP=14, GRAIN_TEMPLATE=15)
STATUS_COUNT = 8
STATUS_REBUILDS = 5          # slot of the candidate-list rebuild counter (not an error)
DIAG_COUNT = 8
DIAG_NAMES = ("KE", "E_bond", "Px", "Py", "Lz", "n_broken", "E_contact", "E_wall")

# public C-ABI symbols (checked by the test-suite against include/peridem.h)
SYMBOLS = ("pd_last_error", "pd_create", "pd_destroy", "pd_mesh_grains", "pd_build_bonds", "pd_arena_bytes",
           "pd_bind_arena", "pd_step", "pd_get_state", "pd_set_state", "pd_eval_forces", "pd_diagnostics",
           "pd_status", "pd_info", "pd_set_timing", "pd_kernel_times", "pd_set_aggregates", "pd_autotune", "pd_set_path", "pd_mlp_create", "pd_mlp_destroy",
           "pd_mlp_arena_bytes", "pd_mlp_bind_arena", "pd_mlp_set_params", "pd_mlp_get_params", "pd_mlp_forward",
           "pd_mlp_loss_grad", "pd_mlp_train_step", "pd_surrogate_setup", "pd_surrogate_set_mlp",
           "pd_surrogate_enable", "pd_surrogate_sample", "pd_surrogate_stats", "pd_surrogate_inspect",
           "pd_diagnostics_noalloc", "pd_observables", "pd_set_materials", "pd_check_sqrt",
           "pd_surrogate_basis", "pd_clear_status", "pd_set_wait_test")


class PdParams(ctypes.Structure):
    _fields_ = [("E", c_double), ("nu", c_double), ("k_bulk", c_double), ("rho", c_double), ("Gc", c_double),
                ("horizon_ratio", c_double), ("rc_ratio", c_double), ("damping_ratio", c_double),
                ("friction", c_double), ("gravity", c_double * 2), ("dt", c_double),
                ("wall_lo", c_double * 2), ("wall_hi", c_double * 2), ("wall_vel_lo", c_double * 2),
                ("wall_vel_hi", c_double * 2), ("micromodulus", c_int32), ("precision", c_int32),
                ("store_parts", c_int32), ("lanes", c_int32)]


class PeridemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"peridem error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load():
    """Load libperidem.so, building it in-tree first if nvcc is available."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libperidem.so is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(_build.LIB)
            vp, ip = c_void_p, c_int32
            L.pd_last_error.restype = ctypes.c_char_p
            L.pd_create.argtypes = [ctypes.POINTER(c_void_p), ctypes.POINTER(PdParams), vp]
            L.pd_destroy.argtypes = [vp]
            L.pd_mesh_grains.argtypes = [vp, ip, vp, vp, vp, ip, vp, vp, ctypes.POINTER(c_int64)]
            L.pd_build_bonds.argtypes = [vp, ctypes.POINTER(c_int64)]
            L.pd_arena_bytes.argtypes = [vp, ctypes.POINTER(c_size_t)]
            L.pd_bind_arena.argtypes = [vp, vp, c_size_t]
            L.pd_step.argtypes = [vp, ip]
            L.pd_get_state.argtypes = [vp, ip, vp, c_size_t, ip]
            L.pd_set_state.argtypes = [vp, ip, vp, c_size_t, ip]
            L.pd_eval_forces.argtypes = [vp]
            L.pd_diagnostics.argtypes = [vp, vp]
            L.pd_status.argtypes = [vp, vp]
            L.pd_clear_status.argtypes = [vp]
            L.pd_set_wait_test.argtypes = [vp, ip, ctypes.c_longlong]
            L.pd_info.argtypes = [vp, vp]
            L.pd_set_timing.argtypes = [vp, ip]
            L.pd_kernel_times.argtypes = [vp, vp]
            L.pd_set_aggregates.argtypes = [vp, ip, vp, vp]
            L.pd_set_materials.argtypes = [vp, ip, vp, vp]
            L.pd_autotune.argtypes = [vp, vp]
            L.pd_set_path.argtypes = [vp, ip, ip, ip]
            L.pd_mlp_create.argtypes = [ctypes.POINTER(c_void_p), ip, vp]
            L.pd_mlp_destroy.argtypes = [vp]
            L.pd_mlp_arena_bytes.argtypes = [vp, ctypes.POINTER(c_size_t)]
            L.pd_mlp_bind_arena.argtypes = [vp, vp, c_size_t]
            L.pd_mlp_set_params.argtypes = [vp, vp]
            L.pd_mlp_get_params.argtypes = [vp, vp]
            L.pd_mlp_forward.argtypes = [vp, vp, vp, ip]
            L.pd_mlp_loss_grad.argtypes = [vp, vp, vp, ip, vp, vp]
            L.pd_mlp_train_step.argtypes = [vp, vp, vp, ip, ctypes.c_float, vp]
            L.pd_surrogate_setup.argtypes = [vp, ip, vp, vp, ip, c_double, c_double]
            L.pd_surrogate_set_mlp.argtypes = [vp, ip, vp]
            L.pd_surrogate_enable.argtypes = [vp, ip]
            L.pd_surrogate_sample.argtypes = [vp, vp, vp]
            L.pd_surrogate_stats.argtypes = [vp, vp, vp, vp]
            L.pd_surrogate_basis.argtypes = [vp, ip, vp, ctypes.POINTER(c_size_t), vp, vp]
            L.pd_check_sqrt.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, vp, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(c_double)]
            for name in SYMBOLS:
                if name != "pd_last_error":
                    getattr(L, name).restype = ip
            _lib = L
    return _lib


def _check(rc):
    if rc != PD_OK:
        raise PeridemError(rc, load().pd_last_error().decode())
    return rc


def make_params(p: dict, precision: int = PD_FP64, store_parts: bool = False, lanes: int = 0) -> PdParams:
    q = PdParams()
    for name in ("E", "nu", "k_bulk", "rho", "Gc", "horizon_ratio", "rc_ratio", "damping_ratio", "friction", "dt"):
        setattr(q, name, float(p[name]))
    q.gravity[:] = (float(p["gx"]), float(p["gy"]))
    q.wall_lo[:] = tuple(map(float, p["wall_lo"]))
    q.wall_hi[:] = tuple(map(float, p["wall_hi"]))
    q.wall_vel_lo[:] = tuple(map(float, p["wall_vel_lo"]))
    q.wall_vel_hi[:] = tuple(map(float, p["wall_vel_hi"]))
    q.micromodulus = int(p["micromodulus"])
    q.precision = int(precision)
    q.store_parts = 1 if store_parts else 0
    q.lanes = int(lanes)
    return q


def check_sqrt(n: int, seed: int = 1, stream=None) -> tuple:
    """pd_check_sqrt: (mismatches, first mismatching input or None) of the FP64
    path's integer square root against the hardware IEEE square root."""
    mm = ctypes.c_longlong(0)
    first = c_double(float("nan"))
    s = c_void_p(stream.cuda_stream) if stream is not None else None
    _check(load().pd_check_sqrt(int(n), int(seed), s, ctypes.byref(mm), ctypes.byref(first)))
    return int(mm.value), (None if mm.value == 0 else first.value)


def _ptr(a: np.ndarray):
    return c_void_p(a.ctypes.data)


class Simulation:
    """One PeriDEM problem bound to the library.

    ``device=None`` meshes and builds bonds only (host work; no GPU needed).
    With a CUDA device the state lives in one torch-allocated arena and all
    work runs on ``stream`` (default: the current torch stream).
    """

    def __init__(self, workload, precision: int | str = PD_FP64, store_parts: bool = False, device=None,
                 stream=None, lanes: int = 0, surrogate=None):
        L = load()
        if isinstance(precision, str):
            precision = {"fp64": PD_FP64, "fp32": PD_FP32_SPLIT, "fp32_split": PD_FP32_SPLIT}[precision]
        self.precision = precision
        self.workload = workload
        self.device = device
        self._arena = None
        self._stream = None
        sptr = None
        if device is not None:
            import torch
            self._stream = stream if stream is not None else torch.cuda.current_stream(torch.device(device))
            sptr = c_void_p(self._stream.cuda_stream)
        self._params = make_params(workload.params, precision, store_parts, lanes)
        ctx = c_void_p()
        _check(L.pd_create(ctypes.byref(ctx), ctypes.byref(self._params), sptr))
        self._ctx = ctx
        sls, lvs, vtx = workload.flat_shapes()
        gs = np.ascontiguousarray(workload.grain_shape, dtype=np.int32)
        gg = np.ascontiguousarray(workload.grain_geom, dtype=np.float64)
        n = c_int64()
        _check(L.pd_mesh_grains(ctx, len(workload.shapes), _ptr(sls), _ptr(lvs), _ptr(vtx), workload.n_grains,
                                _ptr(gs), _ptr(gg), ctypes.byref(n)))
        self.N = n.value
        nb = c_int64()
        _check(L.pd_build_bonds(ctx, ctypes.byref(nb)))
        self.n_bonds = nb.value
        agg = getattr(workload, "grain_agg", None)
        if agg is not None:
            ga = np.ascontiguousarray(agg, dtype=np.int32)
            walls = np.ascontiguousarray(workload.agg_walls, dtype=np.float64).reshape(-1)
            _check(L.pd_set_aggregates(ctx, int(walls.size // 8), _ptr(ga), _ptr(walls)))
        mats = getattr(workload, "materials", None)
        if mats is not None:
            props = np.ascontiguousarray(mats[0], dtype=np.float64).reshape(-1)
            gm = np.ascontiguousarray(mats[1], dtype=np.int32)
            _check(L.pd_set_materials(ctx, int(props.size // 4), _ptr(props), _ptr(gm)))
        self.surrogate_basis = None
        if surrogate is not None:
            # surrogate = dict(basis=..., lambda_=..., n_modes=, judge_every=, gate=, err_tol=) or a callable
            cfg = surrogate(self) if callable(surrogate) else surrogate
            basis = np.ascontiguousarray(cfg["basis"], dtype=np.float32)
            lam = np.ascontiguousarray(cfg["lambda_"], dtype=np.float32)
            _check(L.pd_surrogate_setup(ctx, int(cfg["n_modes"]), _ptr(basis), _ptr(lam), int(cfg.get("judge_every", 50)),
                                        float(cfg.get("gate", 0.5)), float(cfg.get("err_tol", 1e-3))))
            self.surrogate_basis = cfg
        if device is not None:
            self.bind()

    # -- lifecycle ----------------------------------------------------------
    def bind(self):
        import torch
        L = load()
        nbytes = c_size_t()
        _check(L.pd_arena_bytes(self._ctx, ctypes.byref(nbytes)))
        with torch.cuda.stream(self._stream):
            self._arena = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        base = self._arena.data_ptr()
        aligned = (base + 255) & ~255
        _check(L.pd_bind_arena(self._ctx, c_void_p(aligned), nbytes.value))
        self.arena_bytes = int(nbytes.value)

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            load().pd_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping -------------------------------------------------------------
    def step(self, n: int = 1):
        _check(load().pd_step(self._ctx, int(n)))

    def eval_forces(self):
        _check(load().pd_eval_forces(self._ctx))

    # -- state access -----------------------------------------------------------
    _SHAPES = {
        "X": (np.float64, 2), "DISP": (np.float64, 2), "VEL": (np.float64, 2), "ACC": (np.float64, 2),
        "POS": (np.float64, 2), "FORCE": (np.float64, 2), "FORCE_PARTS": (np.float64, 8),
        "DAMAGE": (np.float64, 1), "GRAIN": (np.int32, 1), "VOLUME": (np.float64, 1),
        "LATTICE": (np.int32, 2),
    }

    def _alloc(self, field):
        if field in self._SHAPES:
            dt, k = self._SHAPES[field]
            shape = (self.N, 2) if k == 2 else ((4, self.N, 2) if k == 8 else (self.N,))
            return np.zeros(shape, dtype=dt)
        if field == "BROKEN":
            return np.zeros(self.n_bonds, dtype=np.uint8)
        if field == "ROW_PTR":
            return np.zeros(self.N + 1, dtype=np.int32)
        if field == "COL":
            return np.zeros(self.n_bonds, dtype=np.int32)
        if field == "STEP":
            return np.zeros(1, dtype=np.int64)
        if field == "GRAIN_TEMPLATE":
            return np.zeros(self.workload.n_grains, dtype=np.int32)
        raise KeyError(field)

    def get(self, field: str) -> np.ndarray:
        """Host copy of a state field (waits for the stream)."""
        out = self._alloc(field)
        _check(load().pd_get_state(self._ctx, FIELDS[field], _ptr(out) if out.nbytes else None, out.nbytes, 0))
        return out

    def get_device(self, field: str, out):
        """Stream-ordered device-to-device copy into a torch tensor ``out``."""
        _check(load().pd_get_state(self._ctx, FIELDS[field], c_void_p(out.data_ptr()),
                                   out.numel() * out.element_size(), 1))
        return out

    def set(self, field: str, value) -> None:
        if hasattr(value, "data_ptr"):
            if getattr(value, "is_cuda", True):
                _check(load().pd_set_state(self._ctx, FIELDS[field], c_void_p(value.data_ptr()),
                                           value.numel() * value.element_size(), PD_MEM_DEVICE))
                return
            if value.is_pinned():
                # page-locked host tensor: enqueued on the stream without waiting
                _check(load().pd_set_state(self._ctx, FIELDS[field], c_void_p(value.data_ptr()),
                                           value.numel() * value.element_size(), PD_MEM_HOST_ASYNC))
                return
            value = value.numpy()
        ref = self._alloc(field)
        arr = np.ascontiguousarray(np.asarray(value, dtype=ref.dtype).reshape(ref.shape))
        _check(load().pd_set_state(self._ctx, FIELDS[field], _ptr(arr), arr.nbytes, 0))

    def diagnostics(self) -> dict:
        out = np.zeros(DIAG_COUNT)
        _check(load().pd_diagnostics(self._ctx, _ptr(out)))
        d = dict(zip(DIAG_NAMES, out[: len(DIAG_NAMES)]))
        d["n_broken"] = int(d["n_broken"])
        return d

    def observables(self) -> np.ndarray:
        """Per aggregate: volume fraction, bulk damage, y force on the top wall,
        y force on the bottom wall (pd_observables)."""
        n_agg = int(self.info()["n_agg"])
        out = np.zeros((n_agg, 4))
        _check(load().pd_observables(self._ctx, _ptr(out)))
        return out

    def status(self):
        out = np.zeros(STATUS_COUNT, dtype=np.int32)
        rc = load().pd_status(self._ctx, _ptr(out))
        return rc, out

    def clear_status(self):
        """Zero the status words and the grid barrier; the next step rebuilds the
        contact candidate lists (pd_clear_status)."""
        _check(load().pd_clear_status(self._ctx))

    def set_wait_test(self, withhold_block: int = -1, max_spins: int = 0):
        """Test hook of the persistent kernel's bounded barrier waits (pd_set_wait_test)."""
        _check(load().pd_set_wait_test(self._ctx, int(withhold_block), int(max_spins)))

    def set_timing(self, enable: bool):
        _check(load().pd_set_timing(self._ctx, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """Milliseconds of the kernel groups of the last timed step."""
        out = np.zeros(4)
        _check(load().pd_kernel_times(self._ctx, _ptr(out)))
        return dict(predict=out[0], bin=out[1], force=out[2], step=out[3])

    def info(self) -> dict:
        out = np.zeros(15)
        _check(load().pd_info(self._ctx, _ptr(out)))
        keys = ("N", "n_bonds", "G", "h_min", "Rc", "Kn", "dt", "steps", "max_row", "buckets", "mode", "lanes",
                "block", "n_agg", "n_templates")
        return dict(zip(keys, out))

    # -- learned modal surrogate ---------------------------------------------------
    def surrogate_set_mlp(self, tmpl: int, mlp):
        self._mlps = getattr(self, "_mlps", {})
        self._mlps[tmpl] = mlp           # keep the network alive while the context uses it
        _check(load().pd_surrogate_set_mlp(self._ctx, int(tmpl), mlp._h if mlp is not None else None))

    def surrogate_enable(self, on: bool = True):
        _check(load().pd_surrogate_enable(self._ctx, 1 if on else 0))

    def surrogate_sample(self):
        M = int(self.surrogate_basis["n_modes"])
        G = self.workload.n_grains
        q = np.zeros((G, M), dtype=np.float32)
        f = np.zeros((G, M), dtype=np.float32)
        _check(load().pd_surrogate_sample(self._ctx, _ptr(q), _ptr(f)))
        return q, f

    def surrogate_stats(self):
        """Per grain: active flag, judged nodal error, judged modal error, judged max |s|/s0."""
        G = self.workload.n_grains
        a = np.zeros(G, dtype=np.int32)
        e = np.zeros(G, dtype=np.float32)
        me = np.zeros(G, dtype=np.float32)
        m = np.zeros(G, dtype=np.float32)
        _check(load().pd_surrogate_stats(self._ctx, _ptr(a), _ptr(e), _ptr(me), _ptr(m)))
        return a, e, me, m

    def surrogate_inspect(self):
        """Network input q and modal force f of every grain at the current state."""
        M = int(self.surrogate_basis["n_modes"])
        G = self.workload.n_grains
        q = np.zeros((G, M), dtype=np.float32)
        y = np.zeros((G, M), dtype=np.float32)
        _check(load().pd_surrogate_inspect(self._ctx, _ptr(q), _ptr(y)))
        return q, y

    def set_path(self, mode: int, lanes: int = 8, block: int = 128):
        """0 = graph of separate kernels, 1 = persistent cooperative kernel."""
        _check(load().pd_set_path(self._ctx, int(mode), int(lanes), int(block)))

    def autotune(self) -> dict:
        """Time the candidate step paths on the current state and keep the fastest."""
        out = np.zeros(4)
        _check(load().pd_autotune(self._ctx, _ptr(out)))
        return dict(mode=int(out[0]), lanes=int(out[1]), block=int(out[2]), ms_per_step=float(out[3]))


MLP_NPARAMS = 24864


class MLP:
    """The surrogate network (32 -> 128 -> 128 -> 32, GELU) on the tensor cores.

    Device arena and stream from PyTorch; inputs and outputs are CUDA float32
    tensors of shape (batch, 32)."""

    def __init__(self, max_batch: int, device="cuda:0", stream=None, params=None):
        import torch
        L = load()
        self.device = torch.device(device)
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = c_void_p()
        _check(L.pd_mlp_create(ctypes.byref(h), int(max_batch), c_void_p(self._stream.cuda_stream)))
        self._h = h
        self.max_batch = int(max_batch)
        nbytes = c_size_t()
        _check(L.pd_mlp_arena_bytes(h, ctypes.byref(nbytes)))
        self._arena = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        aligned = (self._arena.data_ptr() + 255) & ~255
        _check(L.pd_mlp_bind_arena(h, c_void_p(aligned), nbytes.value))
        if params is not None:
            self.set_params(params)

    def set_params(self, flat):
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32).reshape(-1))
        assert a.size == MLP_NPARAMS
        _check(load().pd_mlp_set_params(self._h, _ptr(a)))

    def get_params(self) -> np.ndarray:
        a = np.zeros(MLP_NPARAMS, dtype=np.float32)
        _check(load().pd_mlp_get_params(self._h, _ptr(a)))
        return a

    def forward(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty((x.shape[0], 32), dtype=torch.float32, device=self.device)
        _check(load().pd_mlp_forward(self._h, c_void_p(x.data_ptr()), c_void_p(y.data_ptr()), int(x.shape[0])))
        return y

    def loss_grad(self, x, t):
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(MLP_NPARAMS, dtype=np.float32)
        _check(load().pd_mlp_loss_grad(self._h, c_void_p(x.data_ptr()), c_void_p(t.data_ptr()), int(x.shape[0]),
                                       _ptr(loss), _ptr(g)))
        return float(loss[0]), g

    def train_step(self, x, t, lr: float) -> float:
        loss = np.zeros(1, dtype=np.float32)
        _check(load().pd_mlp_train_step(self._h, c_void_p(x.data_ptr()), c_void_p(t.data_ptr()), int(x.shape[0]),
                                        ctypes.c_float(lr), _ptr(loss)))
        return float(loss[0])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
