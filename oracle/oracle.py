"""ctypes front end of the FP64 CPU oracle (``peridem_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg.  Nothing here is used by the GPU library.

The oracle meshes every grain on its own lattice, builds the reference
neighbour lists with the exact segment-in-domain definition of the non-convex
horizon (Sec. 4, set C_x), and runs Algorithm 1 (velocity Verlet) with the
force laws of Secs. 3-4.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "peridem_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libperidem_oracle.so")
# the same source built with -fopenmp: the node loop of the force evaluation and
# the update loops split over the host cores (same arithmetic per node)
_LIB_OMP = os.path.join(_LIBDIR, "libperidem_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

# parameter-vector slots (mirror of the enum in peridem_oracle.c)
P_RHO, P_KN, P_RC, P_RD, P_MU, P_GX, P_GY, P_DT = range(8)
P_WX0, P_WX1, P_WY0, P_WY1, P_VX0, P_VX1, P_VY0, P_VY1 = range(8, 16)
P_MICRO, P_SEARCH, P_PE5, P_NPARAM = 16, 17, 18, 19

MESH_CLEARANCE = 1e-6      # nodes closer than this * h to the boundary are dropped
SEGMENT_TOL = 1e-10        # closed-domain tolerance of the visibility test, * h


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, plain -O2): the
    single-threaded library and the all-core (-fopenmp) one."""
    os.makedirs(_LIBDIR, exist_ok=True)
    for path, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, path)
    return _LIB


def threads_available() -> int:
    """Host threads the all-core build uses (OMP_NUM_THREADS, else the cores)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit():
        return int(env)
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def lib(omp: bool = False):
    with _lock:
        if omp not in _libs:
            build()
            L = ctypes.CDLL(_LIB_OMP if omp else _LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_ubyte)
            c_d, c_i, c_l = ctypes.c_double, ctypes.c_int, ctypes.c_long
            L.or_mesh_grain.argtypes = [dp, ip, c_i, c_d, c_d, c_d, c_d, c_d, c_d, c_i, dp, ip]
            L.or_mesh_grain.restype = c_i
            L.or_segment_in_domain.argtypes = [c_d, c_d, c_d, c_d, dp, ip, c_i, c_d, c_d]
            L.or_segment_in_domain.restype = c_i
            L.or_grain_bonds.argtypes = [dp, ip, c_i, c_d, c_d, c_d, c_d, c_i, ip, ip, ip, c_i]
            L.or_grain_bonds.restype = c_i
            L.or_bond_constants.argtypes = [c_d, c_d, c_d, c_d, c_i, dp, dp]
            L.or_contact_stiffness.argtypes = [c_d, c_d]
            L.or_contact_stiffness.restype = c_d
            L.or_wall_segment.argtypes = [c_d, c_d, dp, dp]
            L.or_corner_region.argtypes = [c_d, c_d, c_d, dp, dp, dp]
            L.or_forces.argtypes = [dp, c_d, c_i, dp, dp, dp, dp, ip, dp, dp, dp, dp, ip, ip, up, dp, dp, ip]
            L.or_run.argtypes = [dp, c_l, c_i, c_i, dp, dp, dp, dp, dp, ip, dp, dp, dp, dp, ip, ip, up, dp, dp,
                                 ip]
            L.or_init_accel.argtypes = [dp, c_d, c_i, dp, dp, dp, dp, dp, ip, dp, dp, dp, dp, ip, ip, up, ip]
            L.or_diagnostics.argtypes = [dp, c_i, dp, dp, dp, dp, ip, dp, dp, dp, ip, ip, up, dp]
            L.or_wall_sums.argtypes = [dp, c_d, c_i, dp, dp, dp, dp, ip, dp, dp]
            L.or_wall_segment_energy.argtypes = [c_d, c_d]
            L.or_wall_segment_energy.restype = c_d
            L.or_energies.argtypes = [dp, c_d, c_i, dp, dp, dp, ip, dp, dp, ip, ip, up, dp]
            _libs[omp] = L
    return _libs[omp]


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _dp(a):
    return _p(a, ctypes.c_double)


def _dpn(a):
    """Double pointer, or NULL for None."""
    return None if a is None else _dp(a)


def _ip(a):
    return _p(a, ctypes.c_int)


def _up(a):
    return _p(a, ctypes.c_ubyte)


# ---------------------------------------------------------------------------
# closed-form helpers exposed for pinning


def bond_constants(E, nu, Gc, eps, micromodulus=0):
    cw, s0 = ctypes.c_double(), ctypes.c_double()
    lib().or_bond_constants(E, nu, Gc, eps, micromodulus, ctypes.byref(cw), ctypes.byref(s0))
    return cw.value, s0.value


def contact_stiffness(k_bulk, eps):
    return lib().or_contact_stiffness(k_bulk, eps)


def wall_segment(d, Rc):
    A, c = ctypes.c_double(), ctypes.c_double()
    lib().or_wall_segment(d, Rc, ctypes.byref(A), ctypes.byref(c))
    return A.value, c.value


def corner_region(di, dj, Rc):
    A, Ix, Iy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_corner_region(di, dj, Rc, ctypes.byref(A), ctypes.byref(Ix), ctypes.byref(Iy))
    return A.value, Ix.value, Iy.value


def wall_segment_energy(d, Rc):
    """R_c^4 J(theta): the single-wall contact potential of Sec. 4.5 per unit K_n V_x."""
    return lib().or_wall_segment_energy(d, Rc)


def _loops_arrays(loops):
    xy = np.ascontiguousarray(np.vstack([np.asarray(l, dtype=np.float64) for l in loops]).reshape(-1))
    ls = np.zeros(len(loops) + 1, dtype=np.int32)
    for k, l in enumerate(loops):
        ls[k + 1] = ls[k] + len(l)
    return xy, ls


def segment_in_domain(a, b, loops, scale=1.0, tol=0.0):
    xy, ls = _loops_arrays(loops)
    return bool(lib().or_segment_in_domain(a[0], a[1], b[0], b[1], _dp(xy), _ip(ls), len(loops), scale, tol))


def mesh_grain(loops, R, h, cx=0.0, cy=0.0, theta=0.0, clear=MESH_CLEARANCE):
    xy, ls = _loops_arrays(loops)
    L = lib()
    n = L.or_mesh_grain(_dp(xy), _ip(ls), len(loops), R, h, cx, cy, theta, clear, 0, None, None)
    X = np.zeros((max(n, 1), 2))
    lat = np.zeros((max(n, 1), 2), dtype=np.int32)
    L.or_mesh_grain(_dp(xy), _ip(ls), len(loops), R, h, cx, cy, theta, clear, n, _dp(X), _ip(lat))
    return X[:n], lat[:n]


def grain_bonds(loops, R, h, lat, horizon_ratio=3.0, tol=SEGMENT_TOL):
    xy, ls = _loops_arrays(loops)
    n = lat.shape[0]
    lat = np.ascontiguousarray(lat, dtype=np.int32)
    row = np.zeros(n + 1, dtype=np.int32)
    cap = 64 * max(n, 1)
    col = np.zeros(cap, dtype=np.int32)
    nb = lib().or_grain_bonds(_dp(xy), _ip(ls), len(loops), R, h, horizon_ratio, tol, n, _ip(lat),
                              _ip(row), _ip(col), cap)
    assert nb <= cap
    return row, col[:nb].copy()


# ---------------------------------------------------------------------------
# whole problems


def param_vector(params: dict, h_min: float, search_grid: bool = True) -> np.ndarray:
    """Oracle parameter vector; R_c = rc_ratio h_min, K_n from eps_c = horizon_ratio h_min."""
    prm = np.zeros(P_NPARAM)
    prm[P_RHO] = params["rho"]
    prm[P_RC] = params["rc_ratio"] * h_min
    prm[P_KN] = contact_stiffness(params["k_bulk"], params["horizon_ratio"] * h_min)
    prm[P_RD] = params["damping_ratio"]
    prm[P_MU] = params["friction"]
    prm[P_GX], prm[P_GY] = params["gx"], params["gy"]
    prm[P_DT] = params["dt"]
    prm[P_WX0], prm[P_WY0] = params["wall_lo"]
    prm[P_WX1], prm[P_WY1] = params["wall_hi"]
    prm[P_VX0], prm[P_VY0] = params["wall_vel_lo"]
    prm[P_VX1], prm[P_VY1] = params["wall_vel_hi"]
    prm[P_MICRO] = params["micromodulus"]
    prm[P_SEARCH] = 1.0 if search_grid else 0.0
    eps_c = params["horizon_ratio"] * h_min
    prm[P_PE5] = math.pi * eps_c * eps_c * eps_c * eps_c * eps_c     # K_n = 18 k / (pi eps_c^5)
    return prm


class OracleProblem:
    """Nodes, bonds and state of one problem; see :meth:`from_workload`.

    X (N,2) reference positions, V (N,) volumes, grain (N,) grain ids,
    row_ptr/col the CSR reference neighbour lists (ascending columns),
    g_cw/g_s0/g_eps per-grain bond constants, prm the parameter vector,
    g_mat (G,2) per-grain (density, bulk modulus) or None (one material: prm).
    """

    omp = False     # True: time steps and force evaluations run in the all-core build

    def __init__(self, X, V, grain, row_ptr, col, g_cw, g_s0, g_eps, prm, v0=None, g_mat=None):
        self.X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 2)
        self.N = self.X.shape[0]
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.grain = np.ascontiguousarray(grain, dtype=np.int32)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        if self.col.size == 0:
            self.col = np.zeros(1, dtype=np.int32)[:0]
        self.g_cw = np.ascontiguousarray(g_cw, dtype=np.float64)
        self.g_s0 = np.ascontiguousarray(g_s0, dtype=np.float64)
        self.g_eps = np.ascontiguousarray(g_eps, dtype=np.float64)
        self.prm = np.ascontiguousarray(prm, dtype=np.float64)
        self.g_mat = None if g_mat is None else np.ascontiguousarray(g_mat, dtype=np.float64).reshape(-1, 2)
        self.broken = np.zeros(max(len(self.col), 1), dtype=np.uint8)
        self.u = np.zeros((self.N, 2))
        self.v = np.zeros((self.N, 2)) if v0 is None else np.array(v0, dtype=np.float64).reshape(-1, 2)
        self.a = np.zeros((self.N, 2))
        self.step = 0
        self.status = np.zeros(3, dtype=np.int32)

    @classmethod
    def from_workload(cls, w, search_grid: bool = True):
        p = w.params
        Xs, lats, grains, Vs, rows, cols = [], [], [], [], [], []
        g_cw = np.zeros(w.n_grains)
        g_s0 = np.zeros(w.n_grains)
        g_eps = np.zeros(w.n_grains)
        grain_start = np.zeros(w.n_grains + 1, dtype=np.int64)
        # materials (E, k_bulk, rho, Gc) per grain; the workload's params are material 0
        mats = getattr(w, "materials", None)
        if mats is not None:
            props, gmat = np.asarray(mats[0], dtype=np.float64).reshape(-1, 4), np.asarray(mats[1])
        else:
            props = np.array([[p["E"], p["k_bulk"], p["rho"], p["Gc"]]])
            gmat = np.zeros(w.n_grains, dtype=np.int64)
        node0 = 0
        bond0 = 0
        vel = []
        for g in range(w.n_grains):
            cx, cy, R, th, vx, vy, h = w.grain_geom[g]
            loops = w.shapes[w.grain_shape[g]]
            X, lat = mesh_grain(loops, R, h, cx, cy, th)
            row, col = grain_bonds(loops, R, h, lat, p["horizon_ratio"])
            n = X.shape[0]
            Xs.append(X)
            lats.append(lat)
            grains.append(np.full(n, g, dtype=np.int32))
            Vs.append(np.full(n, h * h))
            rows.append(row[:-1] + bond0)
            cols.append(col + node0)
            vel.append(np.tile([vx, vy], (n, 1)))
            eps = p["horizon_ratio"] * h
            g_eps[g] = eps
            E_g, Gc_g = props[gmat[g], 0], props[gmat[g], 3]
            g_cw[g], g_s0[g] = bond_constants(E_g, p["nu"], Gc_g, eps, int(p["micromodulus"]))
            node0 += n
            bond0 += len(col)
            grain_start[g + 1] = node0
        h_min = float(np.min(w.grain_geom[:, 6]))
        prm = param_vector(p, h_min, search_grid)
        g_mat = np.stack([props[gmat, 2], props[gmat, 1]], 1) if mats is not None else None
        self = cls(np.vstack(Xs), np.concatenate(Vs), np.concatenate(grains),
                   np.concatenate(rows + [np.array([bond0], dtype=np.int32)]),
                   np.concatenate(cols), g_cw, g_s0, g_eps, prm, np.vstack(vel), g_mat)
        self.w = w
        self.lat = np.vstack(lats)
        self.grain_start = grain_start
        self.h_min = h_min
        return self

    # -- internals ---------------------------------------------------------
    def _sys(self):
        return (self.N, _dp(self.X), _dp(self.u), _dp(self.v))

    def init_accel(self):
        """a^0 from the forces of the initial state (first line of Algorithm 1)."""
        L = lib(self.omp)
        L.or_init_accel(_dp(self.prm), self.step * self.prm[P_DT], self.N, _dp(self.X), _dp(self.u),
                        _dp(self.v), _dp(self.a), _dp(self.V), _ip(self.grain), _dp(self.g_cw),
                        _dp(self.g_s0), _dp(self.g_eps), _dpn(self.g_mat), _ip(self.row_ptr), _ip(self.col),
                        _up(self.broken), _ip(self.status))
        return self

    def run(self, n_steps: int, want_parts: bool = False):
        """Advance n_steps; returns (F_last, parts_last) of the final step."""
        L = lib(self.omp)
        F = np.zeros((self.N, 2))
        parts = np.zeros((4, self.N, 2)) if want_parts else None
        L.or_run(_dp(self.prm), self.step, n_steps, self.N, _dp(self.X), _dp(self.u), _dp(self.v),
                 _dp(self.a), _dp(self.V), _ip(self.grain), _dp(self.g_cw), _dp(self.g_s0),
                 _dp(self.g_eps), _dpn(self.g_mat), _ip(self.row_ptr), _ip(self.col), _up(self.broken),
                 _dp(F), _dp(parts) if parts is not None else None, _ip(self.status))
        self.step += n_steps
        return F, parts

    def forces(self, t=None, keep_broken=True):
        """Force evaluation at the current state; returns (F, parts[4,N,2])."""
        L = lib(self.omp)
        if t is None:
            t = self.step * self.prm[P_DT]
        F = np.zeros((self.N, 2))
        parts = np.zeros((4, self.N, 2))
        br = self.broken.copy() if keep_broken else self.broken
        L.or_forces(_dp(self.prm), t, self.N, _dp(self.X), _dp(self.u), _dp(self.v), _dp(self.V),
                    _ip(self.grain), _dp(self.g_cw), _dp(self.g_s0), _dp(self.g_eps), _dpn(self.g_mat),
                    _ip(self.row_ptr), _ip(self.col), _up(br), _dp(F), _dp(parts), _ip(self.status))
        return F, parts

    def diagnostics(self):
        out = np.zeros(7)
        lib().or_diagnostics(_dp(self.prm), self.N, _dp(self.X), _dp(self.u), _dp(self.v), _dp(self.V),
                             _ip(self.grain), _dp(self.g_cw), _dp(self.g_eps), _dpn(self.g_mat),
                             _ip(self.row_ptr), _ip(self.col), _up(self.broken), _dp(out))
        return dict(KE=out[0], E_bond=out[1], E_contact=out[2], Px=out[3], Py=out[4], Lz=out[5],
                    n_broken=int(out[6]))

    def energies(self, t=None):
        """Potential energies of the contact laws at the current state (walls at
        time t, default now): E_contact (inter-grain), E_self (self-contact),
        E_wall (single-wall segments)."""
        if t is None:
            t = self.step * self.prm[P_DT]
        out = np.zeros(3)
        lib().or_energies(_dp(self.prm), t, self.N, _dp(self.X), _dp(self.u), _dp(self.V), _ip(self.grain),
                          _dp(self.g_cw), _dpn(self.g_mat), _ip(self.row_ptr), _ip(self.col), _up(self.broken),
                          _dp(out))
        return dict(E_contact=out[0], E_self=out[1], E_wall=out[2])

    @property
    def positions(self):
        return self.X + self.u

    def damage(self):
        """Per-node damage: broken / reference bonds (Sec. 3.1)."""
        cnt = np.diff(self.row_ptr)
        csum = np.concatenate([[0], np.cumsum(self.broken.astype(np.int64))])
        br = csum[self.row_ptr[1:]] - csum[self.row_ptr[:-1]]
        return np.where(cnt > 0, br / np.maximum(cnt, 1), 0.0)

    # -- observables of the settling and compaction sections (Sec. 6) -------
    def walls(self, t=None):
        """Wall positions x_lo, x_hi, y_lo, y_hi at time t (default: now)."""
        if t is None:
            t = self.step * self.prm[P_DT]
        return np.array([self.prm[P_WX0 + l] + self.prm[P_VX0 + l] * t for l in range(4)])

    def volume_fraction(self, t=None):
        """phi(t) = sum of particle volumes / (container width x height)."""
        w = self.walls(t)
        return float(self.V.sum() / ((w[1] - w[0]) * (w[3] - w[2])))

    def particle_damage(self):
        """Mean node damage of every grain."""
        dmg = self.damage()
        G = int(self.grain.max()) + 1
        return np.bincount(self.grain, weights=dmg, minlength=G) / np.bincount(self.grain, minlength=G)

    def bulk_damage(self):
        """Average particle damage over all particles."""
        return float(self.particle_damage().mean())

    def wall_sums(self, t=None):
        """Sums over nodes of each wall's own term (4 x 2) and of the corner
        terms (4 x 2) that eq:wall-total subtracts."""
        if t is None:
            t = self.step * self.prm[P_DT]
        out = np.zeros(16)
        lib().or_wall_sums(_dp(self.prm), t, self.N, _dp(self.X), _dp(self.u), _dp(self.v), _dp(self.V),
                           _ip(self.grain), _dpn(self.g_mat), _dp(out))
        return out[:8].reshape(4, 2), out[8:].reshape(4, 2)

    def wall_reaction(self, wall, t=None):
        """Force the aggregate exerts on wall l (x_lo, x_hi, y_lo, y_hi): minus the
        force of that wall on the nodes, its own term less half of each corner
        term it shares (a corner region belongs to two walls)."""
        single, corner = self.wall_sums(t)
        shares = {0: (0, 1), 1: (2, 3), 2: (0, 2), 3: (1, 3)}[wall]   # corners (x_lo,y_lo),(x_lo,y_hi),(x_hi,y_lo),(x_hi,y_hi)
        f = single[wall] - 0.5 * (corner[shares[0]] + corner[shares[1]])
        return -f
