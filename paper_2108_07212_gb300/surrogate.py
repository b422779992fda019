"""Set-up and training of the learned per-grain modal surrogate.

Per bond-network template (grains of one shape meshed at the same h/R) the
basis is the n_modes softest non-rigid eigenvectors of the template's
dimensionless linearised bond operator K/E, and ``lambda_`` their eigenvalues;
the library assembles the operator from its own bond constants and solves for
them (pd_surrogate_basis).  The network of a template learns the
nonlinear part of the modal bond force, f - (-lambda q), from training pairs
that the simulation itself produces (:func:`collect_samples`), and is trained
on the GPU by the library's own forward/backward kernels (:class:`~.binding.MLP`).
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B


def build_basis(sim: "B.Simulation", n_modes: int = 32, judge_every: int = 50, gate: float = 0.5,
                err_tol: float = 1e-3, source: tuple | None = None) -> dict:
    """Basis and modal stiffness of every template of a meshed (unbound) simulation.

    ``source = (sim_src, cfg_src)`` reuses the basis of every template that the
    source simulation shares (same :func:`template_keys`), so that networks
    trained on the source's snapshots see the same modal coordinates (the
    eigenvectors of repeated eigenvalues are not unique)."""
    tmpl = sim.get("GRAIN_TEMPLATE")
    grain = sim.get("GRAIN")
    lat = sim.get("LATTICE")
    row = sim.get("ROW_PTR")
    col = sim.get("COL")
    starts = np.searchsorted(grain, np.arange(sim.workload.n_grains + 1))
    reuse = {}
    if source is not None:
        sim_src, cfg_src = source
        offs = np.concatenate([[0], np.cumsum([2 * d["nodes"] * n_modes for d in cfg_src["templates"]])])
        lam_src = cfg_src["lambda_"].reshape(-1, n_modes)
        for ts, key in enumerate(template_keys(sim_src, cfg_src)):
            reuse[key] = (cfg_src["basis"][offs[ts]:offs[ts + 1]], lam_src[ts], cfg_src["templates"][ts])
    my_keys = template_keys(sim, dict(template_of_grain=tmpl, templates=[
        dict(nodes=int(starts[int(np.argmax(tmpl == t)) + 1] - starts[int(np.argmax(tmpl == t))]))
        for t in range(int(tmpl.max()) + 1)])) if reuse else None
    # every template's basis from the library (pd_surrogate_basis); templates
    # shared with the source simulation keep the source's
    import ctypes
    L = B.load()
    n_t = int(tmpl.max()) + 1
    need = ctypes.c_size_t(0)
    B._check(L.pd_surrogate_basis(sim._ctx, n_modes, None, ctypes.byref(need), None, None))
    lib_basis = np.zeros(int(need.value), dtype=np.float32)
    lib_lam = np.zeros(n_t * n_modes, dtype=np.float32)
    rigid = np.zeros(3 * n_t)
    B._check(L.pd_surrogate_basis(sim._ctx, n_modes, B._ptr(lib_basis), ctypes.byref(need), B._ptr(lib_lam),
                                  B._ptr(rigid)))
    bases, lams, info = [], [], []
    off = 0
    for t in range(n_t):
        g = int(np.argmax(tmpl == t))
        n = int(starts[g + 1] - starts[g])
        piece = lib_basis[off:off + 2 * n * n_modes]
        off += 2 * n * n_modes
        if reuse and my_keys[t] in reuse:
            b, l, d = reuse[my_keys[t]]
            bases.append(np.asarray(b, dtype=np.float64))
            lams.append(np.asarray(l, dtype=np.float64))
            info.append(dict(d, template=t))
            continue
        bases.append(piece.astype(np.float64))
        lams.append(lib_lam[t * n_modes:(t + 1) * n_modes].astype(np.float64))
        info.append(dict(template=t, nodes=n, rigid=rigid[3 * t:3 * t + 3].tolist(),
                         first=float(lib_lam[t * n_modes])))
    return dict(basis=np.concatenate(bases).astype(np.float32), lambda_=np.concatenate(lams).astype(np.float32),
                n_modes=n_modes, judge_every=judge_every, gate=gate, err_tol=err_tol, templates=info,
                template_of_grain=tmpl)


def template_keys(sim: "B.Simulation", cfg: dict) -> list:
    """A key per template that is equal for equal templates of different
    simulations: node count, bond count and the grain shape's outline."""
    import hashlib
    tmpl = cfg["template_of_grain"]
    row = sim.get("ROW_PTR")
    grain = sim.get("GRAIN")
    starts = np.searchsorted(grain, np.arange(sim.workload.n_grains + 1))
    keys = []
    for t, d in enumerate(cfg["templates"]):
        g = int(np.argmax(tmpl == t))
        loops = sim.workload.shapes[int(sim.workload.grain_shape[g])]
        hsh = hashlib.sha1(b"".join(np.ascontiguousarray(l, dtype=np.float64).tobytes() for l in loops)).hexdigest()
        keys.append((int(d["nodes"]), int(row[starts[g + 1]] - row[starts[g]]), hsh))
    return keys


def modal_field(sim: "B.Simulation", cfg: dict, coeffs: np.ndarray) -> np.ndarray:
    """World-frame nodal field sum_m coeffs[g, m] Phi_m h of every templated grain
    (rotated by the grain's orientation; zero on grains without a template):
    a deformation (DISP) with modal coefficients q = coeffs."""
    tmpl = cfg["template_of_grain"]
    M = cfg["n_modes"]
    grain = sim.get("GRAIN")
    starts = np.searchsorted(grain, np.arange(sim.workload.n_grains + 1))
    offs = np.concatenate([[0], np.cumsum([2 * d["nodes"] * M for d in cfg["templates"]])])
    out = np.zeros((sim.N, 2))
    for g in range(sim.workload.n_grains):
        t = int(tmpl[g])
        if t < 0:
            continue
        n = int(starts[g + 1] - starts[g])
        Phi = cfg["basis"][offs[t]:offs[t + 1]].astype(np.float64).reshape(n, 2, M)
        wl = Phi @ coeffs[g] * sim.workload.grain_geom[g, 6]
        th = sim.workload.grain_geom[g, 3]
        c, s = math.cos(th), math.sin(th)
        out[starts[g]:starts[g + 1], 0] = c * wl[:, 0] - s * wl[:, 1]
        out[starts[g]:starts[g + 1], 1] = s * wl[:, 0] + c * wl[:, 1]
    return out


def collect_samples(sim: "B.Simulation", steps: int, every: int) -> dict:
    """Run ``steps`` steps, sampling (q, f_full) of every templated grain every
    ``every`` steps; returns {template: (q[n, M], f[n, M])}."""
    tmpl = sim.surrogate_basis["template_of_grain"]
    out = {}
    for _ in range(steps // every):
        sim.step(every)
        q, f = sim.surrogate_sample()
        for t in np.unique(tmpl):
            sel = tmpl == t
            out.setdefault(int(t), []).append((q[sel], f[sel]))
    return {t: (np.vstack([a for a, _ in v]), np.vstack([b for _, b in v])) for t, v in out.items()}


def residual_targets(q: np.ndarray, f: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """What the network learns: f - (-lambda q)."""
    return f + lam[None, :] * q


def _unpack(flat):
    o = 0
    out = []
    for shape in ((128, 32), (128,), (128, 128), (128,), (32, 128), (32,)):
        n = int(np.prod(shape))
        out.append(np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    return out


def _pack(parts):
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def fold_scaling(params, mu_in, sd_in, sd_out):
    """Parameters of a network trained on standardised data, rewritten to act on
    raw inputs and produce raw outputs (exact for the affine first/last layers)."""
    W1, b1, W2, b2, W3, b3 = _unpack(params)
    W1f = W1 / sd_in[None, :]
    b1f = b1 - W1f @ mu_in
    W3f = W3 * sd_out[:, None]
    b3f = b3 * sd_out
    return _pack([W1f, b1f, W2, b2, W3f, b3f])


def init_params(seed: int = 0) -> np.ndarray:
    """He initialisation with a zero last layer: an untrained network adds no
    correction, so the surrogate starts as the linear modal model."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2.0 / 32), (128, 32))
    W2 = rng.normal(0, math.sqrt(2.0 / 128), (128, 128))
    return _pack([W1, np.zeros(128), W2, np.zeros(128), np.zeros((32, 128)), np.zeros(32)])


def train_template(q: np.ndarray, f: np.ndarray, lam: np.ndarray, epochs: int = 400, lr: float = 2e-3,
                   batch: int = 1024, seed: int = 0, device="cuda:0"):
    """Train one template's network on the GPU; returns (raw-unit parameters, losses)."""
    import torch
    y = residual_targets(q, f, lam)
    mu_in = q.mean(axis=0)
    # input scales floored at 1e-3 h: snapshots with almost no deformation must
    # not turn into a network that amplifies every later input
    sd_in = np.maximum(q.std(axis=0), 1e-3)
    sd_out = np.maximum(np.abs(y).std(axis=0), 1e-12)
    xs = ((q - mu_in) / sd_in).astype(np.float32)
    ys = (y / sd_out).astype(np.float32)
    n = xs.shape[0]
    bsz = min(batch, n)
    net = B.MLP(max_batch=bsz, device=device, params=init_params(seed))
    X = torch.from_numpy(xs).to(device)
    Y = torch.from_numpy(ys).to(device)
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        idx = torch.from_numpy(rng.choice(n, size=bsz, replace=False)).to(device)
        losses.append(net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr))
    return fold_scaling(net.get_params(), mu_in, sd_in, sd_out), losses
