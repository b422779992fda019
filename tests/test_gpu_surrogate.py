"""The learned per-grain modal surrogate on the GPU.

1. The co-rotated modal projection agrees with the full bond kernel: a grain
   deformed along one basis mode (and moved rigidly) gives q = alpha e_m and a
   modal bond force -lambda_m alpha e_m.
2. The tensor-core basis products (projection and expansion over several grain
   tiles, chunks and row tiles) agree with the CUDA-core projection and with
   R(theta + phi) Phi f E h evaluated in FP64 on the host.
3. A network trained (on the GPU, by the library's kernels) on snapshots of
   freely vibrating grains predicts their modal bond force better than the
   linear modal model it corrects, on vibrations it has not seen.
4. On the settling aggregate the surrogate keeps intact grains, its judged
   error stays within the tolerance, and the trajectory stays close to the
   full FP32 path.
"""
import math

import numpy as np
import pytest

from paper_2108_07212_gb300 import binding as B
from paper_2108_07212_gb300 import inputs as I
from paper_2108_07212_gb300 import surrogate as SU

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _one_grain(shape="hexagon", theta=0.7):
    R = 1e-3
    return I.Workload(shapes=[I.SHAPE_MAKERS[shape]()], grain_shape=np.array([0], np.int32),
                      grain_geom=np.array([[5e-3, 5e-3, R, theta, 0, 0, R / 15]]),
                      params=I.default_params(gy=0.0, wall_lo=(0.0, 0.0), wall_hi=(1e-2, 1e-2)), n_steps=1)


@pytest.mark.parametrize("mode", [0, 5, 31])
def test_modal_projection_matches_full_bond_kernel(mode):
    w = _one_grain()
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0",
                     surrogate=lambda s: SU.build_basis(s, n_modes=32))
    cfg = S.surrogate_basis
    X = S.get("X")
    n = X.shape[0]
    Phi = cfg["basis"].reshape(n, 2, 32)
    lam = cfg["lambda_"]
    h = w.grain_geom[0, 6]
    th = w.grain_geom[0, 3]
    alpha = 1e-3
    wl = alpha * h * Phi[:, :, mode]                              # lattice-frame deformation
    c, s = math.cos(th), math.sin(th)
    wworld = np.stack([c * wl[:, 0] - s * wl[:, 1], s * wl[:, 0] + c * wl[:, 1]], axis=1)
    xbar = X.mean(axis=0)
    psi = 0.3                                                      # rigid rotation + translation on top
    cp, sp = math.cos(psi), math.sin(psi)
    rel = X - xbar + wworld
    p = xbar + np.array([2e-4, -1e-4]) + np.stack([cp * rel[:, 0] - sp * rel[:, 1], sp * rel[:, 0] + cp * rel[:, 1]], 1)
    S.set("DISP", p - X)
    q, f = S.surrogate_sample()
    e = np.zeros(32)
    e[mode] = 1.0
    assert np.abs(q[0] - alpha * e).max() <= 2e-3 * alpha
    assert np.abs(f[0] - (-lam[mode] * alpha) * e).max() <= 2e-3 * lam[mode] * alpha


def _kabsch(Xg, pg):
    A = Xg - Xg.mean(0)
    Bq = pg - pg.mean(0)
    return math.atan2((A[:, 0] * Bq[:, 1] - A[:, 1] * Bq[:, 0]).sum(), (A * Bq).sum())


def _deformed(S, cfg, amp, seed):
    """Random modal deformation (max nodal displacement about amp h per grain)
    plus a rigid rotation and translation of every grain."""
    rng = np.random.default_rng(seed)
    G = S.workload.n_grains
    lam = cfg["lambda_"].reshape(-1, 32)
    tmpl = cfg["template_of_grain"]
    coeffs = rng.normal(size=(G, 32)) / np.sqrt(lam[tmpl])
    u = SU.modal_field(S, cfg, coeffs)
    X = S.get("X")
    grain = S.get("GRAIN")
    for g in range(G):                                        # largest nodal displacement amp h
        m = grain == g
        f = amp * S.workload.grain_geom[g, 6] / np.sqrt((u[m] ** 2).sum(1)).max()
        coeffs[g] *= f
        u[m] *= f
    for g in range(G):
        m = grain == g
        psi = rng.uniform(-0.5, 0.5)
        c, s = math.cos(psi), math.sin(psi)
        xb = X[m].mean(0)
        rel = X[m] - xb + u[m]
        u[m] = xb + rng.normal(size=2) * 1e-4 + np.stack([c * rel[:, 0] - s * rel[:, 1], s * rel[:, 0] + c * rel[:, 1]], 1) - X[m]
    return coeffs, u


def test_tensor_core_products_match_fp64_host():
    # 150 hexagons (two grain tiles, 510 rows: two row tiles, four chunks) and 12 disks
    w = I.free_grains(shapes=("hexagon", "disk"), n_per_shape=150, h_ratio=10)
    keep = np.r_[np.arange(150), np.arange(150, 162)]
    w.grain_shape = w.grain_shape[keep]
    w.grain_geom = w.grain_geom[keep]
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0",
                     surrogate=lambda s: SU.build_basis(s, judge_every=50))
    cfg = S.surrogate_basis
    counts = np.bincount(cfg["template_of_grain"])
    nets = [B.MLP(max_batch=int(c), params=SU.init_params(t)) for t, c in enumerate(counts)]
    for t, net in enumerate(nets):
        S.surrogate_set_mlp(t, net)
    S.surrogate_enable(True)
    coeffs, u = _deformed(S, cfg, amp=0.05, seed=3)
    S.set("DISP", u)
    S.set("STEP", np.array([7], np.int64))                   # not a judge step
    q_tc, y = S.surrogate_inspect()
    Fb = S.get("FORCE_PARTS")[0]
    q_cc, _ = S.surrogate_sample()
    lam = cfg["lambda_"].reshape(-1, 32)[cfg["template_of_grain"]]
    # projection: tensor cores (BF16 split, chunked) vs CUDA cores (FP32)
    assert np.abs(q_tc - q_cc).max() <= 1e-4 * np.abs(q_cc).max()
    assert np.abs(q_cc - coeffs).max() <= 2e-2 * np.abs(coeffs).max()
    # an untrained network adds nothing: f = -lambda q
    assert np.abs(y + lam * q_tc).max() <= 1e-6 * np.abs(lam * q_tc).max()
    # expansion: surrogate nodal bond force vs R(theta + phi) Phi f E h in FP64
    X = S.get("X")
    grain = S.get("GRAIN")
    E = w.params["E"]
    offs = np.concatenate([[0], np.cumsum([2 * d["nodes"] * 32 for d in cfg["templates"]])])
    worst = 0.0
    for g in range(w.n_grains):
        m = grain == g
        t = int(cfg["template_of_grain"][g])
        n = int(m.sum())
        Phi = cfg["basis"][offs[t]:offs[t + 1]].astype(np.float64).reshape(n, 2, 32)
        fl = Phi @ y[g].astype(np.float64)
        ang = w.grain_geom[g, 3] + _kabsch(X[m], X[m] + u[m])
        c, s = math.cos(ang), math.sin(ang)
        h = w.grain_geom[g, 6]
        ref = np.stack([c * fl[:, 0] - s * fl[:, 1], s * fl[:, 0] + c * fl[:, 1]], 1) * E * h
        worst = max(worst, np.abs(Fb[m] - ref).max() / np.abs(ref).max())
    assert worst <= 1e-4, worst


def test_in_step_networks_match_the_network_oracle():
    """The networks as the step runs them (every template's tiles in one
    launch, f = net(q) - Lambda q formed in the output epilogue) against the
    oracle network with the same bfloat16 rounding, element by element, on the
    modal coefficients the step fed them.  Random networks (every layer
    non-zero), 150 hexagons (two 128-row tiles of one template) and 12 disks."""
    from oracle import mlp_oracle as M
    w = I.free_grains(shapes=("hexagon", "disk"), n_per_shape=150, h_ratio=10)
    keep = np.r_[np.arange(150), np.arange(150, 162)]
    w.grain_shape = w.grain_shape[keep]
    w.grain_geom = w.grain_geom[keep]
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0",
                     surrogate=lambda s: SU.build_basis(s, judge_every=50))
    cfg = S.surrogate_basis
    tmpl = cfg["template_of_grain"]
    counts = np.bincount(tmpl)
    params = [M.init_params(11 + t) for t in range(len(counts))]
    nets = [B.MLP(max_batch=int(c), params=params[t]) for t, c in enumerate(counts)]
    for t, net in enumerate(nets):
        S.surrogate_set_mlp(t, net)
    S.surrogate_enable(True)
    _, u = _deformed(S, cfg, amp=0.3, seed=5)
    S.set("DISP", u)
    S.set("STEP", np.array([7], np.int64))                   # not a judge step
    q, y = S.surrogate_inspect()
    lam = cfg["lambda_"].reshape(-1, 32)
    worst = 0.0
    for t in range(len(counts)):
        m = tmpl == t
        net_ref, _ = M.forward(params[t].astype(np.float64), q[m], bf16=True)
        lin = lam[t] * q[m].astype(np.float64)
        bound = 2.0 ** -6 * (np.abs(net_ref).max() + np.abs(net_ref)) + 1e-6 * np.abs(lin).max()
        assert np.abs(net_ref).max() > 0
        worst = max(worst, float((np.abs(y[m] - (net_ref - lin)) / bound).max()))
    assert worst <= 1.0, worst


def _static_samples(w, cfg_fn, amp, seed, draws):
    """Training pairs from the full bond kernel at random modal deformations
    (largest nodal displacement up to amp h) of every grain: (q, f) per template."""
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0", surrogate=cfg_fn)
    cfg = S.surrogate_basis
    tmpl = cfg["template_of_grain"]
    rng = np.random.default_rng(seed)
    out = {}
    for k in range(draws):
        _, u = _deformed(S, cfg, amp * rng.uniform(0.2, 1.0), seed * 100003 + k)
        S.set("DISP", u)
        q, f = S.surrogate_sample()
        for t in np.unique(tmpl):
            out.setdefault(int(t), []).append((q[tmpl == t], f[tmpl == t]))
    return cfg, {t: (np.vstack([a for a, _ in v]), np.vstack([b for _, b in v])) for t, v in out.items()}


def test_training_beats_the_linear_modal_model_on_unseen_vibrations():
    w = I.free_grains(shapes=("hexagon", "disk"), n_per_shape=24, h_ratio=10)
    basis = {}

    def cfg_fn(s):
        if "cfg" not in basis:
            basis["cfg"] = SU.build_basis(s, judge_every=50, gate=0.5, err_tol=10.0)
        return basis["cfg"]

    amp = 0.06
    # snapshots of the full bond kernel at random deformations; the test runs
    # free vibrations from other random deformations
    cfg, data = _static_samples(w, cfg_fn, amp, seed=1, draws=200)
    lam = cfg["lambda_"].reshape(-1, 32)
    trained = {t: SU.train_template(q, f, lam[t], epochs=3000, lr=2e-3, batch=512)[0] for t, (q, f) in data.items()}
    untrained = {t: SU.init_params(0) for t in trained}
    merr = {}
    for name, nets in (("linear", untrained), ("trained", trained)):
        S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device="cuda:0", surrogate=cfg)
        _, u = _deformed(S, cfg, amp, seed=2)
        S.set("DISP", u)
        S.eval_forces()
        counts = np.bincount(cfg["template_of_grain"])
        hs = [B.MLP(max_batch=int(counts[t]), params=nets[t]) for t in range(len(counts))]
        for t, h in enumerate(hs):
            S.surrogate_set_mlp(t, h)
        S.surrogate_enable(True)
        errs = []
        for _ in range(6):
            S.step(50)                                        # every 50th step is a judge step
            active, err, me, maxs = S.surrogate_stats()
            assert active.all() and maxs.max() < 0.5
            errs.append(me)
        merr[name] = float(np.median(np.concatenate(errs)))
        rc, _ = S.status()
        assert rc == B.PD_OK
    assert merr["trained"] < 0.33 * merr["linear"], merr


def _thrown(n_grains=12, seed=5):
    w = I.settling(n_grains=n_grains, seed=seed)
    w.grain_geom[:, 5] = -1.5
    w.grain_geom[:, 4] = np.linspace(-0.5, 0.5, n_grains)
    return w


def test_surrogate_settling_stays_within_tolerance():
    w = _thrown()
    S0 = B.Simulation(w, precision=B.PD_FP32_SPLIT, store_parts=True, device="cuda:0",
                      surrogate=lambda s: SU.build_basis(s))
    cfg = S0.surrogate_basis
    data = SU.collect_samples(S0, 600, 20)
    lam = cfg["lambda_"].reshape(-1, 32)
    nets = {t: SU.train_template(q, f, lam[t], epochs=300)[0] for t, (q, f) in data.items()}
    plain = B.Simulation(w, precision=B.PD_FP32_SPLIT, device="cuda:0")
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device="cuda:0", surrogate=cfg)
    counts = np.bincount(cfg["template_of_grain"])
    hs = {t: B.MLP(max_batch=int(counts[t]), params=p) for t, p in nets.items()}
    for t, h in hs.items():
        S.surrogate_set_mlp(t, h)
    S.surrogate_enable(True)
    for _ in range(8):
        plain.step(50)
        S.step(50)
        active, err, me, maxs = S.surrogate_stats()
        assert np.all(err[active == 1] <= cfg["err_tol"])
        assert np.all(maxs[active == 1] <= cfg["gate"])
    assert active.sum() >= 1
    u0, u1 = plain.get("DISP"), S.get("DISP")
    assert np.linalg.norm(u1 - u0) <= 1e-3 * np.linalg.norm(u0)
    assert np.array_equal(plain.get("BROKEN"), S.get("BROKEN"))
    rc, st = S.status()
    assert rc == B.PD_OK


def test_removing_a_network_takes_its_grains_off_the_surrogate():
    w = I.free_grains(shapes=("hexagon", "disk"), n_per_shape=3, h_ratio=8)
    S = B.Simulation(w, precision=B.PD_FP32_SPLIT, device="cuda:0", surrogate=lambda s: SU.build_basis(s))
    cfg = S.surrogate_basis
    hs = [B.MLP(max_batch=3, params=SU.init_params(0)) for _ in range(2)]
    for t, h in enumerate(hs):
        S.surrogate_set_mlp(t, h)
    S.surrogate_enable(True)
    S.step(3)
    S.surrogate_set_mlp(1, None)
    active, *_ = S.surrogate_stats()
    assert np.array_equal(active, (cfg["template_of_grain"] == 0).astype(np.int32))
    S.step(60)
    rc, _ = S.status()
    assert rc == B.PD_OK
