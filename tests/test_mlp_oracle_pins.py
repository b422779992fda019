"""Pins of the NumPy reference network (CPU): its analytic gradient against
central finite differences of its own loss, and the bfloat16 rounding helper
against the format's definition."""
import numpy as np

from oracle import mlp_oracle as M


def test_analytic_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    flat = M.init_params(1).astype(np.float64)
    x = rng.normal(size=(7, M.IN))
    t = rng.normal(size=(7, M.OUT))
    loss, g = M.loss_grad(flat, x, t)
    idx = rng.choice(M.NPARAMS, size=60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(flat)
        e[k] = h
        lp, _ = M.loss_grad(flat + e, x, t)
        lm, _ = M.loss_grad(flat - e, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, k


def test_bf16_rounding_is_round_to_nearest_even_on_8_bit_mantissa():
    # exactly representable values survive
    for v in (1.0, -2.5, 0.15625, 2.0 ** 127):
        assert M.round_bf16(np.array([v]))[0] == np.float32(v)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert M.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert M.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    r = M.round_bf16(np.random.default_rng(0).normal(size=1000))
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
