"""Pins of the NumPy reference network (CPU): its analytic gradient against
central finite differences of its own loss, and the bfloat16 rounding helper
against the format's definition."""
import numpy as np
import pytest

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


def test_forward_of_a_hand_worked_two_unit_network():
    """A network worked by hand.  x = (1, -1, 0, ...); W1 routes x0 to hidden
    unit 0 and x1 to unit 1; W2 forms h1[0] - h1[1] in unit 0 of the second
    layer; W3 doubles that unit into output 0; b3 puts 0.25 on output 1.  For
    the exact GELU g(z) = z Phi(z), g(1) - g(-1) = Phi(1) + (1 - Phi(1)) = 1,
    so the second layer sees exactly 1 and y0 = 2 g(1) = 2 Phi(1), with
    Phi(1) = 0.8413447460685429 from the standard normal table.  The tanh
    approximation of GELU gives 0.84119 there; a swapped layer, a transposed
    weight or a bias added after the activation all move y off these values."""
    P = {name: np.zeros(shape) for name, shape in M.SIZES}
    P["W1"][0, 0] = 1.0
    P["W1"][1, 1] = 1.0
    P["W2"][0, 0] = 1.0
    P["W2"][0, 1] = -1.0
    P["W3"][0, 0] = 2.0
    P["b3"][1] = 0.25
    flat = M.pack(P)
    x = np.zeros((1, M.IN))
    x[0, 0], x[0, 1] = 1.0, -1.0
    y, c = M.forward(flat, x)
    phi1 = 0.8413447460685429
    assert c["h1"][0, 0] == pytest.approx(phi1, abs=1e-15)
    assert c["h1"][0, 1] == pytest.approx(-(1.0 - phi1), abs=1e-15)
    assert c["z2"][0, 0] == pytest.approx(1.0, abs=1e-15)
    expect = np.zeros(M.OUT)
    expect[0] = 2.0 * phi1
    expect[1] = 0.25
    assert np.allclose(y[0], expect, rtol=0, atol=1e-15)
    # the transposed first layer routes x into different units: output changes
    Pt = dict(P)
    Pt["W1"] = np.zeros_like(P["W1"])
    Pt["W1"][0, 1] = 1.0
    Pt["W1"][1, 0] = 1.0
    yt, _ = M.forward(M.pack(Pt), x)
    assert abs(yt[0, 0] - expect[0]) > 1.0


def test_gelu_symmetry_and_derivative_at_zero():
    """g(z) - g(-z) = z for every z (Phi(z) + Phi(-z) = 1); g(0) = 0; g'(0) = 1/2;
    the analytic derivative the backward pass uses integrates back to g."""
    from scipy.integrate import quad

    z = np.linspace(-6, 6, 241)
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, rtol=0, atol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    for b in (-3.0, -0.7, 0.4, 2.5):
        val, _ = quad(lambda s: float(M.gelu_grad(np.array([s]))[0]), 0.0, b, epsabs=1e-13, epsrel=1e-13)
        assert val == pytest.approx(float(M.gelu(np.array([b]))[0]), abs=1e-11)


def test_forward_equals_an_independent_torch_definition_of_the_network():
    """The same 32 -> 128 -> 128 -> 32 network built from torch.nn layers
    (Linear computes x W^T + b with W stored [out][in]; GELU with
    approximate='none' is the erf form), loaded from the flat parameter layout
    W1, b1, W2, b2, W3, b3, in FP64: the oracle's forward must agree."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    flat = rng.normal(scale=0.3, size=M.NPARAMS)
    x = rng.normal(size=(9, M.IN))
    net = torch.nn.Sequential(torch.nn.Linear(M.IN, M.HID), torch.nn.GELU(approximate="none"),
                              torch.nn.Linear(M.HID, M.HID), torch.nn.GELU(approximate="none"),
                              torch.nn.Linear(M.HID, M.OUT)).double()
    off = 0
    layers = [net[0].weight, net[0].bias, net[2].weight, net[2].bias, net[4].weight, net[4].bias]
    with torch.no_grad():
        for prm, (name, shape) in zip(layers, M.SIZES):
            n = int(np.prod(shape))
            assert tuple(prm.shape) == shape, name
            prm.copy_(torch.from_numpy(flat[off:off + n].reshape(shape)))
            off += n
        y_t = net(torch.from_numpy(x)).numpy()
    y, _ = M.forward(flat, x)
    assert np.allclose(y, y_t, rtol=1e-13, atol=1e-13)
