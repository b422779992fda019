"""The surrogate network on the tensor cores (tcgen05, BF16 operands, FP32
accumulation): forward and gradients against the NumPy reference network with
the same bfloat16 rounding, and training that actually reduces the loss."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2108_07212_gb300 import binding as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# Element-wise tolerance of the BF16 network against the reference with the
# same bfloat16 rounding.  Both round every operand to BF16 at the same places;
# they differ in accumulation (FP32 on the tensor cores, FP64 here) and in the
# float erf of the GELU.  Those differences are ~1e-6 relative, but one of them
# can move a hidden activation across a BF16 rounding boundary: that changes it
# by one BF16 unit (2^-8 relative), and the change reaches an output through one
# weight.  So an output may differ by a few 2^-8 of the output scale, never by
# more: |y - y_ref| <= TOL (max|y_ref| + |y_ref|) with TOL = 2^-6 (four units).
TOL = 2.0 ** -6


def _elementwise_ok(a, b, tol=TOL):
    """|a - b| <= tol (max|b| + |b|) for every element; returns the worst ratio."""
    bound = tol * (np.abs(b).max() + np.abs(b))
    ratio = np.abs(a - b) / np.maximum(bound, 1e-300)
    return float(ratio.max())


def _data(n, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 32)).astype(np.float32)
    A = rng.normal(scale=0.3, size=(32, 32))
    t = (np.tanh(x @ A) + 0.1 * x[:, ::-1]).astype(np.float32)
    return x, t


@pytest.mark.parametrize("n", [1, 128, 300])
def test_forward_matches_reference(n):
    params = M.init_params(3)
    x, _ = _data(n, 1)
    net = B.MLP(max_batch=512, params=params)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, _ = M.forward(params.astype(np.float64), x, bf16=True)
    worst = _elementwise_ok(y, y_ref)
    assert worst <= 1.0, worst
    # against the unrounded FP64 network: BF16 weights and activations (8-bit
    # mantissas, 2^-9 relative each) over three layers, element-wise
    y64, _ = M.forward(params.astype(np.float64), x)
    worst64 = _elementwise_ok(y, y64, tol=2.0 ** -4)
    assert worst64 <= 1.0, worst64


@pytest.mark.parametrize("n", [200, 1024])
def test_gradients_match_reference(n):
    params = M.init_params(5)
    x, t = _data(n, 2)
    net = B.MLP(max_batch=2048, params=params)
    loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    loss_ref, g_ref = M.loss_grad(params.astype(np.float64), x, t, bf16=True)
    assert loss == pytest.approx(loss_ref, rel=2e-3)
    off = 0
    for name, shape in M.SIZES:
        k = int(np.prod(shape))
        a, b = g[off:off + k], g_ref[off:off + k]
        # element-wise, block by block: the backward signals are BF16-rounded as
        # in the forward pass, and each gradient entry sums n products of them
        worst = _elementwise_ok(a, b)
        assert worst <= 1.0, (name, worst)
        off += k


def test_training_reduces_the_loss():
    params = M.init_params(7)
    x, t = _data(2048, 3)
    net = B.MLP(max_batch=2048, params=params)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.train_step(xd, td, 3e-3)
    for _ in range(300):
        last = net.train_step(xd, td, 3e-3)
    assert last < 0.1 * first, (first, last)
    p = net.get_params()
    assert np.all(np.isfinite(p)) and not np.array_equal(p, params)
