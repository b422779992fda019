"""Plain NumPy (FP64) reference of the surrogate network -- TEST INFRASTRUCTURE.

y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2
(GELU), loss L = mean over samples and outputs of (y - t)^2, gradients by the
chain rule written out layer by layer.  With ``bf16=True`` the operands of
every product are rounded to bfloat16 (round to nearest even) exactly where
the tensor-core kernels round them -- weights, inputs, hidden activations and
the backward signals -- so a comparison with the GPU isolates accumulation
order.  Parameters are the flat layout W1[128][32], b1, W2[128][128], b2,
W3[32][128], b3.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, HID, OUT = 32, 128, 32
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(flat):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(seed=0):
    """He-style initialisation of the flat parameter vector (FP32 values)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / IN), (HID, IN)), "b1": np.zeros(HID),
         "W2": rng.normal(0, np.sqrt(2.0 / HID), (HID, HID)), "b2": np.zeros(HID),
         "W3": rng.normal(0, np.sqrt(1.0 / HID), (OUT, HID)), "b3": np.zeros(OUT)}
    return pack(d).astype(np.float32)


def forward(flat, x, bf16=False):
    P = unpack(flat)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    xq = r(x)
    z1 = xq @ r(P["W1"]).T + P["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ r(P["W2"]).T + P["b2"]
    h2 = r(gelu(z2))
    y = h2 @ r(P["W3"]).T + P["b3"]
    return y, dict(xq=xq, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_grad(flat, x, t, bf16=False):
    """Loss and flat gradient (same layout as the parameters)."""
    P = unpack(flat)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(flat, x, bf16)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / (B * OUT)
    g = {}
    g["b3"] = dy.sum(axis=0)
    dyq = r(dy)
    g["W3"] = dyq.T @ c["h2"]
    dh2 = dyq @ r(P["W3"])
    dz2 = dh2 * gelu_grad(c["z2"])
    g["b2"] = dz2.sum(axis=0)
    dz2q = r(dz2)
    g["W2"] = dz2q.T @ c["h1"]
    dh1 = dz2q @ r(P["W2"])
    dz1 = dh1 * gelu_grad(c["z1"])
    g["b1"] = dz1.sum(axis=0)
    dz1q = r(dz1)
    g["W1"] = dz1q.T @ c["xq"]
    return loss, pack(g)
