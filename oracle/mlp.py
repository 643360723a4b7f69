"""FP64 reference of the warm-start MLP (test infrastructure only).

69 inputs (zero-padded to 80) -> 128 -> 128 -> 5 (padded to 8), exact GELU
x * Phi(x); loss = mean over rows and the 5 outputs of the squared error.
Flat parameter layout: W1 [80][128], b1 [128], W2 [128][128], b2 [128],
W3 [128][8], b3 [8]; each layer computes y = x W + b.  Written from those
definitions with numpy; it shares nothing with the CUDA kernels.

bf16=True applies the network's stated precision (BF16 weights, inputs and
activations, FP32 accumulation): the hidden activations gelu(z), the output
gradient and the back-propagated pre-activation gradients are rounded to
BF16 where the network stores them in that format; everything else stays
FP64, so the result differs from a BF16/FP32 implementation only by the
rounding of its FP32 sums.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, INP, H, OUT, OUTP = 69, 80, 128, 5, 8
SIZES = [("W1", (INP, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, OUTP)), ("b3", (OUTP,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def _pad(x):
    x = np.asarray(x, np.float64).reshape(-1, IN)
    return np.concatenate([x, np.zeros((x.shape[0], INP - IN))], axis=1)


def forward(w, x, bf16=False):
    q = to_bf16 if bf16 else (lambda a: a)
    p = unpack(w)
    X = _pad(x)
    z1 = X @ p["W1"] + p["b1"]
    h1 = q(gelu(z1))
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = q(gelu(z2))
    y = h2 @ p["W3"] + p["b3"]
    return y[:, :OUT], (X, z1, h1, z2, h2)


def loss_grad(w, x, t, bf16=False):
    q = to_bf16 if bf16 else (lambda a: a)
    p = unpack(w)
    y, (X, z1, h1, z2, h2) = forward(w, x, bf16)
    t = np.asarray(t, np.float64).reshape(-1, OUT)
    n = y.shape[0]
    e = y - t
    loss = float(np.sum(e * e) / (n * OUT))
    dy = np.zeros((n, OUTP))
    dy[:, :OUT] = q(2.0 * e / (n * OUT))
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dz2 = q((dy @ p["W3"].T) * gelu_d(z2))
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = q((dz2 @ p["W2"].T) * gelu_d(z1))
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def init_weights(seed, scale=1.0):
    """He-style random weights (inputs' padding rows and outputs' padding columns zero)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, scale * np.sqrt(2.0 / IN), (INP, H)), "b1": np.zeros(H),
         "W2": rng.normal(0, scale * np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, scale * np.sqrt(1.0 / H), (H, OUTP)), "b3": np.zeros(OUTP)}
    d["W1"][IN:] = 0.0
    d["W3"][:, OUT:] = 0.0
    return pack(d)


def to_bf16(a):
    """Round to bfloat16 (nearest even) and back to float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
