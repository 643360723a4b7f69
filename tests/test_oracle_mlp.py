"""Pins of the FP64 MLP reference: gradients against central finite
differences of its own loss (an independent check of the backward formulas),
and GELU against its integral definition."""
import numpy as np
import pytest
from scipy import integrate, stats

from oracle import mlp


def test_gelu_matches_definition():
    for z in [-3.0, -0.7, 0.0, 0.4, 2.5]:
        assert mlp.gelu(z) == pytest.approx(z * stats.norm.cdf(z), abs=1e-15)
        h = 1e-6
        assert mlp.gelu_d(z) == pytest.approx((mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), abs=1e-8)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    w = mlp.init_weights(1)
    w += rng.normal(0, 0.01, w.size)  # non-zero biases
    x = rng.normal(0, 1, (7, mlp.IN))
    t = rng.normal(0, 1, (7, mlp.OUT))
    loss, g = mlp.loss_grad(w, x, t)
    idx = rng.choice(w.size, 60, replace=False)
    p = mlp.unpack(np.arange(w.size))
    live = set(p["W1"][:mlp.IN].ravel()) | set(p["b1"]) | set(p["W2"].ravel()) | set(p["b2"]) | \
        set(p["W3"][:, :mlp.OUT].ravel()) | set(p["b3"][:mlp.OUT])
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_grad(wp, x, t)[0] - mlp.loss_grad(wm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        if i not in live:
            assert g[i] == 0.0  # padding rows/columns carry no gradient


def test_bf16_rounding():
    # bfloat16 keeps 7 explicit mantissa bits: spacing 2^-7 just above 1
    v = np.array([1.0, 1.0078125, 1.00390625, 1.01171875, -3.14159])
    r = mlp.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0078125
    assert r[2] == 1.0          # halfway, ties to even
    assert r[3] == 1.015625     # halfway between 1.0078125 and 1.015625, ties to even
    assert abs(r[4] - v[4]) <= 2 ** -8 * abs(v[4])
