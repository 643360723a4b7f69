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


def test_bf16_storage_points_against_torch_rounding():
    """The BF16 option rounds exactly the stored activations and gradients:
    re-derived with PyTorch's own float32 -> bfloat16 cast at those points."""
    torch = pytest.importorskip("torch")

    def tb(a):  # torch's round-to-nearest-even bfloat16, back to float64
        return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()

    rng = np.random.default_rng(11)
    w = mlp.init_weights(5)
    x = rng.normal(0, 1, (37, mlp.IN))
    t = rng.normal(0, 0.5, (37, mlp.OUT))
    p = mlp.unpack(w)
    X = np.concatenate([x, np.zeros((37, mlp.INP - mlp.IN))], 1)
    z1 = X @ p["W1"] + p["b1"]
    h1 = tb(mlp.gelu(z1))
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = tb(mlp.gelu(z2))
    y = (h2 @ p["W3"] + p["b3"])[:, :mlp.OUT]
    yo, _ = mlp.forward(w, x, bf16=True)
    np.testing.assert_allclose(yo, y, rtol=1e-13, atol=1e-13)
    e = y - t
    dy = np.zeros((37, mlp.OUTP))
    dy[:, :mlp.OUT] = tb(2 * e / (37 * mlp.OUT))
    dz2 = tb((dy @ p["W3"].T) * mlp.gelu_d(z2))
    dz1 = tb((dz2 @ p["W2"].T) * mlp.gelu_d(z1))
    _, g = mlp.loss_grad(w, x, t, bf16=True)
    gp = mlp.unpack(g)
    np.testing.assert_allclose(gp["W1"], X.T @ dz1, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gp["W2"], h1.T @ dz2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gp["b3"], dy.sum(0), rtol=1e-12, atol=1e-15)
    # and the rounding is visible: the unrounded network differs
    assert np.abs(mlp.forward(w, x)[0] - yo).max() > 1e-4
