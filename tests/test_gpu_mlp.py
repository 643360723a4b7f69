"""Learned warm start: the MLP kernels against the FP64 reference
(oracle/mlp.py), and what the trained network gains in a PT search.

BF16 weights, inputs and activations with FP32 accumulation: outputs and
gradients agree element by element, to 1e-3 of each tensor's largest entry,
with the FP64 reference evaluated at the same BF16-rounded weights and
inputs and rounding its activations and back-propagated gradients to BF16
where the kernels store them (the remaining difference is the FP32 rounding
of the kernels' sums, plus the rare BF16 rounding that this flips).
"""
import numpy as np
import pytest

from oracle import mlp
from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([np.log(rng.exponential(0.08, (n, 5))), rng.dirichlet(np.ones(16), (n, 4)).reshape(n, 64) / 4],
                       axis=1)
    t = rng.normal(0, 0.5, (n, 5))
    return x.astype(np.float32), t.astype(np.float32)


def test_forward_matches_reference():
    w = mlp.init_weights(3).astype(np.float32)
    x, _ = _inputs(333, 1)  # not a multiple of the 64-row tile
    with pt.Context() as ctx:
        ctx.mlp_set_weights(w)
        y = ctx.mlp_forward(x)
        np.testing.assert_array_equal(ctx.mlp_get_weights(), w)
    yo, _ = mlp.forward(mlp.to_bf16(w), mlp.to_bf16(x), bf16=True)
    scale = float(np.abs(yo).max())
    np.testing.assert_allclose(y, yo, rtol=0, atol=1e-3 * scale)
    # the unrounded FP64 network is only close: the BF16 activations matter
    yf, _ = mlp.forward(mlp.to_bf16(w), mlp.to_bf16(x))
    assert np.abs(yf - yo).max() > np.abs(y - yo).max()


def test_gradients_match_reference():
    rng = np.random.default_rng(5)
    p = mlp.unpack(mlp.init_weights(4))
    for k in p:
        p[k] = p[k] + rng.normal(0, 0.02, p[k].shape)  # non-zero biases too
    p["W1"][mlp.IN:] = 0.0
    p["W3"][:, mlp.OUT:] = 0.0
    p["b3"][mlp.OUT:] = 0.0
    w = mlp.pack(p).astype(np.float32)
    x, t = _inputs(512, 2)
    with pt.Context() as ctx:
        ctx.mlp_set_weights(w)
        loss, g = ctx.mlp_loss_grad(x, t)
    lo, go = mlp.loss_grad(mlp.to_bf16(w), mlp.to_bf16(x), t, bf16=True)
    assert loss == pytest.approx(lo, rel=1e-4)
    gp, gop = mlp.unpack(g), mlp.unpack(go)
    for name, _ in mlp.SIZES:
        a, b = gp[name], gop[name]
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-3 * float(np.abs(b).max()), err_msg=name)
    # padding rows / columns carry no gradient
    assert np.all(gp["W1"][mlp.IN:] == 0) and np.all(gp["W3"][:, mlp.OUT:] == 0)


def _search(ctx, aid, e, l, T, rounds=8):
    lmax, front = ctx.begin(aid, e, l, T)
    evals = 0
    r = 0
    while len(front["edges"]) and r < rounds:
        lmax, front = ctx.expand(aid, front["edges"], front["lengths"], T, lmax)
        evals += ctx.stats()["prop_evals"]
        r += 1
    return lmax, ctx.visited(aid), evals


def test_trained_warm_start_saves_newton_evaluations():
    n, sites, T = 18, 800, 6.0
    with pt.Context(precision="mixed", table_log2=18) as ctx:
        # training pairs logged from searches on two alignments
        ctx.training_log(True, 1 << 18)
        for seed in (901, 902, 904):
            a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.08)
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            e, l = synth.random_trees(n, 8, seed)
            _search(ctx, aid, e, l, 30.0, rounds=5)  # a wide threshold to collect many proposals
        ctx.training_log(False)
        x, t = ctx.training_pairs()
        assert len(x) > 2000 and np.all(np.isfinite(x)) and np.all(np.isfinite(t))
        ctx.mlp_set_weights(np.zeros(pt.MLP_PARAMS, np.float32) + mlp.init_weights(7, scale=0.1).astype(np.float32))
        loss0, _ = ctx.mlp_loss_grad(x[:4096], t[:4096])
        final = ctx.mlp_train(600, batch=512, lr=2e-3, seed=11)
        loss1, _ = ctx.mlp_loss_grad(x[:4096], t[:4096])
        assert loss1 < 0.7 * loss0, (loss0, loss1, final)
        # a fresh alignment: plain start vs learned start
        a = synth.simulate(n, sites, 903, model="gtr", alpha=0.5, mean_branch=0.08)
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        e, l = synth.random_trees(n, 4, 903)
        ctx.mlp_enable(False)
        lm0, v0, ev0 = _search(ctx, aid, e, l, T)
        ctx.mlp_enable(True)
        lm1, v1, ev1 = _search(ctx, aid, e, l, T)
    d0 = dict(zip(pt.keys_to_int(v0["keys"]), zip(v0["status"], v0["lnl"])))
    d1 = dict(zip(pt.keys_to_int(v1["keys"]), zip(v1["status"], v1["lnl"])))
    assert set(d0) == set(d1)
    for k in d0:
        assert d0[k][0] == d1[k][0]
        assert abs(d0[k][1] - d1[k][1]) <= 1e-3
    assert abs(lm0 - lm1) <= 1e-3
    print(f"Newton evaluations: plain {ev0}, learned {ev1} ({100 * (1 - ev1 / ev0):.1f}% saved)")
    assert ev1 < ev0
