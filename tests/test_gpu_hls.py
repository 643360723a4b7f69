"""HLS split frequencies (pt_split_frequencies) against the same definition
computed here from the oracle's split sets."""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _reference(n, edges, lnl):
    w = np.exp(np.asarray(lnl) - np.max(lnl))
    acc = {}
    for e, x in zip(edges, w):
        for lo, hi in oracle.tree_splits(n, e):
            k = int(lo) | (int(hi) << 64)
            acc[k] = acc.get(k, 0.0) + x
    return {k: v / w.sum() for k, v in acc.items()}


def test_split_frequencies_of_a_search_hls():
    n, T = 10, 3.0
    a = synth.simulate(n, 500, 501, model="gtr", alpha=0.5)
    with pt.Context(precision="fp64", table_log2=16) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        e, l = synth.random_trees(n, 3, 502)
        lmax, front = ctx.begin(aid, e, l, T)
        hls_e, hls_l = [front["edges"]], [front["lnl"]]
        for _ in range(50):
            if not len(front["edges"]):
                break
            lmax, front = ctx.expand(aid, front["edges"], front["lengths"], T, lmax)
            hls_e.append(front["edges"])
            hls_l.append(front["lnl"])
        edges = np.concatenate(hls_e)
        lnl = np.concatenate(hls_l)
        assert len(edges) > 5
        got = ctx.split_frequencies(aid, edges, lnl)
        ref = _reference(n, edges, lnl)
        keys = pt.keys_to_int(got["splits"])
        assert set(keys) == set(ref)
        for k, f in zip(keys, got["freq"]):
            assert abs(f - ref[k]) <= 1e-12
        assert np.all(np.diff(got["freq"]) <= 0)  # decreasing order
        # majority-rule consensus: the splits above 0.5 are pairwise compatible
        maj = [k for k, f in zip(keys, got["freq"]) if f > 0.5]
        for i in range(len(maj)):
            for j in range(i + 1, len(maj)):
                x, y = maj[i], maj[j]
                assert (x & y) == 0 or (x & y) == x or (x & y) == y
        # tree counts: how many trees hold each split
        sets = [set(int(lo) | (int(hi) << 64) for lo, hi in oracle.tree_splits(n, t)) for t in edges]
        for k, c in zip(keys, got["trees"]):
            assert c == sum(k in s for s in sets)


def test_identical_trees_give_frequency_one():
    n = 12
    a = synth.simulate(n, 200, 503, model="jc")
    with pt.Context(precision="mixed", table_log2=12) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 1.0, 1)
        edges = np.stack([a.tree_edges] * 4)
        got = ctx.split_frequencies(aid, edges, np.array([-10.0, -11.0, -12.5, -10.0]))
        assert len(got["freq"]) == n - 3
        np.testing.assert_allclose(got["freq"], 1.0, rtol=1e-14)
        assert np.all(got["trees"] == 4)
