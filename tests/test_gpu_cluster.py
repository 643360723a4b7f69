"""Proposal kernel with its sites split over a thread-block cluster: each of
K CTAs takes a contiguous share of the site patterns (its sum-table share in
shared memory) and the Newton sums, the scores and the step are reduced over
the cluster.  Forced through an autotune cache entry for K = 1, 2, 4, 8 on an
alignment whose whole sum-table does not fit in one CTA's shared memory;
sampled proposals against the oracle (1e-3 nats, lengths 1e-4 relative) and
the next frontier equal across K."""
import json

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


@pytest.fixture(scope="module")
def case():
    n, sites = 16, 6000
    a = synth.simulate(n, sites, 337, model="gtr", alpha=0.5, mean_branch=0.4)
    tips, w = synth.compress_patterns(a.codes)
    assert tips.shape[1] > 3300  # FP32 sum-table beyond one CTA's shared memory
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    e, l = synth.random_trees(n, 2, 8)
    return n, a, tips.shape[1], pb, e, l


def _round(case, K, tmp_path):
    n, a, P, _, e, l = case
    key = f"prec1_cat4_taxa{(n + 7) // 8 * 8}_patterns{(P + 255) // 256 * 256}"
    path = tmp_path / f"tune{K}.json"
    path.write_text(json.dumps({key: {"prop_threads": 256, "prop_cluster": K, "full_threads": 0, "prop_ms": 0,
                                      "full_ms": 0, "prop_items": 1 << 30, "full_items": 0}}))
    with pt.Context(precision="mixed", table_log2=14) as ctx:
        ctx.autotune(False, str(path))  # the cache entry: K CTAs per proposal
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        lmax, front = ctx.begin(aid, e, l, np.inf)
        lm2, nxt = ctx.expand(aid, front["edges"][:1], front["lengths"][:1], np.inf, lmax)
        props = ctx.last_proposals()
        assert ctx.autotune_report()[key]["prop_cluster"] == K
    return front, props, nxt, lm2


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_cluster_split_proposals_match_oracle(case, K, tmp_path):
    n, a, P, pb, e, l = case
    front, props, nxt, _ = _round(case, K, tmp_path)
    pe, plen = front["edges"][0], front["lengths"][0]
    _, _, nk = oracle.nni_neighbours(n, pe, plen)
    keys = pt.keys_to_int(nk)
    assert set(keys) == set(pt.keys_to_int(props["keys"]))
    for i in range(0, len(props["keys"]), 4):
        j = keys.index(pt.keys_to_int(props["keys"][i])[0])
        lp, _, _ = pb.propose(pe, plen, j)
        assert abs(props["lnl"][i] - lp) <= 1e-3, (K, i, props["lnl"][i], lp)


def test_cluster_split_rounds_agree(case, tmp_path):
    base = _round(case, 1, tmp_path)
    for K in (2, 8):
        other = _round(case, K, tmp_path)
        assert pt.keys_to_int(other[2]["keys"]) == pt.keys_to_int(base[2]["keys"])
        np.testing.assert_allclose(other[2]["lnl"], base[2]["lnl"], rtol=0, atol=1e-3)
        np.testing.assert_allclose(other[1]["len5"], base[1]["len5"], rtol=1e-4, atol=1e-6)
        assert abs(other[3] - base[3]) <= 1e-3


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_cluster_split_full_optimisation_matches_oracle(case, K, tmp_path):
    """The full optimisation with each tree's sites split over a cluster of K
    CTAs (each CTA a slab and a sum-table of its share): lnL and lengths
    against the oracle's full optimisation."""
    n, a, P, pb, e, l = case
    key = f"prec1_cat4_taxa{(n + 7) // 8 * 8}_patterns{(P + 255) // 256 * 256}"
    path = tmp_path / f"tunef{K}.json"
    path.write_text(json.dumps({key: {"prop_threads": 0, "prop_cluster": 0, "full_threads": 256, "full_cluster": K,
                                      "prop_ms": 0, "full_ms": 0, "prop_items": 0, "full_items": 1 << 30}}))
    with pt.Context(precision="mixed", table_log2=14) as ctx:
        ctx.autotune(False, str(path))
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        lnl, lens, _ = ctx.score(aid, e, l, mode="full")
        assert ctx.autotune_report()[key]["full_cluster"] == K
    for i in range(len(e)):
        want, wl, _ = pb.full_optimise(e[i], l[i])
        assert abs(lnl[i] - want) <= 1e-3, (K, i, lnl[i], want)
        np.testing.assert_allclose(lens[i], wl, rtol=1e-4, atol=1e-6)
