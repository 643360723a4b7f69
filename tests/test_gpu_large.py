"""Large problems: sum-tables too big for shared memory (the kernels then
keep them in a global scratch slab), 128 taxa, and a 10,000-site alignment
with ~6000 patterns, checked against the oracle on sampled outputs."""
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


@pytest.mark.parametrize("prec,n,sites,mb", [("mixed", 16, 6000, 0.4), ("fp64", 14, 3000, 0.3)])
def test_scratch_sumtable_path_matches_oracle(prec, n, sites, mb):
    # FP32: 4C+2 floats x ~3500+ patterns > 227 KB; FP64 beyond ~1600 patterns
    a = synth.simulate(n, sites, 321 + n, model="gtr", alpha=0.5, mean_branch=mb)
    tips, w = synth.compress_patterns(a.codes)
    assert tips.shape[1] > (3300 if prec == "mixed" else 1700)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    tol = 1e-3 if prec == "mixed" else 1e-8
    e, l = synth.random_trees(n, 2, 8)
    with pt.Context(precision=prec, table_log2=14) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        lnl, lens, _ = ctx.score(aid, e, l, mode="full")
        for i in range(len(e)):
            want, wl, _ = pb.full_optimise(e[i], l[i])
            assert abs(lnl[i] - want) <= tol, (i, lnl[i], want)
        lmax, front = ctx.begin(aid, e, l, np.inf)
        lm2, nxt = ctx.expand(aid, front["edges"][:1], front["lengths"][:1], np.inf, lmax)
        props = ctx.last_proposals()
    # sampled proposals against the oracle
    pe, plen = front["edges"][0], front["lengths"][0]
    _, _, nk = oracle.nni_neighbours(n, pe, plen)
    keys = pt.keys_to_int(nk)
    for i in range(0, len(props["keys"]), 3):
        kk = pt.keys_to_int(props["keys"][i])[0]
        j = keys.index(kk)
        lp, _, _ = pb.propose(pe, plen, j)
        assert abs(props["lnl"][i] - lp) <= tol, (i, props["lnl"][i], lp)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_128_taxa_10000_sites_round(prec):
    # the largest configuration of the workload set: 128 taxa, 10,000 sites
    # (~6000 patterns), GTR+G4, Exp(0.02) branches, lnL ~ -5e5.  Against the
    # oracle at the precision's absolute tolerance: lnL at fixed lengths; the
    # visit of the generating topology (its lnL is the oracle's at the visit's
    # lengths, and those lengths are stationary: each sampled branch's Newton
    # step -d1/d2 is below 1e-6 relative or the branch sits at its lower bound);
    # one round of proposals, sampled (the oracle needs ~1 s per proposal here)
    tol = {"fp64": 1e-8, "mixed": 1e-3}[prec]
    n, sites = 128, 10000
    a = synth.simulate(n, sites, 5005, model="gtr", alpha=0.5, mean_branch=0.02)
    tips, w = synth.compress_patterns(a.codes)
    assert tips.shape[1] > 4000
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    e, l = a.tree_edges[None], np.full((1, 2 * n - 3), 0.02)
    with pt.Context(precision=prec, table_log2=18) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        lnl_fixed, _, _ = ctx.score(aid, e, a.tree_lengths[None], mode="fixed")
        want = pb.loglik(a.tree_edges, a.tree_lengths)
        assert abs(lnl_fixed[0] - want) <= tol, (lnl_fixed[0], want)
        lmax, front = ctx.begin(aid, e, l, 15.0)
        lm2, nxt = ctx.expand(aid, front["edges"], front["lengths"], 15.0, lmax)
        props = ctx.last_proposals()
        st = ctx.stats()
    assert st["scored"] == 2 * (n - 3) and st["nonconverged"] == 0
    pe, plen = front["edges"][0], front["lengths"][0]
    assert abs(front["lnl"][0] - pb.loglik(pe, plen)) <= tol
    for k in range(0, 2 * n - 3, 37):
        _, d1, d2 = pb.edge_derivs(pe, plen, k)
        assert abs(d1 / d2) <= 1e-5 or (plen[k] <= 1e-6 + 2e-8 and d1 < 0), (k, d1, d2, plen[k])
    _, _, nk = oracle.nni_neighbours(n, pe, plen)
    keys = pt.keys_to_int(nk)
    assert set(keys) == set(pt.keys_to_int(props["keys"]))
    pb.settings()
    for i in range(0, len(props["keys"]), 50):
        kk = pt.keys_to_int(props["keys"][i])[0]
        lp, _, _ = pb.propose(pe, plen, keys.index(kk))
        assert abs(props["lnl"][i] - lp) <= tol, (i, props["lnl"][i], lp)
