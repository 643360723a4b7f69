"""Pins of the oracle's optimisers against an independent maximiser: scipy's
bounded L-BFGS-B over log branch lengths, using only the oracle's
log-likelihood (itself pinned by brute-force summation).

* On four taxa the five branches an NNI touches are the whole tree, so the
  five-branch proposal of a neighbour (sweeps uncapped) is the maximum of that
  neighbour's likelihood over all its lengths.
* On five and six taxa the full optimisation reaches the maximum over all
  2n-3 lengths.
"""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import synth

scipy_opt = pytest.importorskip("scipy.optimize")
LO, HI = np.log(1e-6), np.log(100.0)


def _max_lnl(pb, edges, starts):
    """Best of several L-BFGS-B runs on -lnL(exp(x)), x within the length bounds."""
    best = -np.inf
    for x0 in starts:
        r = scipy_opt.minimize(lambda x: -pb.loglik(edges, np.exp(x)), np.log(x0), method="L-BFGS-B",
                               bounds=[(LO, HI)] * len(x0), options={"ftol": 1e-15, "gtol": 1e-9, "maxiter": 2000})
        best = max(best, -r.fun)
    return best


def _problem(n, sites, seed):
    a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.15)
    tips, w = synth.compress_patterns(a.codes)
    return a, oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_quartet_proposal_is_the_neighbours_maximum(seed):
    a, pb = _problem(4, 400, seed)
    pb.settings(prop_max_sweeps=64)
    lnl, lens, _ = pb.full_optimise(a.tree_edges, np.full(5, 0.1))
    nbe, nbl, _ = oracle.nni_neighbours(4, a.tree_edges, lens)
    assert len(nbe) == 2
    rng = np.random.default_rng(seed)
    for k in range(2):
        lp, pe, plen = pb.propose(a.tree_edges, lens, k)
        want = _max_lnl(pb, nbe[k], [nbl[k], np.full(5, 0.1), rng.exponential(0.2, 5) + 1e-3])
        assert lp >= want - 1e-6, (k, lp, want)
        assert lp <= want + 1e-6  # scipy's result is a lower bound of the true maximum too
        assert lp == pytest.approx(pb.loglik(pe, plen), abs=1e-9)
        lf, _, _ = pb.full_optimise(nbe[k], nbl[k])
        assert lp == pytest.approx(lf, abs=1e-6)


@pytest.mark.parametrize("n,seed", [(5, 51), (6, 61)])
def test_full_optimisation_reaches_the_maximum(n, seed):
    a, pb = _problem(n, 300, seed)
    rng = np.random.default_rng(seed)
    for e in [a.tree_edges, synth.random_trees(n, 1, seed)[0][0]]:
        lf, lens, _ = pb.full_optimise(e, np.full(2 * n - 3, 0.1))
        want = _max_lnl(pb, e, [lens, np.full(2 * n - 3, 0.1), rng.exponential(0.2, 2 * n - 3) + 1e-3])
        assert lf >= want - 1e-6, (lf, want)
        assert lf == pytest.approx(pb.loglik(e, lens), abs=1e-9)
