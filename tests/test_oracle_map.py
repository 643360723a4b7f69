"""Pins of the oracle's MAP objective (an Exponential(rate) prior on every
branch length; "Phylogenetic Topographer", its optional branch-length prior,
with the Exponential(10) prior of the paper's golden runs).

Independent references: a closed-form two-taxon JC69 likelihood whose MAP
distance is found by scipy's brentq on its derivative, the rate -> 0 limit
(maximum likelihood), and stationarity of the penalised objective.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1811_11007_gb300 import synth


def _two_taxon(sites, diff, seed):
    rng = np.random.default_rng(seed)
    s0 = rng.integers(0, 4, sites).astype(np.uint8)
    s1 = s0.copy()
    idx = rng.choice(sites, diff, replace=False)
    s1[idx] = (s1[idx] + rng.integers(1, 4, diff)) % 4
    tips = np.stack([s0, s1, np.full(sites, 4, np.uint8)])
    ptn, w = synth.compress_patterns(tips)
    return oracle.Problem(ptn, w, np.ones(6), np.full(4, 0.25), 1.0, 1)


@pytest.mark.parametrize("sites,diff,rate", [(500, 40, 10.0), (1000, 150, 10.0), (800, 60, 50.0)])
def test_map_two_taxon_closed_form(sites, diff, rate):
    # Third leaf all gaps: lnL depends on d = t0 + t1 only, its pendant length t2
    # only enters the prior (pushed to the lower bound); the MAP d solves
    # dlnL/dd = rate with lnL(d) = (s - k) ln(1/4 + 3/4 e) + k ln(1/4 - 1/4 e) + const, e = exp(-4d/3).
    pb = _two_taxon(sites, diff, sites + diff)
    pb.set_prior(rate)
    edges = np.array([[0, 3], [1, 3], [2, 3]], np.int32)
    score, lens, _ = pb.full_optimise(edges, np.full(3, 0.1))

    def g(d):
        e = math.exp(-4 * d / 3)
        return (sites - diff) * (-e / (0.25 + 0.75 * e)) + diff * (4 * e / 3) / (1 - e) - rate

    d_ml = -0.75 * math.log(1 - 4 * (diff / sites) / 3)
    d_map = brentq(g, 1e-9, d_ml, xtol=1e-14)
    assert d_map < d_ml
    assert lens[0] + lens[1] == pytest.approx(d_map, rel=1e-6, abs=3e-6)
    assert lens[2] == pytest.approx(1e-6, abs=2e-8)
    e = math.exp(-4 * d_map / 3)
    want_lnl = (sites - diff) * math.log(0.25 * (0.25 + 0.75 * e)) + diff * math.log(0.25 * (0.25 - 0.25 * e))
    lnl = pb.loglik(edges, lens)
    assert lnl == pytest.approx(want_lnl, abs=1e-6)
    assert score == pytest.approx(lnl + 3 * math.log(rate) - rate * float(np.sum(lens)), abs=1e-9)


def test_vanishing_rate_is_maximum_likelihood():
    n = 7
    a = synth.simulate(n, 500, 717, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    l_ml, lens_ml, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    pb.set_prior(1e-12)
    s, lens, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    np.testing.assert_allclose(lens, lens_ml, rtol=1e-6, atol=1e-8)
    assert s - (2 * n - 3) * math.log(1e-12) == pytest.approx(l_ml, abs=1e-6)


@pytest.mark.parametrize("rate", [10.0, 2.0])
def test_map_optimum_is_stationary(rate):
    n = 8
    a = synth.simulate(n, 600, 719, model="gtr", alpha=0.5, mean_branch=0.1)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    pb.set_prior(rate)
    _, lens, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    for e in range(2 * n - 3):
        _, d1, d2 = pb.edge_derivs(a.tree_edges, lens, e)
        g = d1 - rate  # slope of the penalised objective
        if lens[e] <= 1e-6 + 2e-8:
            assert g <= 0 or abs(g / d2) < 1e-5
        else:
            assert d2 < 0 and abs(g / d2) <= 1e-5 * max(1.0, lens[e])
    # every proposal score carries the prior too
    lp, pe, plen = pb.propose(a.tree_edges, lens, 0)
    assert lp == pytest.approx(pb.loglik(pe, plen) + (2 * n - 3) * math.log(rate) - rate * float(np.sum(plen)),
                               abs=1e-9)
