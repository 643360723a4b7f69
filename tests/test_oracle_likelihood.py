"""Pins of the oracle's pruning, branch derivatives, Newton and optimisation.

Independent references: brute-force summation over ancestral states, the
total probability of all site patterns, rerooting invariance, the JC69
two-taxon closed form, finite differences, and stationarity conditions.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import linalg

import oracle
from paper_1811_11007_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "published_constants.json")


def _problem(n, sites, seed, ncat=4, gap_frac=0.0, model="gtr", mean_branch=0.1):
    a = synth.simulate(n, sites, seed, model=model, alpha=0.5 if ncat > 1 else None,
                       gap_frac=gap_frac, mean_branch=mean_branch)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, ncat)
    return a, tips, w, pb


def _brute_site_lik(n, edges, lengths, tips, Q, rates, freqs):
    """Sum over every assignment of states to the inner nodes (and to gap
    leaves) of pi(root) * prod over edges of P(t)[parent][child]."""
    nn = 2 * n - 2
    adj = [[] for _ in range(nn)]
    for k, (a, b) in enumerate(edges):
        adj[a].append((b, lengths[k]))
        adj[b].append((a, lengths[k]))
    root = n
    order, par = [], {root: (-1, 0.0)}
    stack = [root]
    while stack:
        v = stack.pop()
        order.append(v)
        for c, t in adj[v]:
            if c not in par:
                par[c] = (v, t)
                stack.append(c)
    inner = list(range(n, nn))
    P = tips.shape[1]
    out = np.zeros(P)
    for r in rates:
        Pm = {v: linalg.expm(Q * r * par[v][1]) for v in order if v != root}
        tot = np.zeros(P)
        for assign in itertools.product(range(4), repeat=len(inner)):
            st = dict(zip(inner, assign))
            base = freqs[st[root]] * np.prod([Pm[v][st[par[v][0]], st[v]] for v in inner if v != root])
            leafp = np.ones(P)
            for leaf in range(n):
                pv = st[par[leaf][0]]
                codes = tips[leaf]
                row = Pm[leaf][pv]
                leafp *= np.where(codes < 4, row[np.minimum(codes, 3)], 1.0)
            tot += base * leafp
        out += tot / len(rates)
    return out


@pytest.mark.parametrize("n,seed,ncat,gap", [(4, 11, 4, 0.0), (5, 12, 4, 0.1), (5, 13, 1, 0.0)])
def test_pruning_matches_brute_force(n, seed, ncat, gap):
    a, tips, w, pb = _problem(n, 60, seed, ncat=ncat, gap_frac=gap)
    Q, rates = pb.model()
    lnl, site = pb.loglik(a.tree_edges, a.tree_lengths, per_site=True)
    want = _brute_site_lik(n, a.tree_edges, a.tree_lengths, tips, Q, rates, a.freqs)
    np.testing.assert_allclose(site, np.log(want), rtol=1e-12, atol=1e-12)
    assert lnl == pytest.approx(float(np.sum(w * np.log(want))), rel=1e-12)


@pytest.mark.parametrize("n", [4, 5])
def test_all_site_patterns_sum_to_one(n):
    a, _, _, _ = _problem(n, 10, 20 + n)
    tips = np.array(list(itertools.product(range(4), repeat=n)), np.uint8).T.copy()
    pb = oracle.Problem(tips, np.ones(tips.shape[1]), a.exch, a.freqs, 0.5, 4)
    _, site = pb.loglik(a.tree_edges, a.tree_lengths, per_site=True)
    assert np.exp(site).sum() == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("n,seed", [(7, 31), (12, 32)])
def test_reroot_invariance(n, seed):
    a, _, _, pb = _problem(n, 300, seed, gap_frac=0.05)
    vals = [pb.loglik(a.tree_edges, a.tree_lengths, root=r) for r in range(n, 2 * n - 2)]
    np.testing.assert_allclose(vals, vals[0], rtol=1e-13)


def test_deep_tree_rescaling_is_exact():
    # Long branches on 60 taxa drive every vector below 2^-256 several times;
    # the per-site scaling must leave the log-likelihood continuous and equal
    # under rerooting.
    a, _, _, pb = _problem(60, 200, 41, mean_branch=2.0)
    vals = [pb.loglik(a.tree_edges, a.tree_lengths, root=r) for r in (60, 80, 117)]
    assert np.isfinite(vals[0])
    np.testing.assert_allclose(vals, vals[0], rtol=1e-13)


@pytest.mark.parametrize("sites,diff", json.load(open(GOLDEN))["jc69_two_taxon"]["cases"])
def test_jc69_two_taxon_closed_form(sites, diff):
    # Three leaves, the third all gaps: the likelihood depends only on the sum
    # of the two remaining pendant lengths, which must reach the JC69 ML
    # distance d = -3/4 ln(1 - 4p/3).
    rng = np.random.default_rng(sites + diff)
    s0 = rng.integers(0, 4, sites).astype(np.uint8)
    s1 = s0.copy()
    idx = rng.choice(sites, diff, replace=False)
    s1[idx] = (s1[idx] + rng.integers(1, 4, diff)) % 4
    tips = np.stack([s0, s1, np.full(sites, 4, np.uint8)])
    ptn, w = synth.compress_patterns(tips)
    pb = oracle.Problem(ptn, w, np.ones(6), np.full(4, 0.25), 1.0, 1)
    edges = np.array([[0, 3], [1, 3], [2, 3]], np.int32)
    lnl, lens, _ = pb.full_optimise(edges, np.full(3, 0.1))
    p = diff / sites
    d = -0.75 * math.log(1 - 4 * p / 3)
    assert lens[0] + lens[1] == pytest.approx(d, rel=1e-6, abs=3e-6)
    if diff == 0:  # the optimum d = 0 lies below the bound: both lengths at tmin
        np.testing.assert_allclose(lens[:2], 1e-6, atol=1e-8)
        d = lens[0] + lens[1]
    e = math.exp(-4 * d / 3)
    want = (sites - diff) * math.log(0.25 * (0.25 + 0.75 * e)) + (diff * math.log(0.25 * (0.25 - 0.25 * e))
                                                                     if diff else 0.0)
    assert lnl == pytest.approx(want, abs=1e-7)


@pytest.mark.parametrize("seed", [51, 52])
def test_branch_derivatives_match_finite_differences(seed):
    a, _, _, pb = _problem(8, 400, seed, gap_frac=0.02)
    lens = np.array(a.tree_lengths, copy=True)
    for e in range(2 * 8 - 3):
        f, d1, d2 = pb.edge_derivs(a.tree_edges, lens, e)
        t = lens[e]
        assert f == pytest.approx(pb.loglik(a.tree_edges, lens), rel=1e-13)

        def fl(x):
            l2 = lens.copy()
            l2[e] = x
            return pb.loglik(a.tree_edges, l2)
        h = 1e-5 * t
        g = (fl(t + h) - fl(t - h)) / (2 * h)
        assert d1 == pytest.approx(g, rel=1e-5, abs=1e-4)
        h = 1e-3 * t
        hh = (-fl(t + 2 * h) + 16 * fl(t + h) - 30 * f + 16 * fl(t - h) - fl(t - 2 * h)) / (12 * h * h)
        assert d2 == pytest.approx(hh, rel=1e-4, abs=1e-2)


def _stationary(pb, edges, lens, e, tmin=1e-6):
    f, d1, d2 = pb.edge_derivs(edges, lens, e)
    if lens[e] <= tmin + 1e-7:  # within the Newton tolerance of the bound
        return d1 <= 0 or abs(d1 / d2) < 1e-5
    return d2 < 0 and abs(d1 / d2) <= 1e-5 * max(1.0, lens[e])


@pytest.mark.parametrize("n,seed,ncat", [(6, 61, 4), (9, 62, 4), (7, 63, 1)])
def test_full_optimisation_reaches_stationary_point(n, seed, ncat):
    a, _, _, pb = _problem(n, 500, seed, ncat=ncat)
    lnl0 = pb.loglik(a.tree_edges, np.full(2 * n - 3, 0.1))
    lnl, lens, sweeps = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    assert lnl > lnl0
    assert lnl == pytest.approx(pb.loglik(a.tree_edges, lens), abs=1e-9)
    assert sweeps < 64
    for e in range(2 * n - 3):
        # the central-difference slope is an independent check of d1
        t = lens[e]
        h = 1e-6 * max(t, 1e-4)
        l2, l3 = lens.copy(), lens.copy()
        l2[e] = t + h
        l3[e] = max(t - h, 1e-6)
        g = (pb.loglik(a.tree_edges, l2) - pb.loglik(a.tree_edges, l3)) / (l2[e] - l3[e])
        if t > 1e-6 * 1.001:
            f, d1, d2 = pb.edge_derivs(a.tree_edges, lens, e)
            assert abs(g / d2) < 1e-4 * max(t, 1e-3)
        else:
            assert g < 1e-3
        assert _stationary(pb, a.tree_edges, lens, e)


def test_newton_bound_handling():
    # Identical sequences drive every length to the lower bound.
    sites = 200
    s = np.random.default_rng(5).integers(0, 4, sites).astype(np.uint8)
    tips = np.stack([s, s, s, s])
    ptn, w = synth.compress_patterns(tips)
    pb = oracle.Problem(ptn, w, np.ones(6), np.full(4, 0.25), 1.0, 1)
    edges = np.array([[0, 4], [1, 4], [4, 5], [2, 5], [3, 5]], np.int32)
    lnl, lens, _ = pb.full_optimise(edges, np.full(5, 0.3))
    np.testing.assert_allclose(lens, 1e-6, atol=1e-8)  # within the Newton tolerance of the bound
    assert pb.counter(1) == 0  # every Newton converged
