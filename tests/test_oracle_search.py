"""Pins of the oracle's NNI neighbourhoods, split-set keys and PT search.

Independent references: the (2n-5)!! count of unrooted binary topologies,
the definition of NNI (one split replaced, 2(n-3) distinct neighbours,
symmetric), key invariance under relabelling, injectivity checked against
exact split sets, and the search rules re-checked on the search's output.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "published_constants.json")
COUNTS = {int(k): v for k, v in json.load(open(GOLDEN))["unrooted_topology_counts"].items() if k[0] != "_"}
M128 = (1 << 128) - 1


def _k(pair):
    return int(pair[0]) | (int(pair[1]) << 64)


def _splitset(n, edges):
    return frozenset(_k(s) for s in oracle.tree_splits(n, edges))


@pytest.mark.parametrize("n,seed", [(5, 1), (7, 2), (16, 3), (70, 4), (128, 5)])
def test_nni_neighbourhood(n, seed):
    rng = np.random.default_rng(seed)
    e = synth.random_topology(n, rng)
    lens = rng.exponential(0.1, 2 * n - 3)
    nbe, nbl, nbk = oracle.nni_neighbours(n, e, lens)
    assert len(nbe) == 2 * (n - 3)
    parent = _splitset(n, e)
    pkey = _k(oracle.tree_key(n, e))
    keys = {_k(k) for k in nbk}
    assert len(keys) == 2 * (n - 3) and pkey not in keys
    for i in range(len(nbe)):
        s = _splitset(n, nbe[i])
        # exactly one split replaced (Robinson-Foulds distance 2)
        assert len(s - parent) == 1 and len(parent - s) == 1
        # key is the sum of split hashes: the incremental update is exact
        old, new = next(iter(parent - s)), next(iter(s - parent))
        ho = oracle.split_hash(old & ((1 << 64) - 1), old >> 64)
        hn = oracle.split_hash(new & ((1 << 64) - 1), new >> 64)
        assert (pkey - _k(ho) + _k(hn)) & M128 == _k(nbk[i])
        assert _k(oracle.tree_key(n, nbe[i])) == _k(nbk[i])
        # every branch keeps its length (the multiset of lengths is unchanged)
        np.testing.assert_allclose(np.sort(nbl[i]), np.sort(lens))
        if n <= 16:
            # symmetry: the parent is an NNI neighbour of its neighbour
            _, _, back = oracle.nni_neighbours(n, nbe[i], nbl[i])
            assert pkey in {_k(k) for k in back}
    # splits are normalised to the side without taxon 0
    for s in parent:
        assert not (s & 1)


@pytest.mark.parametrize("n,seed", [(6, 7), (40, 8), (128, 9)])
def test_key_invariant_under_relabelling(n, seed):
    rng = np.random.default_rng(seed)
    e = synth.random_topology(n, rng)
    k = oracle.tree_key(n, e)
    for _ in range(5):
        assert oracle.tree_key(n, synth.relabel_inner(e, n, rng)) == k


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_infinite_threshold_visits_every_topology(n):
    a = synth.simulate(n, 300, 100 + n, model="jc", alpha=None)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 1.0, 1)
    e, l = synth.random_trees(n, 1, 7 + n)
    s = oracle.Search(pb, e, l, np.inf)
    s.run()
    v = s.visited(with_trees=True)
    assert len(v["keys"]) == COUNTS[n]
    assert not s.collision
    # keys distinct, split sets distinct, stored keys equal recomputed keys
    assert len({_k(k) for k in v["keys"]}) == COUNTS[n]
    assert len({_splitset(n, t) for t in v["edges"]}) == COUNTS[n]
    for k, t in zip(v["keys"], v["edges"]):
        assert _k(oracle.tree_key(n, t)) == _k(k)
    # at T = inf everything visited is GOOD
    assert np.all(v["status"] == oracle.GOOD)


def _rules_hold(n, T, v, starts):
    """Re-derives the round rules from the search output alone."""
    rounds = v["round"]
    lnl, plnl, st = v["lnl"], v["plnl"], v["status"]
    visited = st != oracle.REJECTED
    for r in range(1, rounds.max() + 1):
        prior = visited & (rounds < r)
        lmax0 = lnl[prior].max()
        here = rounds == r
        assert np.all(plnl[here & (st == oracle.REJECTED)] < lmax0 - T)
        kept = here & visited
        assert np.all(plnl[kept] >= lmax0 - T)
        lmax1 = max(lmax0, lnl[kept].max()) if kept.any() else lmax0
        assert np.all(lnl[here & (st == oracle.GOOD)] >= lmax1 - T)
        assert np.all(lnl[here & (st == oracle.BAD)] < lmax1 - T)
        # every topology of round r is an NNI neighbour of a GOOD one of round r-1
        parents = np.nonzero((rounds == r - 1) & (st == oracle.GOOD))[0]
        reach = set()
        for p in parents:
            _, _, nk = oracle.nni_neighbours(n, v["edges"][p], v["lengths"][p])
            reach |= {_k(k) for k in nk}
        for i in np.nonzero(here)[0]:
            assert _k(v["keys"][i]) in reach


@pytest.mark.parametrize("T", [0.0, 2.0, 6.0])
def test_finite_threshold_rules_and_brute_force(T):
    n = 6
    a = synth.simulate(n, 400, 606, model="gtr", alpha=0.5, mean_branch=0.15)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    # brute force: every topology, fully optimised
    e, l = synth.random_trees(n, 1, 3)
    full = oracle.Search(pb, e, l, np.inf)
    full.run()
    fv = full.visited()
    brute = {_k(k): x for k, x in zip(fv["keys"], fv["lnl"])}
    best = max(brute.values())
    # PT from the generating tree, hill-climbed
    lhc, he, hl, _ = pb.hill_climb(a.tree_edges, np.full(2 * n - 3, 0.1))
    s = oracle.Search(pb, he[None], hl[None], T)
    s.run()
    v = s.visited(with_trees=True)
    _rules_hold(n, T, v, he)
    vis = v["status"] != oracle.REJECTED
    for k, x in zip(v["keys"][vis], v["lnl"][vis]):
        assert x == pytest.approx(brute[_k(k)], abs=1e-6)
    assert s.lmax == pytest.approx(best, abs=1e-6)
    # post-filtered HLS = visited topologies within T of the final best, a
    # subset of the brute-force HLS
    hls = {_k(k) for k, x, g in zip(v["keys"], v["lnl"], vis) if g and x >= s.lmax - T}
    bhls = {k for k, x in brute.items() if x >= best - T}
    assert hls <= bhls
    assert _k(oracle.tree_key(n, he)) in hls
    # proposal lnL never exceeds the full optimum of the same topology
    for k, p in zip(v["keys"], v["plnl"]):
        if np.isfinite(p):
            assert p <= brute[_k(k)] + 1e-6


def test_proposal_touches_only_five_branches():
    n = 9
    a = synth.simulate(n, 500, 909, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    lnl, lens, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    nbe, nbl, _ = oracle.nni_neighbours(n, a.tree_edges, lens)
    for k in range(len(nbe)):
        lp, pe, plen = pb.propose(a.tree_edges, lens, k)
        np.testing.assert_array_equal(pe, nbe[k])
        changed = np.nonzero(np.abs(plen - nbl[k]) > 0)[0]
        assert len(changed) <= 5
        assert lp >= pb.loglik(nbe[k], nbl[k]) - 1e-9
        assert lp == pytest.approx(pb.loglik(pe, plen), abs=1e-9)
        # the changed branches are incident to the ends of the new inner edge
        # (the one whose split is not in the parent)
        psplits = _splitset(n, a.tree_edges)
        new_split = next(iter(_splitset(n, pe) - psplits))
        ends = None
        for x, y in pe:
            if x >= n and y >= n:
                # the split of edge (x, y): leaves reachable from y without x
                adj = {}
                for u, v in pe:
                    adj.setdefault(int(u), []).append(int(v))
                    adj.setdefault(int(v), []).append(int(u))
                seen, stack = {int(x), int(y)}, [int(y)]
                leaves = 0
                while stack:
                    c = stack.pop()
                    if c < n:
                        leaves |= 1 << c
                    for d in adj[c]:
                        if d not in seen:
                            seen.add(d)
                            stack.append(d)
                if leaves & 1:
                    leaves = ((1 << n) - 1) ^ leaves
                if leaves == new_split:
                    ends = {int(x), int(y)}
        assert ends is not None
        for i in changed:
            assert ends & {int(pe[i][0]), int(pe[i][1])}
    # radius 0: only the central branch moves
    pb.settings(prop_mode=1)
    for k in range(len(nbe)):
        lp, pe, plen = pb.propose(a.tree_edges, lens, k)
        assert np.count_nonzero(np.abs(plen - nbl[k]) > 0) <= 1


@pytest.mark.parametrize("n,seed", [(10, 4), (8, 5)])
def test_hill_climb_stop_rule(n, seed):
    """The hill-climb's result re-checked against its rules: it starts from the
    full optimisation, each move gains, the final lengths are a full optimum,
    and at the final tree the neighbour with the best proposal score (ties: the
    smallest key), fully optimised from its proposal lengths, gains <= 1e-6."""
    a = synth.simulate(n, 600, 1000 + seed, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    e, l = synth.random_trees(n, 1, seed)
    l0, _, _ = pb.full_optimise(e[0], l[0])
    lhc, he, hl, moves = pb.hill_climb(e[0], l[0])
    assert moves >= 1  # a random start is improved at least once
    assert lhc > l0 + 1e-6 * moves
    assert lhc == pytest.approx(pb.loglik(he, hl), abs=1e-8)
    assert pb.full_optimise(he, hl)[0] == pytest.approx(lhc, abs=1e-7)
    _, _, nk = oracle.nni_neighbours(n, he, hl)
    best = max(range(len(nk)), key=lambda k: (pb.propose(he, hl, k)[0], -_k(nk[k])))
    _, be, bl = pb.propose(he, hl, best)
    assert pb.full_optimise(be, bl)[0] <= lhc + 1e-6


def test_full_radius_proposal_is_full_optimisation():
    """prop_mode 2 (the paper's radius -1): the proposal of a neighbour is the
    full optimisation of that neighbour from its inherited lengths."""
    n = 8
    a = synth.simulate(n, 400, 919, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    lnl, lens, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    nbe, nbl, _ = oracle.nni_neighbours(n, a.tree_edges, lens)
    pb.settings(prop_mode=2)
    for k in range(len(nbe)):
        lp, pe, plen = pb.propose(a.tree_edges, lens, k)
        lf, lensf, _ = pb.full_optimise(nbe[k], nbl[k])
        np.testing.assert_array_equal(pe, nbe[k])
        assert lp == pytest.approx(lf, abs=1e-9)
        np.testing.assert_allclose(plen, lensf, rtol=1e-7, atol=1e-9)
        # no branch of a fully optimised neighbour can improve alone: the Newton
        # step -d1/d2 it would take is within the sweep tolerance's reach
        for e in range(2 * n - 3):
            _, d1, d2 = pb.edge_derivs(pe, plen, e)
            assert abs(d1 / d2) < 1e-5 or (plen[e] <= 1e-6 + 2e-8 and d1 < 0)  # at the bound (Newton tol 1e-8)


def test_full_radius_infinite_threshold_visits_every_topology():
    n = 6
    a = synth.simulate(n, 300, 921, model="jc")
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 1.0, 1)
    pb.settings(prop_mode=2)
    e, l = synth.random_trees(n, 1, 922)
    s = oracle.Search(pb, e, l, float("inf"))
    s.run()
    assert len(s.visited()["keys"]) == COUNTS[n]


def test_min_proposer_arbitration():
    """Within a round, a neighbour proposed by several frontier trees is scored
    once, from the proposer with the smallest (parent key, split of the
    rearranged edge, swap): the round-synchronous reading of the paper's "if
    unvisited" check ("Phylogenetic Topographer", loop step 6).  Re-derived
    from the output: every proposer of each scored key is re-enumerated from
    the previous round's GOOD trees, the recorded winner must be the
    lexicographic minimum, and the stored proposal score and (for rejected
    neighbours) lengths must be the proposal optimisation from that winner's
    inherited lengths -- which differ between proposers, so scoring from any
    other proposer fails the check."""
    n, T = 8, 15.0
    a = synth.simulate(n, 400, 808, model="gtr", alpha=0.5, mean_branch=0.1)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    e, l = synth.random_trees(n, 12, 809)
    s = oracle.Search(pb, e, l, T)
    for _ in range(3):
        if s.frontier_size:
            s.round()
    v = s.visited(with_trees=True)
    pr = s.proposers()
    assert np.all(pr["swap"][v["round"] == 0] == -1)
    contested = distinct_scores = 0
    for r in range(1, int(v["round"].max()) + 1):
        parents = np.nonzero((v["round"] == r - 1) & (v["status"] == oracle.GOOD))[0]
        cands = {}
        for p in parents:
            pe, pl = v["edges"][p], v["lengths"][p]
            splits = sorted(_k(x) for x in oracle.tree_splits(n, pe))  # canonical edge order: ascending split
            _, _, nk = oracle.nni_neighbours(n, pe, pl)
            for k in range(len(nk)):
                cands.setdefault(_k(nk[k]), []).append((_k(v["keys"][p]), splits[k // 2], k % 2, p, k))
        for i in np.nonzero(v["round"] == r)[0]:
            cs = cands[_k(v["keys"][i])]
            win = min(cs)
            assert (_k(pr["parent_key"][i]), _k(pr["split"][i]), int(pr["swap"][i])) == win[:3]
            lp, _, plen = pb.propose(v["edges"][win[3]], v["lengths"][win[3]], win[4])
            assert v["plnl"][i] == pytest.approx(lp, abs=1e-9)
            if v["status"][i] == oracle.REJECTED:
                np.testing.assert_allclose(v["lengths"][i], plen, rtol=1e-12, atol=0)
            others = [c for c in cs if c[:3] != win[:3]]
            if others:
                contested += 1
                lo = pb.propose(v["edges"][others[0][3]], v["lengths"][others[0][3]], others[0][4])[0]
                distinct_scores += abs(lo - lp) > 1e-6
    # the case must exercise the rule: keys with several proposers whose scores differ
    assert contested >= 5 and distinct_scores >= 3, (contested, distinct_scores)
