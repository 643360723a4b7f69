"""GPU path vs the FP64 oracle, through the C ABI (libpt.so).

Tolerances: FP64 path |dlnL| <= 1e-8 nats, mixed precision |dlnL| <= 1e-3
nats (absolute, at every size); branch lengths within 1e-4 relative (1e-6
absolute near the lower bound).  Keys and visited
sets are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "mixed": 1e-3}


def _tol(prec, lnl):
    return TOL[prec]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _setup(n, sites, seed, ncat=4, model="gtr", gap=0.0, mean_branch=0.1, alpha=0.5):
    a = synth.simulate(n, sites, seed, model=model, alpha=alpha if ncat > 1 else None, gap_frac=gap,
                       mean_branch=mean_branch)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, alpha, ncat)
    return a, pb


def _ctx(prec, a, ncat, alpha=0.5, **kw):
    ctx = pt.Context(precision=prec, **kw)
    aid = ctx.load_alignment(a.codes)
    ctx.set_model(aid, a.exch, a.freqs, alpha, ncat)
    return ctx, aid


def _split_lengths(n, edges, lengths):
    """split (side without taxon 0, as an int bitmask) -> length."""
    adj = {}
    for (x, y), l in zip(np.asarray(edges).reshape(-1, 2), lengths):
        adj.setdefault(int(x), []).append((int(y), float(l)))
        adj.setdefault(int(y), []).append((int(x), float(l)))
    full = (1 << n) - 1
    out = {}
    for (x, y), l in zip(np.asarray(edges).reshape(-1, 2), lengths):
        seen, stack, leaves = {int(x), int(y)}, [int(y)], 0
        while stack:
            c = stack.pop()
            if c < n:
                leaves |= 1 << c
            for d, _ in adj[c]:
                if d not in seen:
                    seen.add(d)
                    stack.append(d)
        if leaves & 1:
            leaves = full ^ leaves
        out[leaves] = float(l)
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,sites,ncat,gap", [(7, 500, 1, 0.0), (12, 400, 4, 0.05), (27, 600, 4, 0.0)])
def test_fixed_lnl_and_keys(prec, n, sites, ncat, gap):
    a, pb = _setup(n, sites, 100 + n, ncat=ncat, model="gtr" if ncat > 1 else "jc", gap=gap)
    e, _ = synth.random_trees(n, 6, 7)
    rng = np.random.default_rng(3)
    lens = rng.exponential(0.1, e.shape[:2])
    e = np.concatenate([e, a.tree_edges[None]])
    lens = np.concatenate([lens, a.tree_lengths[None]])
    ctx, aid = _ctx(prec, a, ncat)
    lnl, l2, keys = ctx.score(aid, e, lens, mode="fixed")
    np.testing.assert_array_equal(l2, lens)
    for i in range(len(e)):
        want = pb.loglik(e[i], lens[i])
        assert abs(lnl[i] - want) <= _tol(prec, want), (i, lnl[i], want)
        assert pt.keys_to_int(keys[i])[0] == (lambda k: k[0] | (k[1] << 64))(oracle.tree_key(n, e[i]))
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,sites,ncat", [(5, 300, 1), (9, 500, 4), (20, 800, 4)])
def test_full_optimisation(prec, n, sites, ncat):
    a, pb = _setup(n, sites, 200 + n, ncat=ncat, model="gtr" if ncat > 1 else "jc")
    e, l = synth.random_trees(n, 4, 11)
    e = np.concatenate([e, a.tree_edges[None]])
    l = np.concatenate([l, np.full((1, 2 * n - 3), 0.1)])
    ctx, aid = _ctx(prec, a, ncat)
    lnl, lens, _ = ctx.score(aid, e, l, mode="full")
    for i in range(len(e)):
        want, wl, _ = pb.full_optimise(e[i], l[i])
        assert abs(lnl[i] - want) <= _tol(prec, want), (i, lnl[i], want)
        assert abs(pb.loglik(e[i], lens[i]) - lnl[i]) <= _tol(prec, want)
        if prec == "fp64":
            np.testing.assert_allclose(lens[i], wl, rtol=1e-4, atol=1e-6)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_infinite_threshold_visits_945(prec):
    # 7 taxa, 500 sites, JC69, lengths from 0.1, T = inf: every one of the
    # (2n-5)!! = 945 topologies is visited exactly once
    a, pb = _setup(7, 500, synth.SEED_BASE + 1, ncat=1, model="jc", mean_branch=0.1)
    e, l = synth.random_trees(7, 1, 5)
    ctx, aid = _ctx(prec, a, 1, table_log2=14)
    lmax, rounds = pt.run_search(ctx, aid, e, l, np.inf)
    vis = ctx.visited(aid)
    s = oracle.Search(pb, e, l, np.inf)
    s.run()
    ov = s.visited()
    gk = pt.keys_to_int(vis["keys"])
    ok = pt.keys_to_int(ov["keys"])
    assert len(gk) == 945 and set(gk) == set(ok)
    assert np.all(vis["status"] == pt.ST_GOOD)
    want = dict(zip(ok, ov["lnl"]))
    for k, x in zip(gk, vis["lnl"]):
        assert abs(x - want[k]) <= _tol(prec, x), (k, x, want[k])
    assert abs(lmax - s.lmax) <= _tol(prec, lmax)
    ctx.close()


def _margins(ov, T):
    """Distance of each oracle decision from its threshold (round by round)."""
    rounds, st, lnl, plnl = ov["round"], ov["status"], ov["lnl"], ov["plnl"]
    visited = st != oracle.REJECTED
    m = []
    for r in range(1, rounds.max() + 1):
        lmax0 = lnl[visited & (rounds < r)].max()
        here = rounds == r
        m += list(np.abs(plnl[here] - (lmax0 - T)))
        kept = here & visited
        lmax1 = max(lmax0, lnl[kept].max()) if kept.any() else lmax0
        m += list(np.abs(lnl[kept] - (lmax1 - T)))
    return np.array(m)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,sites,T,seed", [(8, 400, 3.0, 31), (10, 600, 2.0, 32), (12, 300, 4.0, 33)])
def test_finite_threshold_search_matches_oracle(prec, n, sites, T, seed):
    a, pb = _setup(n, sites, seed, ncat=4)
    e, l = synth.random_trees(n, 3, seed + 1)
    s = oracle.Search(pb, e, l, T)
    s.run()
    ov = s.visited()
    margin = _margins(ov, T).min()
    if margin < 10 * TOL[prec]:
        pytest.skip(f"decision within {margin:.2e} of the threshold: ambiguous at {prec} tolerance")
    ctx, aid = _ctx(prec, a, 4, table_log2=16)
    lmax, rounds = pt.run_search(ctx, aid, e, l, T)
    vis = ctx.visited(aid)
    gd = dict(zip(pt.keys_to_int(vis["keys"]), zip(vis["status"], vis["lnl"])))
    od = dict(zip(pt.keys_to_int(ov["keys"]), zip(ov["status"], ov["lnl"])))
    assert set(gd) == set(od)
    for k, (st, x) in od.items():
        assert gd[k][0] == st, (k, gd[k], st)
        assert abs(gd[k][1] - x) <= _tol(prec, x)
    assert abs(lmax - s.lmax) <= _tol(prec, lmax)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["five", "central", "full"])
def test_proposals_match_oracle(prec, mode):
    n = 11
    a, pb = _setup(n, 700, 41, ncat=4)
    pb.settings(prop_mode={"five": 0, "central": 1, "full": 2}[mode])
    e, l = synth.random_trees(n, 2, 42)
    ctx, aid = _ctx(prec, a, 4, table_log2=14, propose=mode)
    lmax, front = ctx.begin(aid, e, l, np.inf)
    lmax2, nxt = ctx.expand(aid, front["edges"], front["lengths"], np.inf, lmax)
    props = ctx.last_proposals()
    assert len(props["keys"]) > 0
    full = (1 << n) - 1
    for i in range(len(props["keys"])):
        f = props["parent"][i]
        pe, plen = front["edges"][f], front["lengths"][f]
        _, _, nk = oracle.nni_neighbours(n, pe, plen)
        kk = pt.keys_to_int(props["keys"][i])[0]
        k = [j for j, x in enumerate(pt.keys_to_int(nk)) if x == kk]
        assert len(k) == 1
        lp, nbe, nbl = pb.propose(pe, plen, k[0])
        assert abs(props["lnl"][i] - lp) <= _tol(prec, lp), (i, props["lnl"][i], lp)
        if prec != "fp64" or mode == "full":  # full radius: len5 holds the inherited lengths
            continue
        # the five lengths by split: central, A, B, C, D
        up = {int(x): int(y) for x, y in pe}
        below = {}
        for leaf in range(n):
            x = leaf
            while x in up and x != 0:
                below[x] = below.get(x, 0) | (1 << leaf)
                x = up[x]
        v = int(props["edge_node"][i])
        u = up[v]
        kids = lambda x: sorted([c for c, p in up.items() if p == x], key=lambda c: (below[c] & -below[c]))
        sib = [c for c in kids(u) if c != v][0]
        c0, c1 = kids(v)
        B, Cc, D = below[sib], below[c0], below[c1]
        A_split = B | Cc | D
        central = B | (D if props["swap"][i] == 0 else Cc)
        sl = _split_lengths(n, nbe, nbl)
        want = [sl[central], sl[A_split], sl[B], sl[Cc], sl[D]]
        np.testing.assert_allclose(props["len5"][i], want, rtol=1e-4, atol=1e-6)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_radius_search_matches_oracle(prec):
    """Radius -1 proposals (every branch optimised before the keep decision)."""
    n, sites, T, seed = 8, 400, 3.0, 35
    a, pb = _setup(n, sites, seed, ncat=4)
    pb.settings(prop_mode=2)
    e, l = synth.random_trees(n, 3, seed + 1)
    s = oracle.Search(pb, e, l, T)
    s.run()
    ov = s.visited()
    margin = _margins(ov, T).min()
    if margin < 10 * TOL[prec]:
        pytest.skip(f"decision within {margin:.2e} of the threshold: ambiguous at {prec} tolerance")
    ctx, aid = _ctx(prec, a, 4, table_log2=16, propose="full")
    lmax, rounds = pt.run_search(ctx, aid, e, l, T)
    vis = ctx.visited(aid)
    gd = dict(zip(pt.keys_to_int(vis["keys"]), zip(vis["status"], vis["lnl"])))
    od = dict(zip(pt.keys_to_int(ov["keys"]), zip(ov["status"], ov["lnl"])))
    assert set(gd) == set(od)
    for k, (st, x) in od.items():
        assert gd[k][0] == st, (k, gd[k], st)
        assert abs(gd[k][1] - x) <= _tol(prec, x)
    assert abs(lmax - s.lmax) <= _tol(prec, lmax)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_map_scoring_matches_oracle(prec):
    """MAP objective (Exponential(10) prior on every length): fixed and fully
    optimised scores and the MAP lengths against the oracle."""
    import math
    n, rate = 10, 10.0
    a, pb = _setup(n, 600, 301, ncat=4)
    pb.set_prior(rate)
    e, l = synth.random_trees(n, 4, 302)
    ctx, aid = _ctx(prec, a, 4, branch_prior_rate=rate)
    fixed, _, _ = ctx.score(aid, e, l, mode="fixed")
    lnl, lens, _ = ctx.score(aid, e, l, mode="full")
    for i in range(len(e)):
        want_fixed = pb.loglik(e[i], l[i]) + (2 * n - 3) * math.log(rate) - rate * float(np.sum(l[i]))
        assert abs(fixed[i] - want_fixed) <= _tol(prec, want_fixed)
        want, wl, _ = pb.full_optimise(e[i], l[i])
        assert abs(lnl[i] - want) <= _tol(prec, want), (i, lnl[i], want)
        if prec == "fp64":
            np.testing.assert_allclose(lens[i], wl, rtol=1e-4, atol=1e-6)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_map_search_matches_oracle(prec):
    n, sites, T, seed, rate = 9, 500, 3.0, 303, 10.0
    a, pb = _setup(n, sites, seed, ncat=4)
    pb.set_prior(rate)
    e, l = synth.random_trees(n, 3, seed + 1)
    s = oracle.Search(pb, e, l, T)
    s.run()
    ov = s.visited()
    margin = _margins(ov, T).min()
    if margin < 10 * TOL[prec]:
        pytest.skip(f"decision within {margin:.2e} of the threshold: ambiguous at {prec} tolerance")
    ctx, aid = _ctx(prec, a, 4, table_log2=16, branch_prior_rate=rate)
    lmax, rounds = pt.run_search(ctx, aid, e, l, T)
    vis = ctx.visited(aid)
    gd = dict(zip(pt.keys_to_int(vis["keys"]), zip(vis["status"], vis["lnl"])))
    od = dict(zip(pt.keys_to_int(ov["keys"]), zip(ov["status"], ov["lnl"])))
    assert set(gd) == set(od)
    for k, (st, x) in od.items():
        assert gd[k][0] == st, (k, gd[k], st)
        assert abs(gd[k][1] - x) <= _tol(prec, x)
    assert abs(lmax - s.lmax) <= _tol(prec, lmax)
    ctx.close()


def test_edge_cases():
    # 3 taxa: no internal edge, no neighbour; 4 taxa with gaps; a start given twice
    for n in (3, 4):
        a, pb = _setup(n, 50, 300 + n, ncat=4, gap=0.2)
        ctx, aid = _ctx("fp64", a, 4, table_log2=10)
        e, l = synth.random_trees(n, 1, 1)
        e2 = np.concatenate([e, synth.relabel_inner(e[0], n, np.random.default_rng(0))[None]])
        l2 = np.concatenate([l, l])
        lmax, front = ctx.begin(aid, e2, l2, 1.0)
        assert len(front["edges"]) == 1
        lmax, nxt = ctx.expand(aid, front["edges"], front["lengths"], np.inf, lmax)
        vis = ctx.visited(aid)
        assert len(vis["keys"]) == (1 if n == 3 else 3)
        want, _, _ = pb.full_optimise(e[0], l[0])
        assert abs(front["lnl"][0] - want) < 1e-8
        ctx.close()


def test_invalid_inputs_rejected():
    a, pb = _setup(6, 100, 5, ncat=4)
    ctx, aid = _ctx("fp64", a, 4, table_log2=10)
    e, l = synth.random_trees(6, 1, 1)
    bad = e.copy()
    bad[0, 0] = [0, 1]  # two leaves joined
    with pytest.raises(pt.PTError) as ex:
        ctx.score(aid, bad, l)
    assert ex.value.status == 1
    bad_l = l.copy()
    bad_l[0, 2] = np.nan
    with pytest.raises(pt.PTError):
        ctx.score(aid, e, bad_l)
    with pytest.raises(pt.PTError):
        ctx.set_model(aid, a.exch, [0.5, 0.5, 0.0, 0.0], 0.5, 4)
    with pytest.raises(pt.PTError):
        ctx.load_alignment(np.full((3, 10), 7, np.uint8))
    ctx.close()


def test_table_full_is_reported():
    # 2^10 slots cannot hold the 945 topologies plus probes of n = 7 at T = inf
    # once the table saturates; the probe limit turns into TABLE_FULL, not a hang
    a, pb = _setup(8, 100, 6, ncat=1, model="jc")
    ctx, aid = _ctx("mixed", a, 1, table_log2=10)
    e, l = synth.random_trees(8, 1, 2)
    with pytest.raises(pt.PTError) as ex:
        pt.run_search(ctx, aid, e, l, np.inf)
    assert ex.value.status == 3
    ctx.close()


def _canonical_split(n, edges, v):
    """Leaf set below node v of a canonical edge list (edge k = (k+1, parent of k+1), rooted at leaf 0)."""
    up = {int(x): int(y) for x, y in np.asarray(edges).reshape(-1, 2)}
    s = 0
    for leaf in range(1, n):
        x = leaf
        while x != 0:
            if x == v:
                s |= 1 << leaf
                break
            x = up[x]
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_proposers_match_oracle(prec):
    """The proposer that wins each contested key (smallest parent key, edge split, swap) is the
    oracle's, bit for bit, round by round (the round-synchronous reading of the paper's
    "if unvisited" check)."""
    n, T = 8, 15.0
    a, pb = _setup(n, 400, 808, ncat=4)
    e, l = synth.random_trees(n, 12, 809)
    s = oracle.Search(pb, e, l, T)
    for _ in range(3):
        if s.frontier_size:
            s.round()
    ov = s.visited()
    if _margins(ov, T).min() < 10 * TOL[prec]:
        pytest.skip("a decision within tolerance of the threshold")
    opr = s.proposers()
    want = {}
    for k, r, pk, sp, sw in zip(pt.keys_to_int(ov["keys"]), ov["round"], opr["parent_key"], opr["split"], opr["swap"]):
        if r >= 1:
            want[k] = (int(r), pt.keys_to_int(pk[None])[0], int(sp[0]) | (int(sp[1]) << 64), int(sw))
    ctx, aid = _ctx(prec, a, 4, table_log2=16)
    lmax, front = ctx.begin(aid, e, l, T)
    got, contested = {}, 0
    for r in range(1, 4):
        if not len(front["edges"]):
            break
        pkeys = pt.keys_to_int(front["keys"])
        lmax, nxt = ctx.expand(aid, front["edges"], front["lengths"], T, lmax)
        pr = ctx.last_proposals()
        for kk, f, v, sw in zip(pt.keys_to_int(pr["keys"]), pr["parent"], pr["edge_node"], pr["swap"]):
            got[kk] = (r, pkeys[f], _canonical_split(n, front["edges"][f], int(v)), int(sw))
        contested += ctx.stats()["candidates"] - ctx.stats()["scored"] - ctx.stats()["duplicates"]
        front = nxt
    ctx.close()
    assert got == want
    assert contested > 0  # some keys had several proposers in a round
