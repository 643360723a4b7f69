"""Graph rounds (pt_graph_*): the batched round recorded once as a CUDA graph
and replayed, against the batched round issued kernel by kernel, the oracle,
and the argument checks of the entry points."""
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


def _alignments(k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(8, 41))
        sites = int(rng.integers(200, 1500))
        out.append(synth.simulate(n, sites, seed * 100 + i, model="gtr", alpha=0.5, mean_branch=0.06))
    return out


def _setup(ctx, alns, T, starts=3, seed=50):
    ids, fronts = [], []
    for i, a in enumerate(alns):
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        e, l = synth.random_trees(a.codes.shape[0], starts, seed + i)
        lmax, front = ctx.begin(aid, e, l, T)
        ids.append(aid)
        fronts.append((lmax, front))
    return ids, fronts


def _visited_dict(ctx, aid):
    v = ctx.visited(aid)
    return dict(zip(pt.keys_to_int(v["keys"]), zip(v["status"], v["lnl"])))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_rounds_equal_batched_rounds(prec):
    """Three replays (advancing the frontier on the device) give bit-identical
    next frontiers, lmax and visited tables to three pt_expand_batch rounds."""
    alns = _alignments(5, 31)
    T = 4.0
    cap = 64
    with pt.Context(precision=prec, table_log2=16) as batch, pt.Context(precision=prec, table_log2=16) as gctx:
        ids_b, fronts_b = _setup(batch, alns, T)
        ids_g, fronts_g = _setup(gctx, alns, T)
        g = gctx.graph(ids_g, [cap] * len(alns), [T] * len(alns))
        try:
            nf = [g.set_frontier(k, f["edges"], f["lengths"]) for k, (_, f) in enumerate(fronts_g)]
            lmax_g = [lm for lm, _ in fronts_g]
            for r in range(3):
                res_b = batch.expand_batch([{"aln": aid, "edges": f["edges"], "lengths": f["lengths"],
                                             "threshold": T, "lmax": lm} for aid, (lm, f) in zip(ids_b, fronts_b)])
                lmax_g, n_next = g.run(nf, lmax_g)
                assert gctx.stats()["launches"] > 0
                for k, (lm_b, f_b) in enumerate(res_b):
                    assert lmax_g[k] == lm_b
                    assert n_next[k] == len(f_b["keys"])
                    f_g = g.next(k)
                    np.testing.assert_array_equal(f_g["keys"], f_b["keys"])
                    np.testing.assert_array_equal(f_g["lnl"], f_b["lnl"])
                    np.testing.assert_array_equal(f_g["lengths"], f_b["lengths"])
                    np.testing.assert_array_equal(f_g["edges"], f_b["edges"])
                if max(n_next) > cap:
                    break
                fronts_b = res_b
                nf = g.advance()
            for aid_b, aid_g in zip(ids_b, ids_g):
                assert _visited_dict(batch, aid_b) == _visited_dict(gctx, aid_g)
        finally:
            g.close()


def test_graph_round_matches_oracle():
    alns = _alignments(3, 37)
    T = 3.0
    with pt.Context(precision="fp64", table_log2=16) as ctx:
        ids, fronts = _setup(ctx, alns, T, starts=1, seed=80)
        before = [set(_visited_dict(ctx, aid)) for aid in ids]
        g = ctx.graph(ids, [max(1, len(f["keys"])) for _, f in fronts], [T] * len(ids))
        try:
            nf = [g.set_frontier(k, f["edges"], f["lengths"]) for k, (_, f) in enumerate(fronts)]
            lm_out, _ = g.run(nf, [lm for lm, _ in fronts])
        finally:
            g.close()
        for i, (a, aid, (lm, f)) in enumerate(zip(alns, ids, fronts)):
            tips, w = synth.compress_patterns(a.codes)
            pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
            s = oracle.Search(pb, f["edges"], f["lengths"], T, frontier_lmax=lm)
            s.round()
            ov = s.visited()
            od = dict(zip(pt.keys_to_int(ov["keys"]), zip(ov["status"], ov["lnl"])))
            gd = _visited_dict(ctx, aid)
            assert set(gd) - before[i] == set(od) - before[i]
            for k, (st, x) in od.items():
                if k in before[i]:
                    continue
                assert gd[k][0] == st
                assert abs(gd[k][1] - x) <= 1e-8
            assert abs(lm_out[i] - s.lmax) <= 1e-8


def test_graph_with_learned_start_equals_batched():
    """The warm start (random weights: any prediction is only a starting
    point) enters the graph as in the batched round."""
    alns = _alignments(3, 41)
    T = 4.0
    rng = np.random.default_rng(5)
    w = (rng.standard_normal(pt.MLP_PARAMS) * 0.05).astype(np.float32)
    with pt.Context(precision="mixed", table_log2=16) as batch, pt.Context(precision="mixed", table_log2=16) as gctx:
        for c in (batch, gctx):
            c.mlp_set_weights(w)
            c.mlp_enable(True)
        ids_b, fronts_b = _setup(batch, alns, T)
        ids_g, fronts_g = _setup(gctx, alns, T)
        g = gctx.graph(ids_g, [48] * len(alns), [T] * len(alns))
        try:
            nf = [g.set_frontier(k, f["edges"], f["lengths"]) for k, (_, f) in enumerate(fronts_g)]
            res_b = batch.expand_batch([{"aln": aid, "edges": f["edges"], "lengths": f["lengths"], "threshold": T,
                                         "lmax": lm} for aid, (lm, f) in zip(ids_b, fronts_b)])
            lmax_g, n_next = g.run(nf, [lm for lm, _ in fronts_g])
            for k, (lm_b, f_b) in enumerate(res_b):
                assert lmax_g[k] == lm_b
                f_g = g.next(k)
                np.testing.assert_array_equal(f_g["keys"], f_b["keys"])
                np.testing.assert_array_equal(f_g["lnl"], f_b["lnl"])
        finally:
            g.close()


def test_graph_argument_checks():
    a = _alignments(1, 43)[0]
    with pt.Context(precision="mixed", table_log2=14) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        with pytest.raises(pt.PTError):
            ctx.graph([aid], [0], [3.0])          # capacity below one tree
        with pytest.raises(pt.PTError):
            ctx.graph([aid, aid], [4, 4], [3.0, 3.0])  # an alignment twice
        with pytest.raises(pt.PTError):
            ctx.graph([aid], [4], [-1.0])         # negative threshold
        g = ctx.graph([aid], [2], [3.0])
        try:
            e, l = synth.random_trees(a.codes.shape[0], 3, 9)
            with pytest.raises(pt.PTError):
                g.set_frontier(0, e, l)           # 3 trees, capacity 2
            with pytest.raises(pt.PTError):
                g.run([3], [-1e300])              # count above capacity
            lmax, front = ctx.begin(aid, e[:2], l[:2], 3.0)
            nf = g.set_frontier(0, front["edges"][:2], front["lengths"][:2])
            _, n_next = g.run([nf], [lmax])
            if n_next[0] > 2:
                with pytest.raises(pt.PTError):
                    g.advance()                   # next frontier above capacity
        finally:
            g.close()
