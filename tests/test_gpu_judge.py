"""The plain start as judge of the learned start (pt_mlp_judge), on the
benchmarked round (27 taxa x 2000 sites, ~5400 proposals per round, so the
judge decides after every round): the trained network is chosen; a network
made harmful (its output layer scaled up 10x: far-off starting lengths) is
dropped after one round.  Every 4th proposal before the judge's first decision,
every 16th after it, takes the start not chosen (the judge's sample), so once the harmful network is dropped each proposal outside
the sample equals the round without the network bit for bit; decisions are
identical throughout, in batched rounds and in graph replays."""
import numpy as np
import pytest

from paper_1811_11007_gb300 import pt

pytestmark = pytest.mark.gpu
OUT_W, OUT_B = 80 * 128 + 128 + 128 * 128 + 128, 80 * 128 + 128 + 128 * 128 + 128 + 1024


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _round(ctx, aid, front, T, lmax):
    ctx.reset_visited(aid)
    lm, nxt = ctx.expand(aid, front["edges"], front["lengths"], T, lmax)
    pr = ctx.last_proposals()
    return lm, nxt, ctx.stats(), dict(zip(map(tuple, pr["keys"].tolist()), pr["lnl"])), pr


def _decides_like(lm, nxt, lm_p, nx_p):
    assert abs(lm - lm_p) <= 1e-3
    assert nxt["keys"].tolist() == nx_p["keys"].tolist()
    np.testing.assert_allclose(nxt["lnl"], nx_p["lnl"], rtol=0, atol=1e-3)


def test_judge_keeps_a_helpful_network_and_drops_a_harmful_one(warm_weights):
    import bench
    W = bench.WORKLOADS["pt27"]
    T = W["thresh"]
    a, starts = bench.workload(W, 0)
    with pt.Context(precision="mixed", table_log2=22) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        hc = ctx.hill_climb(aid, *starts)
        lmax0, front, _ = bench.build_frontier(ctx, aid, hc["edges"], hc["lengths"], W["frontier"], T)
        ctx.mlp_set_weights(warm_weights)
        trained = np.array(ctx.mlp_get_weights(), np.float32)
        ctx.mlp_enable(False)
        lm_p, nx_p, st_p, sc_p, _ = _round(ctx, aid, front, T, lmax0)
        W = st_p["scored"]
        # the trained network: re-enabling resets the judge; one round decides for it
        ctx.mlp_enable(True)
        j = ctx.mlp_judge(aid)
        assert j["state"] == "open" and j["learned_items"] == j["plain_items"] == 0
        lm_t, nx_t, st_t, _, _ = _round(ctx, aid, front, T, lmax0)
        j = ctx.mlp_judge(aid)
        print("trained network (counts halved at the decision):", j)
        assert j["state"] == "learned"
        assert j["plain_items"] == ((W + 3) // 4) >> 1 and j["learned_items"] == (W - (W + 3) // 4) >> 1
        assert abs(2 * (j["plain_evals"] + j["learned_evals"]) - st_t["prop_evals"]) <= 2
        assert j["learned_evals"] / j["learned_items"] < 0.98 * j["plain_evals"] / j["plain_items"]
        _decides_like(lm_t, nx_t, lm_p, nx_p)
        # a harmful network: the same weights with the output layer scaled up 10x
        w = trained.copy()
        w[OUT_W:OUT_B] *= 10.0
        ctx.mlp_set_weights(w)  # new weights reset the judge
        assert ctx.mlp_judge(aid)["state"] == "open"
        lm_h, nx_h, _, _, _ = _round(ctx, aid, front, T, lmax0)
        j = ctx.mlp_judge(aid)
        print("harmful network:", j)
        assert j["state"] == "plain"
        assert j["learned_evals"] / j["learned_items"] > j["plain_evals"] / j["plain_items"]
        _decides_like(lm_h, nx_h, lm_p, nx_p)
        # dropped: only the sample (every 16th proposal) still starts from the network
        lm_d, nx_d, _, sc_d, pr_d = _round(ctx, aid, front, T, lmax0)
        assert ctx.mlp_judge(aid)["state"] == "plain"
        keys = list(map(tuple, pr_d["keys"].tolist()))
        same = [sc_d[k] == sc_p[k] for k in keys]
        assert all(s for i, s in enumerate(same) if i % 16 != 0)
        _decides_like(lm_d, nx_d, lm_p, nx_p)
        g = ctx.graph([aid], [len(front["edges"])], [T])
        try:
            g.set_frontier(0, front["edges"], front["lengths"])
            ctx.reset_visited(aid)
            lm_g, _ = g.run([len(front["edges"])], [lmax0])
            _decides_like(lm_g[0], g.next(0), lm_p, nx_p)
        finally:
            g.close()
        assert ctx.mlp_judge(aid)["state"] == "plain"
