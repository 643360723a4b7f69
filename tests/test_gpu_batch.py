"""Batched rounds over uneven alignments (one persistent launch for the
neighbours of every frontier) against per-alignment rounds and the oracle."""
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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_round_equals_single_rounds(prec):
    alns = _alignments(5, 17)
    T = 4.0

    def setup(ctx):
        ids, fronts = [], []
        for i, a in enumerate(alns):
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            e, l = synth.random_trees(a.codes.shape[0], 3, 50 + i)
            lmax, front = ctx.begin(aid, e, l, T)
            ids.append(aid)
            fronts.append((lmax, front))
        return ids, fronts

    with pt.Context(precision=prec, table_log2=16) as single, pt.Context(precision=prec, table_log2=16) as batch:
        ids_s, fronts_s = setup(single)
        ids_b, fronts_b = setup(batch)
        for r in range(3):
            res_s = [single.expand(aid, f["edges"], f["lengths"], T, lm) for aid, (lm, f) in zip(ids_s, fronts_s)]
            res_b = batch.expand_batch([{"aln": aid, "edges": f["edges"], "lengths": f["lengths"], "threshold": T,
                                         "lmax": lm} for aid, (lm, f) in zip(ids_b, fronts_b)])
            for (lm_s, f_s), (lm_b, f_b) in zip(res_s, res_b):
                assert lm_s == lm_b
                np.testing.assert_array_equal(f_s["keys"], f_b["keys"])
                np.testing.assert_array_equal(f_s["lnl"], f_b["lnl"])
                np.testing.assert_array_equal(f_s["lengths"], f_b["lengths"])
            fronts_s, fronts_b = res_s, res_b
        for aid_s, aid_b in zip(ids_s, ids_b):
            vs, vb = single.visited(aid_s), batch.visited(aid_b)
            ds = dict(zip(pt.keys_to_int(vs["keys"]), zip(vs["status"], vs["lnl"])))
            db = dict(zip(pt.keys_to_int(vb["keys"]), zip(vb["status"], vb["lnl"])))
            assert ds == db


def test_batched_round_matches_oracle():
    alns = _alignments(4, 23)
    T = 3.0
    with pt.Context(precision="fp64", table_log2=16) as ctx:
        parts, before = [], []
        for i, a in enumerate(alns):
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            n = a.codes.shape[0]
            e, l = synth.random_trees(n, 1, 70 + i)
            lmax, front = ctx.begin(aid, e, l, T)
            before.append(set(pt.keys_to_int(ctx.visited(aid)["keys"])))
            parts.append({"aln": aid, "edges": front["edges"], "lengths": front["lengths"], "threshold": T,
                          "lmax": lmax})
        res = ctx.expand_batch(parts)
        for i, (a, p, (lm, nxt)) in enumerate(zip(alns, parts, res)):
            tips, w = synth.compress_patterns(a.codes)
            pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
            s = oracle.Search(pb, p["edges"], p["lengths"], T, frontier_lmax=p["lmax"])
            s.round()
            ov = s.visited()
            gv = ctx.visited(p["aln"])
            od = dict(zip(pt.keys_to_int(ov["keys"]), zip(ov["status"], ov["lnl"])))
            gd = dict(zip(pt.keys_to_int(gv["keys"]), zip(gv["status"], gv["lnl"])))
            # every entry of this round must agree (the frontier itself was visited before)
            assert set(gd) - before[i] == set(od) - before[i]
            for k, (st, x) in od.items():
                if k in before[i]:
                    continue
                assert gd[k][0] == st
                assert abs(gd[k][1] - x) <= 1e-8
            assert abs(lm - s.lmax) <= 1e-8
