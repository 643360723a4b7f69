"""Two workload configurations beyond the benchmarked round, as GPU parity cases:

* learned warm start on fresh 64-taxon x 1500-site GTR+G4 alignments: a
  network trained on PT runs of other (27-taxon and 7-taxon) alignments, a
  multi-round search from 8 hill-climbed starts run from the plain and from
  the learned start, deciding identically (next frontiers, statuses), the
  learned start needing fewer Newton evaluations (the saving is printed);
* PT at scale: 128 taxa x 10000 sites (~6000 patterns), Exp(0.02) branches,
  32 random starts, threshold 15, a 2^24-slot visited table; the learned +
  mixed-precision round against the plain FP64 GPU path on the same frontier
  (scored key sets bit-exact, keep decisions equal except for neighbours
  within twice the tolerance of the threshold, which are listed).  Scores
  agree within 1e-3 nats at lnL ~ -5e5: the mixed path's scores come from
  compensated FP32 pairs, so the FP32 rounding of partials that recur at
  thousands of sites (constant columns below a node) does not add up.
"""
import numpy as np
import pytest

from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _keys(k):
    return [(int(lo), int(hi)) for lo, hi in np.asarray(k, np.uint64).reshape(-1, 2)]


def _round(ctx, aid, front, T, lmax):
    """One round from a fresh visited table: (lmax, next frontier, proposals, stats)."""
    ctx.reset_visited(aid)
    lm, nxt = ctx.expand(aid, front["edges"], front["lengths"], T, lmax)
    return lm, nxt, ctx.last_proposals(), ctx.stats()


def test_learned_start_on_fresh_64_taxa(warm_weights):
    """Fresh 64-taxon x 1500-site alignments, searched as PT searches them: 8
    hill-climbs from random trees give the starts, threshold 10, four rounds
    (frontier capped at 256 trees) from the plain and from the learned start.
    The learned start must decide identically and need fewer proposal Newton
    evaluations; the saving is printed."""
    n, sites, T = 64, 1500, 10.0
    saved = []
    with pt.Context(precision="mixed", table_log2=20) as ctx:
        ctx.mlp_set_weights(warm_weights)  # trained on runs of 27-taxon and 7-taxon alignments
        for seed in (synth.SEED_BASE + 640, synth.SEED_BASE + 641):
            a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.05)
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            ctx.mlp_enable(False)
            hc = ctx.hill_climb(aid, *synth.random_trees(n, 8, seed + 1))
            lmax, front = ctx.begin(aid, hc["edges"], hc["lengths"], T)
            trails = {}
            for on in (False, True):
                ctx.mlp_enable(on)
                ctx.reset_visited(aid)
                lm, f = lmax, front
                fronts, evals, scored = [], np.zeros(2, np.int64), 0
                for _ in range(4):
                    if not len(f["edges"]):
                        break
                    lm, f = ctx.expand(aid, f["edges"][:256], f["lengths"][:256], T, lm)
                    st = ctx.stats()
                    evals += (st["prop_evals"], st["full_evals"])
                    scored += st["scored"]
                    fronts.append((lm, f))
                v = ctx.visited(aid)
                trails[on] = (fronts, evals, scored, dict(zip(_keys(v["keys"]), zip(v["status"], v["lnl"]))))
            (f0, ev0, s0, v0), (f1, ev1, s1, v1) = trails[False], trails[True]
            assert len(f0) == len(f1) >= 2 and s0 == s1
            for (lm0, a0), (lm1, a1) in zip(f0, f1):
                assert abs(lm0 - lm1) <= TOL
                assert _keys(a0["keys"]) == _keys(a1["keys"])
                np.testing.assert_allclose(a0["lnl"], a1["lnl"], rtol=0, atol=TOL)
            assert set(v0) == set(v1)
            assert all(v0[k][0] == v1[k][0] for k in v0)  # every status (kept / rejected / frontier) identical
            saved.append(1 - ev1[0] / ev0[0])
            print(f"64 taxa x {sites} sites (seed {seed}), {len(v0)} topologies visited, {s0} proposals: "
                  f"proposal Newton evaluations plain {ev0[0]} ({ev0[0] / s0:.1f} per proposal), learned {ev1[0]} "
                  f"({ev1[0] / s1:.1f}; {100 * saved[-1]:.1f}% saved); visit evaluations plain {ev0[1]}, "
                  f"learned {ev1[1]}; judge {ctx.mlp_judge(aid)}")
    assert all(x > 0 for x in saved)  # the network pays on every fresh alignment


def test_scale_128_taxa_learned_mixed_vs_plain_fp64(warm_weights):
    n, sites, T = 128, 10000, 15.0
    seed = synth.SEED_BASE + 1280
    a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.02)
    e, l = synth.random_trees(n, 32, seed + 1)
    with pt.Context(precision="mixed", table_log2=24) as mx, pt.Context(precision="fp64", table_log2=20) as dp:
        mx.mlp_set_weights(warm_weights)
        am = mx.load_alignment(a.codes)
        mx.set_model(am, a.exch, a.freqs, 0.5, 4)
        ad = dp.load_alignment(a.codes)
        dp.set_model(ad, a.exch, a.freqs, 0.5, 4)
        assert mx.alignment_info(am)[1] > 4000
        mx.mlp_enable(False)
        lmax, front = mx.begin(am, e, l, T)
        rounds = 0
        for _ in range(3):
            if not len(front["edges"]):
                break
            mx.mlp_enable(True)
            lm_l, nx_l, pr_l, st_l = _round(mx, am, front, T, lmax)
            mx.mlp_enable(False)
            lm_m, nx_m, pr_m, _ = _round(mx, am, front, T, lmax)
            lm_d, nx_d, pr_d, _ = _round(dp, ad, front, T, lmax)
            assert st_l["nonconverged"] == 0
            # the same neighbours scored by all three, keys bit for bit
            kl, km, kd = _keys(pr_l["keys"]), _keys(pr_m["keys"]), _keys(pr_d["keys"])
            assert set(kl) == set(km) == set(kd) and len(kd) == len(set(kd))
            # precision: mixed vs FP64 from the same (plain) start
            tol = TOL
            sm, sd = dict(zip(km, pr_m["lnl"])), dict(zip(kd, pr_d["lnl"]))
            worst = max(abs(sm[k] - sd[k]) for k in kd)
            assert worst <= tol, worst
            cut = lmax - T
            near = sorted(k for k in kd if abs(sd[k] - cut) <= 2 * tol)
            if near:
                print(f"round {rounds}: {len(near)} neighbour(s) within {2 * tol:.1e} nats of the threshold: {near}")
            assert all((sm[k] >= cut) == (sd[k] >= cut) for k in kd if k not in near)
            assert abs(lm_m - lm_d) <= tol
            fm = dict(zip(_keys(nx_m["keys"]), nx_m["lnl"]))
            fd = dict(zip(_keys(nx_d["keys"]), nx_d["lnl"]))
            # after the visits the threshold is lmax' - T: trees within 2 tol of it may differ too
            near_v = {k for k, x in list(fm.items()) + list(fd.items()) if abs(x - (lm_d - T)) <= 2 * tol}
            assert set(fm) ^ set(fd) <= set(near) | near_v
            wv = max([abs(fm[k] - fd[k]) for k in set(fm) & set(fd)], default=0.0)
            assert wv <= tol, wv
            # warm start: the learned round decides as the plain one
            sl = dict(zip(kl, pr_l["lnl"]))
            assert {k for k in kl if sl[k] >= cut} == {k for k in km if sm[k] >= cut}
            assert _keys(nx_l["keys"]) == _keys(nx_m["keys"])
            np.testing.assert_allclose(nx_l["lnl"], nx_m["lnl"], rtol=0, atol=TOL)
            assert abs(lm_l - lm_m) <= TOL
            print(f"round {rounds}: lnL {lmax:.1f}, frontier {len(front['edges'])}, scored {len(kd)}, "
                  f"next {len(fd)}, max |mixed - fp64| proposals {worst:.2e}, visits {wv:.2e}, "
                  f"lmax {abs(lm_m - lm_d):.2e} nats")
            lmax, front = lm_l, nx_l
            rounds += 1
        assert rounds >= 1
