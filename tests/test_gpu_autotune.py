"""Autotuner: a bucket is tuned on a launch that fills the GPU, the choice is
persisted as JSON and reloaded by a new context, and a tuned round gives the
same visited set and likelihoods as an untuned one (which the parity tests
pin to the oracle)."""
import json

import numpy as np
import pytest

from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu
CANDIDATES = {64, 96, 128, 192, 256, 384, 512}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _round(ctx, a, front_e, front_l):
    aid = ctx.load_alignment(a.codes)
    ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
    lmax, nxt = ctx.expand(aid, front_e, front_l, np.inf, -1e300)
    v = ctx.visited(aid)
    return lmax, dict(zip(pt.keys_to_int(v["keys"]), zip(v["status"], v["lnl"])))


def test_autotune_tunes_persists_and_keeps_results(tmp_path):
    n = 30
    a = synth.simulate(n, 600, 616, model="gtr", alpha=0.5, mean_branch=0.08)
    e, l = synth.random_trees(n, 24, 6)  # 24 x 54 = 1296 neighbours, all kept at T = inf
    cache = str(tmp_path / "tune.json")
    with pt.Context(precision="mixed", table_log2=16) as tuned:
        tuned.autotune(True, cache)
        lm_t, vt = _round(tuned, a, e, l)
        rep = tuned.autotune_report()
    with pt.Context(precision="mixed", table_log2=16) as plain:
        lm_p, vp = _round(plain, a, e, l)
    assert rep
    (key, v), = rep.items()
    assert key.startswith("prec1_cat4_taxa32")
    assert v["prop_threads"] in CANDIDATES and v["full_threads"] in CANDIDATES
    assert v["prop_items"] >= 1296 - 24 and v["full_items"] >= 1000
    on_disk = json.load(open(cache))
    assert on_disk[key]["prop_threads"] == v["prop_threads"] and on_disk[key]["full_threads"] == v["full_threads"]
    with pt.Context(precision="mixed") as again:
        again.autotune(False, cache)
        assert again.autotune_report()[key]["full_threads"] == v["full_threads"]
    assert set(vt) == set(vp)
    for k in vt:
        assert vt[k][0] == vp[k][0]
        if np.isnan(vt[k][1]) and np.isnan(vp[k][1]):
            continue  # the frontier itself (entered without a likelihood)
        assert abs(vt[k][1] - vp[k][1]) <= 1e-3
    assert abs(lm_t - lm_p) <= 1e-3
