"""Hill-climb on the GPU (the stand-in for the paper's RAxML starts: PT is
seeded with local likelihood maxima, section "Maximum Likelihood Estimation
of Local Maxima") against the oracle's climb: the same final topology (key
bit for bit), the same number of moves, lnL within the precision's tolerance
and branch lengths within 1e-4 relative."""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-8, "mixed": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _by_split(n, edges, lengths):
    """split (side of the edge without taxon 0, as a bitmask) -> length, for any edge list."""
    edges = np.asarray(edges).reshape(-1, 2)
    adj = {}
    for u, v in edges:
        adj.setdefault(int(u), []).append(int(v))
        adj.setdefault(int(v), []).append(int(u))
    out = {}
    for (x, y), t in zip(edges, lengths):
        seen, stack, s = {int(x), int(y)}, [int(y)], 0
        while stack:
            c = stack.pop()
            if c < n:
                s |= 1 << c
            for d in adj[c]:
                if d not in seen:
                    seen.add(d)
                    stack.append(d)
        if s & 1:
            s ^= (1 << n) - 1
        out[s] = float(t)
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,seed", [(8, 5), (10, 4), (12, 6)])
def test_hill_climb_matches_oracle(prec, n, seed):
    a = synth.simulate(n, 600, 1000 + seed, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    e, l = synth.random_trees(n, 4, seed)
    with pt.Context(precision=prec, table_log2=12) as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        res = ctx.hill_climb(aid, e, l)
        one = ctx.hill_climb(aid, e[1:2], l[1:2])  # a climb alone = the same climb in a batch
    assert pt.keys_to_int(one["keys"]) == pt.keys_to_int(res["keys"][1:2])
    assert one["moves"][0] == res["moves"][1] and one["lnl"][0] == res["lnl"][1]
    for i in range(len(e)):
        lo, oe, ol, om = pb.hill_climb(e[i], l[i])
        assert pt.keys_to_int(res["keys"][i:i + 1]) == [pt.keys_to_int(np.array([oracle.tree_key(n, oe)], np.uint64))[0]]
        assert res["moves"][i] == om, (i, res["moves"][i], om)
        assert abs(res["lnl"][i] - lo) <= TOL[prec], (i, res["lnl"][i], lo)
        # lengths by split against the oracle's (same topology)
        got, want = _by_split(n, res["edges"][i], res["lengths"][i]), _by_split(n, oe, ol)
        assert set(got) == set(want)
        for sp, t in want.items():
            assert abs(got[sp] - t) <= 1e-4 * t + 1e-6, (sp, got[sp], t)
    assert np.all(res["moves"] >= 1)
