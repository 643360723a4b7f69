"""pt_set_allocator: the context's device memory from the caller (here
PyTorch's caching allocator through counting callbacks).  A search (start
trees, rounds, a graph round, the learned start) on it gives the same results
as on cudaMalloc, bit for bit; every block it allocated is returned exactly
once when the context closes; an allocator with no memory gives PT_ERR_OOM."""
import numpy as np
import pytest

from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()


def _search(ctx, a):
    aid = ctx.load_alignment(a.codes)
    ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
    rng = np.random.default_rng(3)
    ctx.mlp_set_weights((rng.standard_normal(pt.MLP_PARAMS) * 0.05).astype(np.float32))
    ctx.mlp_enable(True)
    e, l = synth.random_trees(a.codes.shape[0], 4, 17)
    lmax, front = ctx.begin(aid, e, l, 4.0)
    out = [front]
    for _ in range(2):
        lmax, front = ctx.expand(aid, front["edges"], front["lengths"], 4.0, lmax)
        out.append(front)
    assert len(front["edges"]) > 0
    g = ctx.graph([aid], [len(front["edges"])], [4.0])
    try:
        g.set_frontier(0, front["edges"], front["lengths"])
        lm, _ = g.run([len(front["edges"])], [lmax])
        out.append(g.next(0))
    finally:
        g.close()
    v = ctx.visited(aid)
    return lm[0], out, v


def test_search_on_callers_memory_equals_cudamalloc():
    import torch
    a = synth.simulate(16, 700, 2024, model="gtr", alpha=0.5, mean_branch=0.06)
    stream = torch.cuda.current_stream()
    alloc_t, free_t = pt.torch_allocator(0, stream)
    live, made, returned = {}, [], []

    def alloc(n):
        p = alloc_t(n)
        if p:
            assert p % 256 == 0
            live[p] = n
            made.append(p)
        return p

    def free(p):
        assert p in live  # only blocks this allocator made, each once
        del live[p]
        returned.append(p)
        free_t(p)

    with pt.Context(precision="mixed", table_log2=16, stream=stream) as ref:
        lm_r, out_r, v_r = _search(ref, a)
    before = torch.cuda.memory_allocated()
    ctx = pt.Context(precision="mixed", table_log2=16, stream=stream)
    ctx.set_allocator(alloc, free)
    lm_u, out_u, v_u = _search(ctx, a)
    held = torch.cuda.memory_allocated() - before
    assert made and held >= sum(live.values()) > 0  # the context's memory is PyTorch's
    ctx.close()
    assert not live and sorted(returned) == sorted(made)
    assert lm_u == lm_r
    for x, y in zip(out_u, out_r):
        for k in ("keys", "lnl", "lengths", "edges"):
            np.testing.assert_array_equal(x[k], y[k])
    ku, kr = pt.keys_to_int(v_u["keys"]), pt.keys_to_int(v_r["keys"])
    assert dict(zip(ku, zip(v_u["status"], v_u["lnl"]))) == dict(zip(kr, zip(v_r["status"], v_r["lnl"])))


def test_allocator_without_memory_reports_oom():
    a = synth.simulate(8, 200, 7, model="gtr", alpha=0.5)
    with pt.Context(precision="mixed", table_log2=12) as ctx:
        ctx.set_allocator(lambda n: 0, lambda p: None)
        with pytest.raises(pt.PTError) as ex:
            ctx.load_alignment(a.codes)
        assert ex.value.status == 2  # PT_ERR_OOM
        ctx.set_allocator(None)  # back to cudaMalloc
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        e, l = synth.random_trees(8, 1, 1)
        lnl, _, _ = ctx.score(aid, e, l, mode="fixed")
        assert np.isfinite(lnl[0])
