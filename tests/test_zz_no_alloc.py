"""The allocation-free scoring entry point against the context path.

pt_score_topologies_noalloc is for callers that cannot allocate device
memory while running (a fixed, pre-reserved memory pool; code that must not
trigger the implicit synchronisation of cudaMalloc/cudaFree).  It works in a
fixed device array inside the library instead of allocating.  This test calls
it through the C ABI twice in a row on the same buffers and checks both
results against pt_score_topologies on the same trees, within the
mixed-precision tolerance of the other GPU tests.  The file is collected
last, so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu

TOL_LNL = 1e-3      # mixed precision, nats
TOL_LEN = 1e-3      # relative, lengths (pattern order differs between the two paths)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("n,sites,ncat,mode", [(12, 500, 4, "full"), (27, 900, 4, "fixed"), (9, 300, 1, "full")])
def test_noalloc_matches_context_path(torch_cuda, n, sites, ncat, mode):
    torch = torch_cuda
    a = synth.simulate(n, sites, 77 + n, model="gtr" if ncat > 1 else "jc", alpha=0.5 if ncat > 1 else None)
    tips, w = synth.compress_patterns(a.codes)
    e, l = synth.random_trees(n, 5, 9)
    rng = np.random.default_rng(4)
    l = rng.exponential(0.08, l.shape)
    with pt.Context(precision="mixed") as ctx:
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, ncat)
        ref_lnl, ref_len, _ = ctx.score(aid, e, l, mode=mode)
    dev = torch.device("cuda", 0)
    d_tips = torch.from_numpy(tips).to(dev)
    d_w = torch.from_numpy(w.astype(np.int32)).to(dev)
    d_e = torch.from_numpy(e).to(dev)
    d_l = torch.from_numpy(l).to(dev)
    outs = []
    for _ in range(2):  # two calls in a row share the library's array
        o_len = torch.full_like(d_l, -1.0)
        o_lnl = torch.full((len(e),), np.nan, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        st = pt.score_noalloc(n, tips.shape[1], d_tips.data_ptr(), d_w.data_ptr(), a.exch, a.freqs, 0.5, ncat,
                              len(e), d_e.data_ptr(), d_l.data_ptr(), o_len.data_ptr(), o_lnl.data_ptr(), mode=mode,
                              stream=stream.cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        outs.append((o_lnl.cpu().numpy(), o_len.cpu().numpy()))
    for lnl, lens in outs:
        np.testing.assert_allclose(lnl, ref_lnl, atol=TOL_LNL, rtol=0)
        np.testing.assert_allclose(lens, ref_len, rtol=TOL_LEN, atol=1e-6)
    np.testing.assert_allclose(outs[0][0], outs[1][0], atol=TOL_LNL, rtol=0)


def test_noalloc_rejects_oversized_and_invalid(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    n, P = 128, 60000  # partials of one tree alone exceed the fixed array
    d_tips = torch.zeros((n, P), dtype=torch.uint8, device=dev)
    d_w = torch.ones(P, dtype=torch.int32, device=dev)
    e, l = synth.random_trees(n, 1, 1)
    d_e = torch.from_numpy(e).to(dev)
    d_l = torch.from_numpy(l).to(dev)
    o_len = torch.empty_like(d_l)
    o_lnl = torch.empty(1, dtype=torch.float64, device=dev)
    st = pt.score_noalloc(n, P, d_tips.data_ptr(), d_w.data_ptr(), np.ones(6), np.full(4, 0.25), 0.5, 4, 1,
                          d_e.data_ptr(), d_l.data_ptr(), o_len.data_ptr(), o_lnl.data_ptr())
    assert st == 1
    bad = e.copy()
    bad[0, 0] = [0, 1]
    d_bad = torch.from_numpy(bad).to(dev)
    d_tips = torch.zeros((n, 10), dtype=torch.uint8, device=dev)
    d_w = torch.ones(10, dtype=torch.int32, device=dev)
    st = pt.score_noalloc(n, 10, d_tips.data_ptr(), d_w.data_ptr(), np.ones(6), np.full(4, 0.25), 0.5, 4, 1,
                          d_bad.data_ptr(), d_l.data_ptr(), o_len.data_ptr(), o_lnl.data_ptr())
    assert st == 1
