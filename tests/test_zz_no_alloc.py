"""The allocation-free scoring entry point against the FP64 oracle.

pt_score_topologies_noalloc is for callers that cannot allocate device
memory while they run: a process whose device memory is reserved up front by
another allocator (a serving process with a fixed pool), or code that must not
trigger the implicit device synchronisation of cudaMalloc/cudaFree.  It works
in a fixed device array inside the library instead of allocating.  These tests
call it through the C ABI, twice in a row on the same buffers, and check both
results against the oracle (lnL at the given lengths, or its full
optimisation) at the tolerances of the other GPU tests: 1e-8 nats in FP64,
1e-3 nats in mixed precision, lengths within 1e-4 relative.  The cases cover
more trees than persistent CTAs fit in the array (CTAs reuse their slab tree
after tree) and an FP64 sum-table too large for shared memory (kept in the
array).  The file is collected last, so a run that stops at the first failure
has run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import pt, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "mixed": 1e-3}
TOL_LEN = 1e-4  # relative (absolute 1e-6 near the lower bound)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11007_gb300 import build
    build.build()
    return torch


def _run(torch, a, tips, w, ncat, e, l, mode, prec):
    dev = torch.device("cuda", 0)
    cfg = pt.default_config()
    cfg.precision = pt.PREC_FP64 if prec == "fp64" else pt.PREC_MIXED
    d_tips = torch.from_numpy(tips).to(dev)
    d_w = torch.from_numpy(w.astype(np.int32)).to(dev)
    d_e = torch.from_numpy(np.ascontiguousarray(e)).to(dev)
    d_l = torch.from_numpy(np.ascontiguousarray(l)).to(dev)
    outs = []
    for _ in range(2):  # two calls in a row share the library's array
        o_len = torch.full_like(d_l, -1.0)
        o_lnl = torch.full((len(e),), np.nan, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        st = pt.score_noalloc(a.codes.shape[0], tips.shape[1], d_tips.data_ptr(), d_w.data_ptr(), a.exch, a.freqs,
                              0.5, ncat, len(e), d_e.data_ptr(), d_l.data_ptr(), o_len.data_ptr(), o_lnl.data_ptr(),
                              mode=mode, stream=stream.cuda_stream, cfg=cfg)
        assert st == 0
        torch.cuda.synchronize()
        outs.append((o_lnl.cpu().numpy(), o_len.cpu().numpy()))
    return outs


@pytest.mark.parametrize("n,sites,ncat,mode,prec,ntrees", [
    (12, 500, 4, "full", "mixed", 5),
    (12, 500, 4, "full", "fp64", 5),
    (27, 900, 4, "fixed", "mixed", 5),
    (9, 300, 1, "full", "fp64", 5),
    (40, 3000, 4, "fixed", "mixed", 8),   # ~3 CTAs fit in the array: each scores several trees
    (14, 3000, 4, "full", "fp64", 3),     # FP64 sum-table beyond shared memory, kept in the array
])
def test_noalloc_matches_oracle(torch_cuda, n, sites, ncat, mode, prec, ntrees):
    a = synth.simulate(n, sites, 77 + n, model="gtr" if ncat > 1 else "jc", alpha=0.5 if ncat > 1 else None)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, ncat)
    e, _ = synth.random_trees(n, ntrees, 9)
    l = np.random.default_rng(4).exponential(0.08, (ntrees, 2 * n - 3))
    outs = _run(torch_cuda, a, tips, w, ncat, e, l, mode, prec)
    for i in range(ntrees):
        if mode == "fixed":
            want, wl = pb.loglik(e[i], l[i]), l[i]
        else:
            want, wl, _ = pb.full_optimise(e[i], l[i])
        for lnl, lens in outs:
            assert abs(lnl[i] - want) <= TOL[prec], (i, lnl[i], want)
            np.testing.assert_allclose(lens[i], wl, rtol=TOL_LEN, atol=1e-6)
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


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
    d_tips = torch.zeros((n, 10), dtype=torch.uint8, device=dev)
    d_w = torch.ones(10, dtype=torch.int32, device=dev)
    bad = e.copy()
    bad[0, 0] = [0, 1]  # not a tree
    st = pt.score_noalloc(n, 10, d_tips.data_ptr(), d_w.data_ptr(), np.ones(6), np.full(4, 0.25), 0.5, 4, 1,
                          torch.from_numpy(bad).to(dev).data_ptr(), d_l.data_ptr(), o_len.data_ptr(), o_lnl.data_ptr())
    assert st == 1
    for x in (np.nan, -0.5, np.inf):  # lengths must be finite and >= 0
        lb = l.copy()
        lb[0, 3] = x
        st = pt.score_noalloc(n, 10, d_tips.data_ptr(), d_w.data_ptr(), np.ones(6), np.full(4, 0.25), 0.5, 4, 1,
                              d_e.data_ptr(), torch.from_numpy(lb).to(dev).data_ptr(), o_len.data_ptr(),
                              o_lnl.data_ptr(), mode="fixed")
        assert st == 1, x
