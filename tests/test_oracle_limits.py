"""Pins of the oracle's likelihood by two limits it must reproduce:

* site patterns: the log-likelihood of the compressed patterns with their
  integer weights equals the sum over the raw columns, each with weight 1
  (catches a weight or pattern-indexing mistake);
* rate variation: as the Gamma shape alpha grows, every category rate tends
  to 1, so four categories give the single-category log-likelihood, with a
  gap proportional to 1/alpha (catches a mistake in the category rates or
  their 1/C weights).
"""
import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import synth


@pytest.mark.parametrize("n,sites,seed,gap", [(6, 400, 71, 0.0), (9, 600, 72, 0.1)])
def test_compressed_patterns_equal_raw_columns(n, sites, seed, gap):
    a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, gap_frac=gap, mean_branch=0.1)
    tips, w = synth.compress_patterns(a.codes)
    assert tips.shape[1] < sites  # some columns repeat
    pc = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    pr = oracle.Problem(a.codes, np.ones(sites), a.exch, a.freqs, 0.5, 4)
    e, l = a.tree_edges, a.tree_lengths
    lc, site_c = pc.loglik(e, l, per_site=True)
    lr, site_r = pr.loglik(e, l, per_site=True)
    assert lc == pytest.approx(lr, rel=1e-13)
    # each raw column's value is its pattern's value
    index = {tuple(tips[:, p]): p for p in range(tips.shape[1])}
    for c in range(sites):
        assert site_r[c] == pytest.approx(site_c[index[tuple(a.codes[:, c])]], rel=1e-13)


@pytest.mark.parametrize("seed", [81, 82])
def test_large_gamma_shape_is_no_rate_variation(seed):
    n, sites = 8, 500
    a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.1)
    tips, w = synth.compress_patterns(a.codes)
    one = oracle.Problem(tips, w, a.exch, a.freqs, 1.0, 1)
    rates = oracle.gamma_rates(1e6, 4)
    assert np.max(np.abs(rates - 1.0)) < 5e-3
    four = oracle.Problem(tips, w, a.exch, a.freqs, 1e6, 4)
    e, l = a.tree_edges, a.tree_lengths
    l1 = one.loglik(e, l)
    assert abs(four.loglik(e, l) - l1) < 1e-3
    # the category rates average to 1 and spread by O(alpha^-1/2), so the gap is
    # second order: proportional to their variance, 1/alpha (a wrong weight or
    # rate would leave a first-order or constant gap)
    scaled = [(oracle.Problem(tips, w, a.exch, a.freqs, s, 4).loglik(e, l) - l1) * s for s in (1e4, 1e5, 1e6)]
    assert scaled[0] != 0.0
    np.testing.assert_allclose(scaled[1:], scaled[0], rtol=2e-2)
