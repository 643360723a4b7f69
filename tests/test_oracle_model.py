"""Pins of the oracle's model layer: discrete Gamma rates, GTR Q, P(t), hashes.

Every check compares the oracle with something other than itself: a library
routine (scipy), a closed form, or a published constant.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, linalg, special, stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "published_constants.json")


@pytest.mark.parametrize("a,x", [(0.5, 0.1), (0.5, 3.0), (1.5, 0.7), (1.5, 9.0), (6.0, 2.0), (6.0, 12.0),
                                 (0.05, 0.001), (30.0, 28.0)])
def test_incomplete_gamma_matches_scipy(a, x):
    assert oracle.gamma_p(a, x) == pytest.approx(special.gammainc(a, x), rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("alpha", [0.1, 0.5, 1.0, 2.3, 20.0])
@pytest.mark.parametrize("ncat", [2, 4, 8])
def test_gamma_category_means_match_quadrature(alpha, ncat):
    # Category bounds from scipy's quantile, category means by numerical
    # integration of x * pdf(x) over each bound pair (Yang 1994, mean method).
    dist = stats.gamma(a=alpha, scale=1.0 / alpha)
    bounds = [0.0] + [dist.ppf(k / ncat) for k in range(1, ncat)] + [np.inf]
    want = []
    for k in range(ncat):
        val, _ = integrate.quad(lambda x: x * dist.pdf(x), bounds[k], bounds[k + 1], limit=400,
                                epsabs=1e-14, epsrel=1e-12)
        want.append(ncat * val)
    want = np.array(want)
    want *= ncat / want.sum()
    got = oracle.gamma_rates(alpha, ncat)
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-10)
    assert got.mean() == pytest.approx(1.0, abs=1e-14)
    assert np.all(np.diff(got) > 0)


def test_single_category_is_no_rate_variation():
    np.testing.assert_array_equal(oracle.gamma_rates(0.5, 1), [1.0])


def _rand_model(seed):
    rng = np.random.default_rng(seed)
    return rng.dirichlet(np.ones(6)), rng.dirichlet(np.full(4, 5.0))


def test_jc_transition_matrix_closed_form():
    Q = oracle.gtr_q(np.ones(6), np.full(4, 0.25))
    for t in [1e-6, 0.01, 0.1, 0.7, 3.0, 40.0]:
        P = oracle.expm(Q, t)
        e = math.exp(-4.0 * t / 3.0)
        want = np.full((4, 4), 0.25 - 0.25 * e)
        np.fill_diagonal(want, 0.25 + 0.75 * e)
        np.testing.assert_allclose(P, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gtr_normalisation_and_reversibility(seed):
    exch, freqs = _rand_model(seed)
    Q = oracle.gtr_q(exch, freqs)
    np.testing.assert_allclose(Q.sum(1), 0.0, atol=1e-14)
    assert -np.sum(freqs * np.diag(Q)) == pytest.approx(1.0, abs=1e-14)
    # detailed balance pi_i Q_ij = pi_j Q_ji
    F = freqs[:, None] * Q
    np.testing.assert_allclose(F, F.T, atol=1e-15)
    # off-diagonal rates are proportional to the exchangeabilities
    iu = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    ratios = [Q[i, j] / freqs[j] / exch[k] for k, (i, j) in enumerate(iu)]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-13)


@pytest.mark.parametrize("seed", [4, 5])
@pytest.mark.parametrize("t", [1e-6, 0.05, 0.5, 5.0, 80.0])
def test_expm_matches_scipy(seed, t):
    exch, freqs = _rand_model(seed)
    Q = oracle.gtr_q(exch, freqs)
    np.testing.assert_allclose(oracle.expm(Q, t), linalg.expm(Q * t), rtol=1e-11, atol=1e-14)


def test_mix64_matches_published_splitmix64_outputs():
    g = json.load(open(GOLDEN))["splitmix64"]
    gamma = int(g["gamma"], 16)
    state = 0
    for want in g["outputs_seed0"]:
        state = (state + gamma) % (1 << 64)
        assert oracle.mix64(state) == int(want, 16)


def test_split_hash_definition():
    # h.lo = mix64(lo ^ mix64(hi + c1)), h.hi = mix64(hi ^ mix64(lo + c2)),
    # checked through the pinned mix64 on a few words.
    c1, c2 = 0x9E3779B97F4A7C15, 0xD1B54A32D192ED03
    M = (1 << 64) - 1
    for lo, hi in [(0, 0), (6, 0), (1 << 63, 5), (M, M)]:
        h = oracle.split_hash(lo, hi)
        assert h[0] == oracle.mix64(lo ^ oracle.mix64((hi + c1) & M))
        assert h[1] == oracle.mix64(hi ^ oracle.mix64((lo + c2) & M))
