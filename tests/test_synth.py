"""Pins of the synthetic input generator (Gillespie simulation down the tree)
against closed forms, on a three-taxon star so that leaves 0 and 1 are at
distance d = t0 + t1:

* JC69, no rate variation: P(leaves differ) = 3/4 (1 - exp(-4d/3));
* JC69, Gamma(alpha) site rates: averaging over the rate with the Gamma
  moment-generating function, P(differ) = 3/4 (1 - (1 + 4d/(3 alpha))^-alpha);
* GTR, no rate variation: the joint distribution of the two leaves' states is
  pi_i P_ij(d) with P = expm(Q d) (scipy), Q normalised to one expected
  substitution per unit time -- which also pins the generator's normalisation.

Each proportion is checked within 5 standard errors of its sample size.
"""
import numpy as np
import pytest

from paper_1811_11007_gb300 import synth

scipy_linalg = pytest.importorskip("scipy.linalg")
STAR = np.array([[0, 3], [1, 3], [2, 3]], np.int32)
N = 200_000


def _within(p_obs, p, n, k=5.0):
    return abs(p_obs - p) <= k * np.sqrt(max(p * (1 - p), 1e-12) / n)


@pytest.mark.parametrize("t0,t1", [(0.05, 0.1), (0.3, 0.4)])
def test_jc_difference_proportion(t0, t1):
    a = synth.simulate(3, N, 91, model="jc", alpha=None, tree=STAR, lengths=np.array([t0, t1, 0.2]))
    d = t0 + t1
    p = 0.75 * (1 - np.exp(-4 * d / 3))
    assert _within(np.mean(a.codes[0] != a.codes[1]), p, N)


@pytest.mark.parametrize("alpha", [0.3, 1.0])
def test_jc_gamma_difference_proportion(alpha):
    t0, t1 = 0.2, 0.25
    a = synth.simulate(3, N, 92, model="jc", alpha=alpha, tree=STAR, lengths=np.array([t0, t1, 0.1]))
    d = t0 + t1
    p = 0.75 * (1 - (1 + 4 * d / (3 * alpha)) ** (-alpha))
    assert _within(np.mean(a.codes[0] != a.codes[1]), p, N)


def test_gtr_joint_distribution():
    t0, t1 = 0.15, 0.25
    a = synth.simulate(3, N, 93, model="gtr", alpha=None, tree=STAR, lengths=np.array([t0, t1, 0.1]))
    exch, pi = a.exch, a.freqs
    # exchangeabilities in the order AC AG AT CG CT GT
    Q = np.zeros((4, 4))
    for (i, j), s in zip([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], exch):
        Q[i, j] = s * pi[j]
        Q[j, i] = s * pi[i]
    np.fill_diagonal(Q, -Q.sum(1))
    Q /= -np.sum(pi * np.diag(Q))
    P = scipy_linalg.expm(Q * (t0 + t1))
    joint = pi[:, None] * P
    counts = np.zeros((4, 4))
    np.add.at(counts, (a.codes[0], a.codes[1]), 1)
    for i in range(4):
        assert _within(np.mean(a.codes[2] == i), pi[i], N)  # stationary composition
        for j in range(4):
            assert _within(counts[i, j] / N, joint[i, j], N), (i, j, counts[i, j] / N, joint[i, j])


def test_reinsert_leaves_gives_binary_trees_near_the_original():
    import oracle
    rng = np.random.default_rng(5)
    n = 40
    e = synth.random_topology(n, rng)
    base = {int(s[0]) | (int(s[1]) << 64) for s in oracle.tree_splits(n, e)}
    assert oracle.tree_key(n, synth.reinsert_leaves(e, n, 0, rng)) == oracle.tree_key(n, e)
    moved = 0
    for k in (1, 3):
        for _ in range(10):
            p = synth.reinsert_leaves(e, n, k, rng)
            deg = np.bincount(p.reshape(-1), minlength=2 * n - 2)
            assert p.shape == (2 * n - 3, 2) and np.all(deg[:n] == 1) and np.all(deg[n:] == 3)
            sp = {int(s[0]) | (int(s[1]) << 64) for s in oracle.tree_splits(n, p)}  # raises if not a tree
            moved += sp != base
    assert moved >= 15
