"""Pins of the oracle's Gamma-shape re-optimisation per visit ("Phylogenetic
Topographer": model optimisation for each visited topology, here the shape of
the Gamma rate heterogeneity).

Independent references: scipy's bounded scalar minimiser on lnL(alpha) at the
visit's final lengths (evaluated through separately built problems), length
stationarity at the final shape, recovery of the simulating shape on a long
alignment, and the no-op cases.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle
from paper_1811_11007_gb300 import synth


def _lnl_at(a, tips, w, edges, lens, alpha):
    return oracle.Problem(tips, w, a.exch, a.freqs, alpha, 4).loglik(edges, lens)


@pytest.mark.parametrize("seed,base", [(611, 1.0), (612, 0.3)])
def test_visit_reaches_the_joint_optimum(seed, base):
    n = 8
    a = synth.simulate(n, 800, seed, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, base, 4)
    pb.set_reopt_alpha(True)
    f, lens, alpha = pb.visit_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    assert 0.02 < alpha < 100
    # the score is lnL at the final shape and lengths
    assert f == pytest.approx(_lnl_at(a, tips, w, a.tree_edges, lens, alpha), abs=1e-9)
    # shape: an independent bounded minimiser at the final lengths agrees
    res = minimize_scalar(lambda u: -_lnl_at(a, tips, w, a.tree_edges, lens, math.exp(u)),
                          bounds=(math.log(0.02), math.log(100.0)), method="bounded",
                          options={"xatol": 1e-8})
    assert math.exp(res.x) == pytest.approx(alpha, rel=1e-4)
    assert -res.fun <= f + 1e-8
    # lengths: stationary at the final shape
    p2 = oracle.Problem(tips, w, a.exch, a.freqs, alpha, 4)
    for e in range(2 * n - 3):
        _, d1, d2 = p2.edge_derivs(a.tree_edges, lens, e)
        assert abs(d1 / d2) < 1e-5 or (lens[e] <= 1e-6 + 2e-8 and d1 < 0)
    # the fixed-shape optimum is no better
    pb.set_reopt_alpha(False)
    f0, _, a0 = pb.visit_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    assert a0 == base
    assert f >= f0 - 1e-9


def test_recovers_the_simulating_shape():
    n = 10
    a = synth.simulate(n, 6000, 613, model="gtr", alpha=0.5, mean_branch=0.15)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 2.0, 4)
    pb.set_reopt_alpha(True)
    _, _, alpha = pb.visit_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    assert 0.35 < alpha < 0.7


def test_single_category_is_a_no_op():
    n = 6
    a = synth.simulate(n, 300, 614, model="jc")
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 1.0, 1)
    f0, l0, _ = pb.full_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    pb.set_reopt_alpha(True)
    f, l, alpha = pb.visit_optimise(a.tree_edges, np.full(2 * n - 3, 0.1))
    assert alpha == 1.0 and f == f0
    np.testing.assert_array_equal(l, l0)


def test_search_with_shape_reoptimisation_visits_every_topology():
    n = 5
    a = synth.simulate(n, 200, 615, model="gtr", alpha=0.5)
    tips, w = synth.compress_patterns(a.codes)
    pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
    pb.set_reopt_alpha(True)
    e, l = synth.random_trees(n, 1, 616)
    s = oracle.Search(pb, e, l, float("inf"))
    s.run()
    assert len(s.visited()["keys"]) == 15
