"""Pins of the oracle's entropy, entropy filter and relevancy score against
closed forms, library routines and brute force (no GPU)."""
import numpy as np
import pytest
import scipy.special
import scipy.stats


def test_entropy_closed_forms(oracle_lib):
    L = 7
    acc = np.zeros((5, L))
    acc[0] = 1.0                       # uniform over L atoms: log L
    acc[1, 3] = 2.5                    # one-hot: 0
    acc[2, [1, 4]] = 0.3               # two equal atoms: log 2
    acc[3] = 0.0                       # empty row: 0 by definition
    acc[4] = [-1.0, 0.0, 2.0, 2.0, -5.0, 0.0, 0.0]  # non-positive entries ignored: log 2
    H = oracle_lib.entropy(acc)
    np.testing.assert_allclose(H, [np.log(L), 0.0, np.log(2), 0.0, np.log(2)], rtol=1e-14, atol=1e-15)


def test_entropy_matches_scipy_and_is_scale_invariant(oracle_lib):
    rng = np.random.default_rng(0)
    acc = rng.dirichlet(np.full(64, 0.3), size=200) * rng.uniform(0.1, 50.0, size=(200, 1))
    acc[acc < 1e-3] = 0.0
    H = oracle_lib.entropy(acc)
    np.testing.assert_allclose(H, scipy.stats.entropy(acc, axis=1), rtol=1e-12)
    np.testing.assert_allclose(oracle_lib.entropy(acc * 1e3), H, rtol=1e-12)


def test_entropy_filter_brute_force(oracle_lib):
    rng = np.random.default_rng(1)
    H = np.round(rng.random(997), 2)  # many ties
    for keep in (0, 1, 498, 996, 997, 2000):
        m = oracle_lib.entropy_filter(H, keep)
        order = np.lexsort((np.arange(H.size), H))  # by H, then index
        want = np.zeros(H.size, np.uint8)
        want[order[:min(keep, H.size)]] = 1
        np.testing.assert_array_equal(m, want)


def test_relevancy_sigmoid_form(oracle_lib):
    rng = np.random.default_rng(2)
    sq = rng.uniform(-1, 1, 300)
    sc = rng.uniform(-1, 1, (300, 1))
    R = oracle_lib.relevancy(sq, sc, alpha=10.0)
    np.testing.assert_allclose(R, scipy.special.expit(10.0 * (sq - sc[:, 0])), rtol=1e-12)


def test_relevancy_invariants(oracle_lib):
    rng = np.random.default_rng(3)
    sq = rng.uniform(-1, 1, 400)
    sc = rng.uniform(-1, 1, (400, 4))
    R = oracle_lib.relevancy(sq, sc, alpha=10.0)
    # the minimum over phrases is set by the most similar canonical phrase
    np.testing.assert_allclose(R, scipy.special.expit(10.0 * (sq - sc.max(axis=1))), rtol=1e-12)
    assert ((R <= 0.5) == (sc.max(axis=1) >= sq)).all()
    # a query identical to a canonical phrase scores exactly 1/2
    sc[:, 2] = sq
    assert np.all(oracle_lib.relevancy(sq, sc, alpha=10.0) <= 0.5 + 1e-15)
