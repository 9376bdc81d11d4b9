"""Pins for the oracle's Algorithm 1 composition (nu search over folds)."""
import numpy as np
import pytest

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl


def test_default_step_hand_case():
    # n = 3, k = 2, nu = 2, sum_delta2 = 1: w_max = 1/2, 2 (n-1) k ((k/2) w)^2 = 2
    assert orc.default_step(3, 2, 2.0, 1.0) == pytest.approx(0.5, rel=1e-15)
    assert orc.default_step(3, 2, 2.0, 1.0, eta0=0.25) == pytest.approx(0.125, rel=1e-15)
    assert orc.default_step(1, 2, 2.0, 1.0) == 0.0


def test_planted_two_features_fit_exactly():
    # with p = 2 a pair's Gini pseudo-distance is 2^(1-nu) |z_1 - z_2|, the k = 2
    # embedding distance of the points themselves: starting each fold at its own
    # rows gives KS = 0 for every nu -- which fails if a fold's starts and rows
    # are not the same points
    n = 60
    X = wl.gaussian_outliers(n, 2, seed=960)
    folds = np.arange(n) % 3
    Y0 = np.stack([X, X + 0.5]).astype(np.float64)  # restart 0 planted, 1 shifted by c.1
    ks, mean_ks, best, Y = orc.nu_search(X, folds, [1.3, 2.0, 4.0], Y0, iters=3)
    assert np.all(ks < 1e-12)
    np.testing.assert_allclose(Y, X, atol=1e-12)


def test_composition_by_hand():
    n, nus, R, T = 40, [1.5, 2.5], 2, 4
    X = wl.gaussian_outliers(n, 5, seed=961)
    folds = np.array([0] * 15 + [1] * 25)
    np.random.default_rng(0).shuffle(folds)
    Y0 = wl.y_init(R * n, 2, seed=962, sd=1.0).reshape(R, n, 2).astype(np.float64)
    ks, mean_ks, best, Y = orc.nu_search(X, folds, nus, Y0, iters=T)
    for q in range(2):
        idx = np.flatnonzero(folds == q)
        D, sd2 = orc.delta(X[idx], nus)
        for v, nu in enumerate(nus):
            finals = []
            for r in range(R):
                _, h = orc.fit(D[v], nu, sd2[v], Y0[r][idx], orc.default_step(len(idx), 2, nu,
                                                                               sd2[v]), T)
                finals.append(h[-1])
            assert ks[v, q] == pytest.approx(np.sqrt(min(finals)), rel=1e-12)  # OpenMP sum order
    assert np.allclose(mean_ks, ks.mean(1))
    assert best == int(np.argmin(mean_ks))
