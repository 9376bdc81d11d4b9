"""Pins for the oracle's evaluation measures (Section V): library routines and
special cases with known values."""
import numpy as np
import pytest

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl


def _data(n, p, k, seed):
    X = wl.gaussian_mixture(n, p, seed=seed, n_clusters=3).astype(np.float64)
    Y = X[:, :k] + 0.3 * np.random.default_rng(seed).standard_normal((n, k))
    labels = (X[:, 0] > np.median(X[:, 0])).astype(np.int32)
    return X, Y, labels


def test_trustworthiness_matches_sklearn():
    sk = pytest.importorskip("sklearn.manifold")
    X, Y, _ = _data(80, 6, 2, 990)
    for k in (1, 5, 10):
        assert orc.trustworthiness(X, Y, k) == pytest.approx(sk.trustworthiness(X, Y, n_neighbors=k),
                                                             abs=1e-12)


def test_trustworthiness_special_cases():
    X, _, _ = _data(40, 5, 2, 991)
    assert orc.trustworthiness(X, X, 5) == 1.0  # the identity keeps every neighbourhood
    # a hand case: points on a line, embedding reverses the middle pair
    X1 = np.array([[0.0], [1.0], [2.1], [3.3]])
    Y1 = np.array([[0.0], [2.1], [1.0], [3.3]])
    # k = 1: N_i in Y: 0->2, 1->2, 2->0, 3->1; ranks in X: r(0,2)=2, r(1,2)=2,
    # r(2,0)=3, r(3,1)=2 -> sum max(0, r-1) = 1+1+2+1 = 5; n k (2n-3k-1) = 16
    assert orc.trustworthiness(X1, Y1, 1) == pytest.approx(1.0 - 2.0 * 5 / 16, abs=1e-15)


def test_nn_agreement_by_hand():
    Y = np.array([[0.0, 0], [0.1, 0], [5, 5], [5.1, 5], [0.2, 0]])
    labels = np.array([0, 0, 1, 1, 1])
    # 1-NN: 0->1 (same), 1->0 (same), 2->3 (same), 3->2 (same), 4->1 (diff)
    assert orc.nn_agreement(Y, labels, 1) == pytest.approx(4 / 5, abs=1e-15)
    assert orc.nn_agreement(Y, np.zeros(5), 3) == 1.0


def test_silhouette_matches_sklearn():
    skm = pytest.importorskip("sklearn.metrics")
    _, Y, labels = _data(120, 6, 2, 992)
    assert orc.silhouette(Y, labels) == pytest.approx(skm.silhouette_score(Y, labels), abs=1e-12)
    lab3 = np.arange(120) % 3
    lab3[0] = 7  # a singleton label: s_0 = 0
    assert orc.silhouette(Y, lab3) == pytest.approx(skm.silhouette_score(Y, lab3), abs=1e-12)


def test_distance_correlations_match_scipy():
    st = pytest.importorskip("scipy.stats")
    from scipy.spatial.distance import pdist
    X, Y, _ = _data(70, 5, 2, 993)
    p, s = orc.distance_correlations(X, Y)
    assert p == pytest.approx(st.pearsonr(pdist(X), pdist(Y))[0], abs=1e-12)
    assert s == pytest.approx(st.spearmanr(pdist(X), pdist(Y))[0], abs=1e-12)
    # integer data: many tied distances, midranks
    Xi = wl.integer_valued(50, 4, seed=994, levels=3).astype(np.float64)
    Yi = Xi[:, :2]
    p, s = orc.distance_correlations(Xi, Yi)
    assert s == pytest.approx(st.spearmanr(pdist(Xi), pdist(Yi))[0], abs=1e-12)
    assert orc.distance_correlations(X, X) == pytest.approx((1.0, 1.0), abs=1e-12)
