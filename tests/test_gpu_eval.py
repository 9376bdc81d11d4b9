"""Evaluation measures (Section V) on the GPU against the oracle's definitions."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _case(kind, n, seed):
    if kind == "mixture":
        X = wl.gaussian_mixture(n, 6, seed=seed, n_clusters=4)
        Y = X[:, :2] + 0.5 * np.random.default_rng(seed).standard_normal((n, 2)).astype(np.float32)
    elif kind == "integer":  # exact ties in both spaces
        X = wl.integer_valued(n, 5, seed=seed, levels=3)
        Y = X[:, :2].copy()
    else:  # image rows, a 3-d embedding
        X = wl.image_like(n, seed=seed)
        Y = wl.y_init(n, 3, seed=seed + 1, sd=1.0)
    labels = (X[:, 0] > np.median(X[:, 0])).astype(np.int32)
    return np.ascontiguousarray(X, dtype=np.float32), np.ascontiguousarray(Y, dtype=np.float32), labels


def _cuda(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


@pytest.mark.parametrize("kind,n", [("mixture", 300), ("integer", 257), ("image", 150)])
def test_neighbour_scores(G, kind, n):
    X, Y, labels = _case(kind, n, 1000)
    Xd, Yd, Ld = _cuda(X, Y, labels)
    for kt, knn in [(5, 10), (1, 1), (12, 0), (0, 7)]:
        out = G.gini_neighbour_scores(Xd, Yd, Ld if knn else None, kt, knn).cpu().numpy()
        if kt:
            assert out[0] == pytest.approx(orc.trustworthiness(X, Y, kt), abs=1e-12), (kt, knn)
        else:
            assert np.isnan(out[0])
        if knn:
            assert out[1] == pytest.approx(orc.nn_agreement(Y, labels, knn), abs=1e-12)
        else:
            assert np.isnan(out[1])


@pytest.mark.parametrize("kind,n", [("mixture", 300), ("integer", 257), ("image", 150)])
def test_silhouette(G, kind, n):
    X, Y, labels = _case(kind, n, 1010)
    Yd, Ld = _cuda(Y, labels)
    assert float(G.gini_silhouette(Yd, Ld)) == pytest.approx(orc.silhouette(Y, labels), rel=1e-10)
    lab5 = (np.arange(n) % 5).astype(np.int32)
    lab5[3] = 5  # a singleton label
    (L5,) = _cuda(lab5)
    assert float(G.gini_silhouette(Yd, L5)) == pytest.approx(orc.silhouette(Y, lab5), rel=1e-10)


@pytest.mark.parametrize("kind,n", [("mixture", 300), ("integer", 257), ("image", 150),
                                    ("mixture", 1100)])
def test_distance_correlations(G, kind, n):
    # n = 1100: 604,450 pairs, 296 radix tiles, a two-level scan of the histogram
    X, Y, _ = _case(kind, n, 1020)
    Xd, Yd = _cuda(X, Y)
    p, s = G.gini_distance_correlations(Xd, Yd).cpu().numpy()
    pr, sr = orc.distance_correlations(X, Y)
    assert p == pytest.approx(pr, abs=1e-10)
    assert s == pytest.approx(sr, abs=1e-10)
    p2, s2 = G.gini_distance_correlations(Xd, Yd, spearman=False).cpu().numpy()
    assert p2 == pytest.approx(pr, abs=1e-10) and np.isnan(s2)


def test_small_sizes_and_errors(G):
    from paper_2605_25124_gb300._lib import GiniError
    X, Y, labels = _case("mixture", 3, 1030)
    Xd, Yd, Ld = _cuda(X, Y, labels)
    p, s = G.gini_distance_correlations(Xd, Yd).cpu().numpy()
    pr, sr = orc.distance_correlations(X, Y)
    assert p == pytest.approx(pr, abs=1e-10) and s == pytest.approx(sr, abs=1e-10)
    with pytest.raises(GiniError, match="EINVAL"):
        G.gini_neighbour_scores(Xd, Yd, Ld, 3, 1)  # k >= n
    X2, Y2, _ = _case("mixture", 2, 1031)
    X2d, Y2d = _cuda(X2, Y2)
    with pytest.raises(GiniError, match="EINVAL"):
        G.gini_neighbour_scores(X2d, Y2d, None, 1, 0)  # 2n - 3k - 1 = 0
