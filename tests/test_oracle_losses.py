"""Pins for the oracle's Euclidean embedding distance and Sammon loss."""
import numpy as np
import pytest

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl


def _delta(n, seed):
    D = orc.delta(wl.gaussian_outliers(n, 6, seed=seed), [1.7])[0][0]
    iu = np.triu_indices(n, 1)
    return D, float(np.sum(D[iu])), float(np.sum(D[iu] ** 2))


def test_euclid_kruskal_two_points():
    Y = np.array([[0.0, 0.0], [3.0, 4.0]])
    D = np.array([[0.0, 2.0], [2.0, 0.0]])
    S, g = orc.stress_grad_ex(Y, 2.0, D, 4.0, metric="euclid", loss="kruskal")
    assert S == pytest.approx((5.0 - 2.0) ** 2 / 4.0)
    # dS/dy_0 = 2 (d - delta)/norm * (y_0 - y_1)/d
    np.testing.assert_allclose(g[0], 2 * 3.0 / 4.0 * np.array([-3.0, -4.0]) / 5.0)
    np.testing.assert_allclose(g[1], -g[0])


def test_sammon_two_points_and_constant_delta():
    Y = np.array([[1.0, 0.0], [0.0, 0.0]])
    D = np.array([[0.0, 4.0], [4.0, 0.0]])
    S, _ = orc.stress_grad_ex(Y, 2.0, D, 4.0, metric="euclid", loss="sammon")
    assert S == pytest.approx((1.0 - 4.0) ** 2 / 4.0 / 4.0)
    # with every delta equal to c, Sammon = Kruskal raw sum / (c * sum delta)
    n = 9
    Yr = wl.y_init(n, 3, seed=3, sd=1.0).astype(np.float64)
    C = np.full((n, n), 2.5) - 2.5 * np.eye(n)
    P = n * (n - 1) / 2
    Sk, _ = orc.stress_grad_ex(Yr, 1.5, C, 1.0, metric="gini", loss="kruskal", grad=False)
    Ss, _ = orc.stress_grad_ex(Yr, 1.5, C, 2.5 * P, metric="gini", loss="sammon", grad=False)
    assert Ss == pytest.approx(Sk / (2.5 * 2.5 * P), rel=1e-13)


@pytest.mark.parametrize("metric,loss", [("euclid", "kruskal"), ("euclid", "sammon"),
                                         ("gini", "sammon")])
def test_central_differences(metric, loss):
    n, k, nu = 12, 3, 1.7
    D, s1, s2 = _delta(n, 10)
    norm = s2 if loss == "kruskal" else s1
    Y = wl.y_init(n, k, seed=11, sd=1.0).astype(np.float64)
    _, g = orc.stress_grad_ex(Y, nu, D, norm, metric, loss)
    h = 1e-6
    for i in range(n):
        for c in range(k):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            fd = (orc.stress_grad_ex(Yp, nu, D, norm, metric, loss, grad=False)[0]
                  - orc.stress_grad_ex(Ym, nu, D, norm, metric, loss, grad=False)[0]) / (2 * h)
            assert g[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(g).max())


def test_euclid_planted_and_rotation_invariance():
    n, k = 15, 3
    Ys = wl.y_init(n, k, seed=12, sd=1.0).astype(np.float64)
    D = np.sqrt(((Ys[:, None, :] - Ys[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(n, 1)
    for loss, norm in (("kruskal", np.sum(D[iu] ** 2)), ("sammon", np.sum(D[iu]))):
        S, g = orc.stress_grad_ex(Ys, 2.0, D, norm, "euclid", loss)
        assert S == pytest.approx(0.0, abs=1e-28) and np.abs(g).max() < 1e-13
    # a rotation and a translation of the embedding leave Euclidean stress unchanged
    D2, _, s2 = _delta(n, 13)
    Y = wl.y_init(n, k, seed=14, sd=1.0).astype(np.float64)
    Q, _ = np.linalg.qr(np.random.default_rng(15).standard_normal((k, k)))
    a, _ = orc.stress_grad_ex(Y, 2.0, D2, s2, "euclid", "kruskal", grad=False)
    b, _ = orc.stress_grad_ex(Y @ Q + 0.7, 2.0, D2, s2, "euclid", "kruskal", grad=False)
    assert a == pytest.approx(b, rel=1e-12)


def test_gini_kruskal_matches_original_entry():
    n, k, nu = 14, 2, 2.3
    D, s1, s2 = _delta(n, 16)
    Y = wl.y_init(n, k, seed=17, sd=1.0).astype(np.float64)
    a, ga = orc.stress_grad_ex(Y, nu, D, s2, "gini", "kruskal")
    b, gb = orc.stress_grad(Y, nu, D, s2)
    assert a == pytest.approx(b, rel=1e-14)
    np.testing.assert_allclose(ga, gb, rtol=1e-13)
