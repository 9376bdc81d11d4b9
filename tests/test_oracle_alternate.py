"""Pins for the oracle's Algorithm 2 alternation (nu update from a fixed fit)."""
import numpy as np

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl


def test_planted_two_features_stay_exact():
    # p = 2: Delta_nu is the k = 2 embedding distance of X itself for every nu,
    # so Y0 = X is a zero of both losses and fits every grid value exactly
    X = wl.heavy_tailed(50, 2, "student", seed=980)
    for loss in ("sammon", "kruskal"):
        Y, path, ks = orc.alternating_nu(X, [1.3, 2.0, 3.5], 1.7, 2, 5, X, loss=loss)
        assert np.all(ks < 1e-12)
        np.testing.assert_allclose(Y, X, atol=1e-12)


def test_ks_table_by_closed_form():
    # no fitting steps: the table is KS of Y0 against each Delta_nu, with the
    # k = 2 embedding distance written out as 2^(1-nu) |(y_i0 - y_i1) - (y_j0 - y_j1)|
    n, nus = 40, [1.2, 2.0, 2.7, 4.0]
    X = wl.heavy_tailed(n, 6, "lognormal", seed=981)
    Y0 = wl.y_init(n, 2, seed=982, sd=1.0).astype(np.float64)
    _, path, ks = orc.alternating_nu(X, nus, 2.0, 1, 0, Y0)
    D, s2 = orc.delta(X, nus)
    u = Y0[:, 0] - Y0[:, 1]
    iu = np.triu_indices(n, 1)
    for v, nu in enumerate(nus):
        d = 2.0 ** (1.0 - nu) * np.abs(u[:, None] - u[None, :])
        want = np.sqrt(np.sum((d[iu] - D[v][iu]) ** 2) / np.sum(D[v][iu] ** 2))
        assert abs(ks[0, v] - want) <= 1e-12 * want
    assert path == [2.0, nus[int(np.argmin(ks[0]))]]
