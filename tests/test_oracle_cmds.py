"""Pins for the oracle's classical MDS: textbook facts of Section IV-A."""
import numpy as np

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl


def _euclid(X):
    return np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))


def test_recovers_a_euclidean_configuration():
    # Delta = Euclidean distances of X (n x q): classical MDS in q dimensions
    # reproduces every distance, and its eigenvalues are the squared singular
    # values of the centred X.
    X = wl.y_init(40, 3, seed=1, sd=1.0).astype(np.float64)
    D = _euclid(X)
    Y, lam = orc.classical_mds(D, 3)
    np.testing.assert_allclose(_euclid(Y), D, atol=1e-10)
    sv = np.linalg.svd(X - X.mean(0), compute_uv=False)
    np.testing.assert_allclose(lam, sv ** 2, rtol=1e-10)


def test_rotation_and_translation_invariance_and_truncation():
    X = wl.y_init(30, 4, seed=2, sd=1.0).astype(np.float64)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))
    _, lam1 = orc.classical_mds(_euclid(X), 2)
    _, lam2 = orc.classical_mds(_euclid(X @ Q + 5.0), 2)
    np.testing.assert_allclose(lam1, lam2, rtol=1e-10)
    # the top-2 embedding is the best rank-2 approximation of the centred Gram matrix
    Xc = X - X.mean(0)
    U, s, _ = np.linalg.svd(Xc, full_matrices=False)
    Y, _ = orc.classical_mds(_euclid(X), 2)
    np.testing.assert_allclose(Y @ Y.T, (U[:, :2] * s[:2]) @ (U[:, :2] * s[:2]).T, atol=1e-9)
