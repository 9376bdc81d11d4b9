"""Classical MDS (Section IV-A) on the GPU against the oracle's eigendecomposition."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import host_col_scale, quantize, tile_pack

pytestmark = pytest.mark.gpu


def _upload(G, D, n, form):
    if form == "full":
        return G.Dissimilarity(torch.from_numpy(D.astype(np.float32)).cuda(), n, "full", "f32",
                               1.0)
    sc = host_col_scale(D) if form == "fp8" else None
    return G.Dissimilarity(torch.from_numpy(tile_pack(D, n, form, sc)).cuda(), n, "tiled", form,
                           1.0, torch.from_numpy(sc).cuda() if sc is not None else None)


def _stored(D, form):
    """The matrix the device sees (symmetric, float64)."""
    if form == "fp8":
        Dq = quantize(D, "fp8", host_col_scale(D))
    else:
        Dq = quantize(D, "f32" if form == "full" else form)
    U = np.triu(Dq, 1)
    return U + U.T


def _compare(Y, lam, Yr, lr, eig_tol=2e-5, sub_tol=1e-4):
    Y = Y.cpu().numpy().astype(np.float64)
    lam = lam.cpu().numpy()
    assert np.all(np.diff(lam) <= 0)
    assert np.max(np.abs(lam - lr)) <= eig_tol * abs(lr[0])
    # Y Y' is unique where the eigenvalues are (signs and rotations within a
    # repeated eigenvalue are not)
    P, Pr = Y @ Y.T, Yr @ Yr.T
    assert np.linalg.norm(P - Pr) <= sub_tol * np.linalg.norm(Pr)


def _planted(n, q, seed):
    Xs = wl.y_init(n, q, seed=seed, sd=1.0).astype(np.float64)
    return np.sqrt(((Xs[:, None, :] - Xs[None, :, :]) ** 2).sum(-1))


@pytest.mark.parametrize("form", ["full", "f32", "bf16x2", "bf16", "fp8"])
@pytest.mark.parametrize("k", [2, 3])
def test_planted_euclidean(G, form, k):
    # B has rank 3: the iterated block loses every other column (zeroed) and
    # the three eigenpairs are still exact
    n = 300
    D = _planted(n, 3, 900 + k)
    Yr, lr = orc.classical_mds(_stored(D, form), k)
    Y, lam = G.gini_classical_mds(_upload(G, D, n, form), k)
    _compare(Y, lam, Yr, lr)


@pytest.mark.parametrize("form", ["full", "f32", "bf16x2", "fp8"])
@pytest.mark.parametrize("nu", [1.5, 3.0])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_gini_dissimilarities(G, form, nu, k):
    # non-Euclidean: B has negative eigenvalues; n = 300 spans three tiles with
    # a ragged edge
    n = 300
    X = wl.gaussian_outliers(n, 7, seed=910)
    D = orc.delta(X, [nu])[0][0]
    Yr, lr = orc.classical_mds(_stored(D, form), k)
    Y, lam = G.gini_classical_mds(_upload(G, D, n, form), k, iters=30)
    _compare(Y, lam, Yr, lr)


def test_image_like_one_tile(G):
    n = 100
    X = wl.image_like(n, seed=920)
    D = orc.delta(X, [2.0])[0][0]
    for form in ("full", "f32"):
        Yr, lr = orc.classical_mds(_stored(D, form), 2)
        Y, lam = G.gini_classical_mds(_upload(G, D, n, form), 2)
        _compare(Y, lam, Yr, lr)


@pytest.mark.parametrize("n,k", [(2, 1), (2, 2), (5, 3), (16, 8), (17, 8), (129, 8)])
def test_small_and_edge_sizes(G, n, k):
    X = wl.gaussian_outliers(n, 5, seed=930 + n)
    D = orc.delta(X, [1.7])[0][0]
    Yr, lr = orc.classical_mds(D, k)
    for form in ("full", "f32"):
        Y, lam = G.gini_classical_mds(_upload(G, D, n, form), k, iters=40)
        lam_h = lam.cpu().numpy()
        assert np.max(np.abs(lam_h - lr)) <= 2e-5 * abs(lr[0])
        # where the top k are separated the embedding is unique up to Y Y'
        if k < n - 1 and np.min(np.abs(np.diff(lr))) > 1e-3 * abs(lr[0]):
            _compare(Y, lam, Yr, lr)


def test_seed_independence(G):
    n = 200
    D = orc.delta(wl.gaussian_outliers(n, 7, seed=940), [2.0])[0][0]
    Dd = _upload(G, D, n, "f32")
    Y1, l1 = G.gini_classical_mds(Dd, 2, seed=1)
    Y2, l2 = G.gini_classical_mds(Dd, 2, seed=12345)
    assert np.allclose(l1.cpu().numpy(), l2.cpu().numpy(), rtol=1e-5)
    P1, P2 = (Y.cpu().numpy().astype(np.float64) for Y in (Y1, Y2))
    assert np.linalg.norm(P1 @ P1.T - P2 @ P2.T) <= 1e-4 * np.linalg.norm(P1 @ P1.T)


def test_start_for_euclidean_fit(G):
    # on a planted Euclidean matrix the classical solution is already a zero of
    # the Euclidean Kruskal stress
    n = 250
    D = _planted(n, 2, 950)
    Dd = _upload(G, D, n, "f32")
    Y, _ = G.gini_classical_mds(Dd, 2)
    iu = np.triu_indices(n, 1)
    S, _ = G.gini_stress_grad(Y.contiguous(), 2.0, Dd, metric="euclid", loss="kruskal",
                              norm=float(np.sum(D[iu] ** 2)))
    assert float(S) < 1e-10


def test_argument_errors(G):
    from paper_2605_25124_gb300 import _lib
    L = _lib.lib()
    n = 50
    D = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    Y = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    lam = torch.empty(8, dtype=torch.float64, device="cuda")
    need = int(L.gini_cmds_workspace_size(n, 2))
    ws = torch.zeros(need, dtype=torch.uint8, device="cuda")
    args = lambda k, iters, wsb: (D.data_ptr(), n, 0, 0, n, None, k, iters, 0, Y.data_ptr(),
                                  lam.data_ptr(), ws.data_ptr(), wsb, None)
    EINVAL, ENOMEM = _lib.GINI_EINVAL, _lib.GINI_ENOMEM
    assert L.gini_classical_mds(*args(9, 10, need)) == EINVAL
    assert L.gini_classical_mds(*args(0, 10, need)) == EINVAL
    assert L.gini_classical_mds(*args(2, 0, need)) == EINVAL
    assert L.gini_classical_mds(*args(2, 10, need - 1)) == ENOMEM
    # a zero matrix: B = 0, every eigenvalue 0
    assert L.gini_classical_mds(*args(2, 10, need)) == 0
    torch.cuda.synchronize()
    assert np.all(lam[:2].cpu().numpy() == 0.0)
