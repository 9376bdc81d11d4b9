"""Euclidean embedding distance and Sammon loss on the GPU against the oracle."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import host_col_scale, quantize, tile_pack

pytestmark = pytest.mark.gpu


def _upload(G, D, n, form, sd2):
    if form == "full":
        return G.Dissimilarity(torch.from_numpy(D.astype(np.float32)).cuda(), n, "full", "f32", sd2)
    sc = host_col_scale(D) if form == "fp8" else None
    return G.Dissimilarity(torch.from_numpy(tile_pack(D, n, form, sc)).cuda(), n, "tiled", form,
                           sd2, torch.from_numpy(sc).cuda() if sc is not None else None)


def _problem(n, nu, seed):
    X = wl.gaussian_outliers(n, 7, seed=seed)
    D = orc.delta(X, [nu])[0][0]
    iu = np.triu_indices(n, 1)
    return D, float(np.sum(D[iu])), float(np.sum(D[iu] ** 2))


@pytest.mark.parametrize("form", ["full", "f32", "bf16x2"])
def test_delta_sums(G, form):
    n = 300
    D, s1, s2 = _problem(n, 1.6, 800)
    Dq = quantize(D, "f32" if form == "full" else form)
    iu = np.triu_indices(n, 1)
    got = G.gini_delta_sums(_upload(G, D, n, form, s2)).cpu().numpy()
    assert got[0] == pytest.approx(np.sum(Dq[iu]), rel=1e-12)
    assert got[1] == pytest.approx(np.sum(Dq[iu] ** 2), rel=1e-12)


@pytest.mark.parametrize("form", ["full", "f32", "bf16x2"])
@pytest.mark.parametrize("metric,loss", [("euclid", "kruskal"), ("euclid", "sammon"),
                                         ("gini", "sammon")])
@pytest.mark.parametrize("k", [2, 3])
def test_stress_grad_losses(G, form, metric, loss, k):
    n, nu = 300, 1.8
    D, s1, s2 = _problem(n, nu, 810 + k)
    norm = s2 if loss == "kruskal" else s1
    Dq = quantize(D, "f32" if form == "full" else form)
    Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
    Y = wl.y_init(n, k, seed=811, sd=1.0)
    Sref, gref = orc.stress_grad_ex(Y.astype(np.float64), nu, Dq, norm, metric, loss)
    S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, _upload(G, D, n, form, s2),
                              metric=metric, loss=loss, norm=norm)
    assert float(S) == pytest.approx(Sref, rel=1e-5)
    assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max()


@pytest.mark.parametrize("metric,loss", [("euclid", "kruskal"), ("euclid", "sammon"),
                                         ("gini", "sammon")])
def test_fit_one_step_losses(G, metric, loss):
    n, k, nu = 200, 2, 2.0
    D, s1, s2 = _problem(n, nu, 820)
    norm = s2 if loss == "kruskal" else s1
    Y0 = wl.y_init(n, k, seed=821, sd=1.0)
    eta = 0.05 * norm / n
    _, gref = orc.stress_grad_ex(Y0.astype(np.float64), nu, D, norm, metric, loss)
    for form in ("full", "f32"):
        Y1, hist, _ = G.gini_mds_fit(torch.from_numpy(Y0).cuda(), nu, _upload(G, D, n, form, s2),
                                     eta, 1, metric=metric, loss=loss, norm=norm)
        step = Y1.cpu().numpy().astype(np.float64) - Y0
        assert np.max(np.abs(step + eta * gref)) <= (1e-5 * eta * np.abs(gref).max()
                                                    + 2e-7 * np.abs(Y0).max())
    # a longer Euclidean fit decreases the stress monotonically at this step
    _, h, _ = G.gini_mds_fit(torch.from_numpy(Y0).cuda(), nu, _upload(G, D, n, "f32", s2), eta,
                             50, metric=metric, loss=loss, norm=norm)
    h = h.cpu().numpy()
    assert h[-1] < h[0] and np.all(np.diff(h) <= 1e-7 * h[0])


def test_euclid_planted_zero_stress(G):
    n, k = 250, 2
    Ys = wl.y_init(n, k, seed=830, sd=1.0)
    D = np.sqrt(((Ys[:, None, :].astype(np.float64) - Ys[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(n, 1)
    for loss, norm in (("kruskal", np.sum(D[iu] ** 2)), ("sammon", np.sum(D[iu]))):
        S, g = G.gini_stress_grad(torch.from_numpy(Ys).cuda(), 2.0, _upload(G, D, n, "f32", 1.0),
                                  metric="euclid", loss=loss, norm=norm)
        assert float(S) < 1e-12
