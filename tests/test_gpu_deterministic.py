"""Deterministic mode (gini_set_deterministic, gini_fit_args.deterministic, the
batched call's flag): fixed-order reductions make repeated runs bit-identical
and a resumed fit continue bit for bit; the results stay within the usual
tolerances of the oracle and of the default (atomic) mode."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _delta(G, X, nu, dtype):
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="tiled", dtype=dtype)
    return mats[0]


@pytest.mark.parametrize("k,dtype", [(2, "f32"), (2, "bf16x2"), (3, "f32"), (5, "bf16")])
def test_fit_repeats_bit_for_bit_and_resumes(G, k, dtype):
    n, nu, T = 777, 1.7, 30  # 7 tiles per edge, ragged tail
    X = wl.gaussian_mixture(n, 12, seed=610 + k)
    D = _delta(G, X, nu, dtype)
    Y0 = torch.from_numpy(wl.y_init(n, k, seed=611, sd=1.0)).cuda()
    eta = G.default_step(n, k, nu, D.sum_delta2)
    runs = [G.gini_mds_fit(Y0, nu, D, eta, T, polish_iters=T, deterministic=True)
            for _ in range(3)]
    for Y, h, S in runs[1:]:
        assert torch.equal(Y, runs[0][0])
        assert torch.equal(h, runs[0][1]) and float(S) == float(runs[0][2])
    # resume: 15 + 15 iterations from the fit's own Y_15 equal 30 in one call
    Y15, _, _ = G.gini_mds_fit(Y0, nu, D, eta, 15, polish_iters=15, deterministic=True)
    Y30, _, S30 = G.gini_mds_fit(Y15, nu, D, eta, 15, polish_iters=15, deterministic=True)
    assert torch.equal(Y30, runs[0][0]) and float(S30) == float(runs[0][2])
    # and the default (atomic) mode follows the same path within rounding
    Ya, ha, _ = G.gini_mds_fit(Y0, nu, D, eta, T, polish_iters=T)
    np.testing.assert_allclose(ha.cpu().numpy(), runs[0][1].cpu().numpy(), rtol=1e-4)


@pytest.mark.parametrize("k", [2, 3])
def test_deterministic_gradient_matches_the_oracle(G, k):
    n, nu = 300, 2.5
    X = wl.gaussian_outliers(n, 9, seed=620 + k)
    Dref, sref = orc.delta(X, [nu])
    D = _delta(G, X, nu, "f32")
    Y0 = wl.y_init(n, k, seed=621, sd=1.0)
    with G.deterministic():
        assert G.is_deterministic()
        S, g = G.gini_stress_grad(torch.from_numpy(Y0).cuda(), nu, D)
        S2, g2 = G.gini_stress_grad(torch.from_numpy(Y0).cuda(), nu, D)
    assert not G.is_deterministic()
    assert torch.equal(g, g2) and float(S) == float(S2)
    Sref, gref = orc.stress_grad(Y0.astype(np.float64), nu, Dref[0], sref[0])
    assert float(S) == pytest.approx(Sref, rel=1e-5)
    assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max()


def test_batched_fits_repeat_bit_for_bit(G):
    Xs = wl.uci_like_batch(6, seed=630)
    Xs = [X[: min(len(X), 700)] for X in Xs]
    nus, R, T = [1.3, 2.0, 3.1], 3, 12
    ns = [len(X) for X in Xs]
    Y0 = torch.from_numpy(np.concatenate(
        [wl.y_init(R * n, 2, seed=631 + q).reshape(-1) for q, n in enumerate(ns)])).cuda()
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    a = G.gini_fit_batched(Xd, nus, R, T, Y0, history=True, deterministic=True)
    a = {key: (v.clone() if torch.is_tensor(v) else v) for key, v in a.items()}
    b = G.gini_fit_batched(Xd, nus, R, T, Y0, history=True, deterministic=True)
    assert torch.equal(a["Y"], b["Y"]) and torch.equal(a["history"], b["history"])
    c = G.gini_fit_batched(Xd, nus, R, T, Y0, history=True)
    np.testing.assert_allclose(c["history"].cpu().numpy(), a["history"].cpu().numpy(),
                               rtol=1e-4)


def test_nu_search_repeats_bit_for_bit(G):
    n, p = 600, 10
    X = wl.gaussian_mixture(n, p, seed=640)
    fold = (np.arange(n) % 3).astype(np.int32)
    nus = [1.3, 1.9, 2.6, 3.4]
    Y0 = torch.from_numpy(wl.y_init(2 * n, 2, seed=641).reshape(2, n, 2)).cuda()
    with G.deterministic():
        r1 = G.gini_nu_search(torch.from_numpy(X).cuda(), fold, nus, 2, 10, Y0)
        r1 = {key: v.clone() for key, v in r1.items()}
        r2 = G.gini_nu_search(torch.from_numpy(X).cuda(), fold, nus, 2, 10, Y0)
    for key in r1:
        assert torch.equal(r1[key], r2[key]), key
