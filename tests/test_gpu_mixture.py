"""The adjoint-check configuration: n = 5,000, p = 50 Gaussian mixture (10
clusters, 3 % Student-t(1.5) rows), k in {2, 3}, FP32 Y.

* GiniStress (the torch.autograd.Function) gradient against central
  differences of the exact stress (FP64, h = 1e-3, reduced near kinks) on 64
  random entries, and against the oracle's gradient rows for the same points
  (relative 1e-3 for the differences, 1e-5 of the largest entry for the
  oracle).  At n = 5,000 the FP32 rounding of the GPU's own stress is as large
  as the change a step of 1e-4 makes, so the differences come from the
  oracle's FP64 pieces (only the pairs holding the moved point change).
* A 500-iteration fit (tiled FP32, deterministic mode) against the oracle's
  500 fixed-step iterations from the same Y0 and step: the stress history
  within the stated bound.
"""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NAME = "mixture-n5000-p50"


@pytest.fixture(scope="module")
def mixture(G):
    w = wl.WORKLOADS[NAME]
    X = wl.make_X(NAME)
    mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), [2.0], layout="full")
    return w, X, mats[0], float(sd2[0])


def _kink_gap(Y, i, c):
    """Distance, along y_ic, to the nearest tie of z_a and z_b over the pairs
    (a, b) of components containing c (where the stress has a kink)."""
    k = Y.shape[1]
    gap = np.inf
    for a in range(k):
        for b in range(a + 1, k):
            if c in (a, b):
                v = Y[:, a].astype(np.float64) - Y[:, b]
                gap = min(gap, np.abs(v[i] - np.delete(v, i)).min())
    return gap


@pytest.mark.parametrize("k", [2, 3])
def test_autograd_gradient_against_central_differences_64_entries(G, mixture, k):
    w, X, Dfull, sd2 = mixture
    n, nu = w["n"], 2.0
    Y = wl.y_init(n, k, seed=7100 + k, sd=1.0)
    Dt = G.gini_pack(Dfull, "f32")
    Yt = torch.from_numpy(Y).cuda().requires_grad_(True)
    S = G.GiniStress.apply(Yt, nu, Dt)
    S.backward()
    g = Yt.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(7200 + k)
    entries = []
    while len(entries) < 64:
        i, c = int(rng.integers(n)), int(rng.integers(k))
        gap = _kink_gap(Y, i, c)
        if gap > 1e-4:  # differences need a step well above FP32 rounding
            entries.append((i, c, float(min(1e-3, 0.3 * gap))))
    # Central differences of the exact (FP64) stress: only the pairs holding
    # point i change, so S(Y+) - S(Y-) is their sum, from the oracle's
    # dissimilarities and embedding distances.
    rows = np.array(sorted({i for i, _, _ in entries}))
    I = np.repeat(rows, n)
    J = np.tile(np.arange(n), len(rows))
    Drows = orc.delta_pairs(X, [nu], I, J)[:, 0].reshape(len(rows), n)
    others = np.arange(n)
    gmax = np.abs(g).max()
    for i, c, h in entries:
        drow = Drows[np.searchsorted(rows, i)]
        keep = others != i
        Yp, Ym = Y.astype(np.float64), Y.astype(np.float64)
        Yp[i, c] = float(np.float32(Y[i, c]) + np.float32(h))
        Ym[i, c] = float(np.float32(Y[i, c]) - np.float32(h))
        Ii = np.full(n - 1, i)
        dp = orc.embed_dist_pairs(Yp, nu, Ii, others[keep])
        dm = orc.embed_dist_pairs(Ym, nu, Ii, others[keep])
        dS = np.sum((dp - drow[keep]) ** 2 - (dm - drow[keep]) ** 2) / sd2
        fd = dS / (Yp[i, c] - Ym[i, c])
        assert g[i, c] == pytest.approx(fd, rel=1e-3, abs=1e-3 * gmax), (i, c, h)
    # the oracle's gradient for the same points
    gref = orc.grad_rows(Y.astype(np.float64), nu, Drows, rows, sd2)
    err = np.max(np.abs(g[rows] - gref))
    assert err <= 1e-5 * np.abs(gref).max(), err / np.abs(gref).max()


def test_fit_500_iterations_against_the_oracle(G, mixture):
    w, X, Dfull, sd2 = mixture
    n, k, nu, T = w["n"], w["k"], 2.0, w["iters"]
    Dref, sref = orc.delta(X, [nu])
    assert sd2 == pytest.approx(sref[0], rel=1e-6)
    Y0 = wl.y_init(n, k, seed=w["seed"] + 1000)
    eta = orc.default_step(n, k, nu, sref[0], 1.0)
    Yr, href = orc.fit(Dref[0], nu, sref[0], Y0.astype(np.float64), eta, T)
    Dt = G.gini_pack(Dfull, "f32")
    Y, hist, final = G.gini_mds_fit(torch.from_numpy(Y0).cuda(), nu, Dt, eta, T,
                                    deterministic=True)
    h = hist.cpu().numpy()
    rel = np.abs(h - href) / href
    yerr = np.abs(Y.cpu().numpy() - Yr).max() / np.abs(Yr).max()
    print(f"500 iterations: history max rel {rel.max():.3e} (first 50: {rel[:50].max():.3e}), "
          f"Y max rel {yerr:.3e}, S {h[-1]:.6f} vs {href[-1]:.6f}")
    assert rel[:50].max() <= 1e-5
    assert rel.max() <= 1e-4
    assert h[-1] < 0.5 * h[0]
