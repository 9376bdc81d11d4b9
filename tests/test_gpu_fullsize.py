"""Parity at the benchmark's full size, in the configuration bench.py times:
image-like data n = 20,000, p = 784, nu = 2, Delta in the tiled FP32 layout,
the fused k = 2 kernel.  The oracle cannot build the whole matrix in seconds,
so it checks sampled outputs it computes one by one (random pairs and whole
rows of Delta, whole rows of the gradient at the seeded Y0); the global sum of
delta^2 is checked as a property (FP64 sum of the stored values).

Tolerances as elsewhere: Delta per entry 1e-5 relative (floor 1e-6 x max);
gradient max-abs 1e-5 x max |grad|.
"""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import rel_err, tiled_flat_index

pytestmark = pytest.mark.gpu

NAME = "image-n20000-p784"


@pytest.fixture(scope="module")
def full(G):
    w = wl.WORKLOADS[NAME]
    X = wl.make_X(NAME)
    Xd = torch.from_numpy(X).cuda()
    mats, sd2 = G.gini_dist(Xd, [2.0], layout="tiled", dtype="f32")
    return w, X, Xd, mats[0], float(sd2[0])


def test_fullsize_delta_sampled_pairs_and_row(G, full):
    w, X, Xd, D, _ = full
    n = w["n"]
    rng = np.random.default_rng(20000)
    I = rng.integers(0, n, 400)
    J = rng.integers(0, n, 400)
    keep = I != J
    I, J = np.minimum(I[keep], J[keep]), np.maximum(I[keep], J[keep])
    row = 12345
    I = np.concatenate([I, np.full(n - 1 - row, row), np.arange(row)])
    J = np.concatenate([J, np.arange(row + 1, n), np.full(row, row)])
    ref = orc.delta_pairs(X, [2.0], I, J)[:, 0]
    idx = torch.from_numpy(tiled_flat_index(I, J, n)).cuda()
    got = D.data[idx].double().cpu().numpy()
    assert rel_err(got, ref, 1e-6 * np.abs(ref).max()) <= 1e-5


def test_fullsize_full_layout_and_sum_of_squares(G, full):
    w, X, Xd, D, sd2 = full
    n = w["n"]
    mats, s_full = G.gini_dist(Xd, [2.0], layout="full")
    F = mats[0].data
    # the two layouts hold the same values (one build, two stores)
    rng = np.random.default_rng(20001)
    I = rng.integers(0, n - 1, 5000)
    J = I + 1 + rng.integers(0, n - 1 - I)
    a = F[torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()]
    b = D.data[torch.from_numpy(tiled_flat_index(I, J, n)).cuda()]
    assert torch.equal(a, b)
    assert torch.equal(F, F.t())
    assert float(F.diagonal().abs().max()) == 0.0
    # the kernel's FP64 sum_{i<j} delta^2 against the FP64 sum of what it stored
    tot = 0.0
    for r0 in range(0, n, 2000):
        blk = F[r0:r0 + 2000].double()
        tot += float((blk * blk).sum())
    assert float(s_full[0]) == pytest.approx(0.5 * tot, rel=1e-9)
    assert sd2 == pytest.approx(float(s_full[0]), rel=1e-12)
    del F, mats


def test_fullsize_gradient_sampled_rows(G, full):
    w, X, Xd, D, _ = full
    n, k, nu = w["n"], w["k"], 2.0
    Y = wl.y_init(n, k, seed=w["seed"] + 1000)  # the benchmark's Y0
    Dg = G.Dissimilarity(D.data, n, "tiled", "f32", 1.0)  # sum_delta2 = 1 on both sides
    _, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dg)
    rows = np.array([0, 777, 12345, n - 1])
    I = np.repeat(rows, n)
    J = np.tile(np.arange(n), len(rows))
    Drows = orc.delta_pairs(X, [nu], I, J)[:, 0].reshape(len(rows), n)
    gref = orc.grad_rows(Y.astype(np.float64), nu, Drows, rows, 1.0)
    err = np.max(np.abs(g.cpu().numpy()[rows] - gref))
    assert err <= 1e-5 * np.abs(gref).max(), err / np.abs(gref).max()


def test_fullsize_deterministic_fit_repeats_and_resumes(G, full):
    # The benchmark's fit (200 fused iterations, tiled FP32) in deterministic
    # mode: two runs give the same bits, and 100 + 100 iterations from the
    # fit's own Y_100 give the same Y_200 and S(Y_200) as 200 in one call.
    w, X, Xd, D, sd2 = full
    n, k, nu, T = w["n"], w["k"], 2.0, w["iters"]
    Y0 = torch.from_numpy(wl.y_init(n, k, seed=w["seed"] + 1000)).cuda()
    eta = G.default_step(n, k, nu, sd2)
    Ya, ha, Sa = G.gini_mds_fit(Y0, nu, D, eta, T, deterministic=True)
    Yb, hb, Sb = G.gini_mds_fit(Y0, nu, D, eta, T, deterministic=True)
    assert torch.equal(Ya, Yb) and torch.equal(ha, hb) and float(Sa) == float(Sb)
    Y1, _, _ = G.gini_mds_fit(Y0, nu, D, eta, T // 2, deterministic=True)
    Y2, _, S2 = G.gini_mds_fit(Y1, nu, D, eta, T - T // 2, deterministic=True)
    assert torch.equal(Y2, Ya) and float(S2) == float(Sa)


def test_fullsize_gradient_rows_at_the_fits_scale(G, full):
    # Near the end of a fit the residuals d - delta are small next to d and
    # delta, which is where cancellation would show.  The evaluation point is
    # built on the host: the seeded Y0 scaled by the factor that best matches
    # the embedding distances to the dissimilarities over a sample of pairs
    # (both from the oracle), so no output of the CUDA path feeds the oracle.
    w, X, Xd, D, _ = full
    n, k, nu = w["n"], w["k"], 2.0
    Y0 = wl.y_init(n, k, seed=w["seed"] + 1000).astype(np.float64)
    rng = np.random.default_rng(20002)
    I = rng.integers(0, n, 3000)
    J = (I + 1 + rng.integers(0, n - 1, 3000)) % n
    dl = orc.delta_pairs(X, [nu], I, J)[:, 0]
    u = Y0[:, 0] - Y0[:, 1]
    d = 2.0 ** (1.0 - nu) * np.abs(u[I] - u[J])  # k = 2 closed form of the pseudo-distance
    alpha = float(np.dot(d, dl) / np.dot(d, d))
    Y = (alpha * Y0).astype(np.float32)
    Dg = G.Dissimilarity(D.data, n, "tiled", "f32", 1.0)
    _, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dg)
    rows = np.array([3, 4321, 15000, n - 2])
    Ir = np.repeat(rows, n)
    Jr = np.tile(np.arange(n), len(rows))
    Drows = orc.delta_pairs(X, [nu], Ir, Jr)[:, 0].reshape(len(rows), n)
    gref = orc.grad_rows(Y.astype(np.float64), nu, Drows, rows, 1.0)
    err = np.max(np.abs(g.cpu().numpy()[rows] - gref))
    assert err <= 1e-5 * np.abs(gref).max(), err / np.abs(gref).max()
