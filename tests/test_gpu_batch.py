"""gini_fit_batched (many problems x nu grid x restarts in one graph) against
independent single fits on the GPU and against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import quantize

pytestmark = pytest.mark.gpu


def _batch(seed, ns, ps, restarts):
    Xs = [wl.gaussian_outliers(n, p, seed=seed + q) for q, (n, p) in enumerate(zip(ns, ps))]
    Y0s = [wl.y_init(restarts * n, 2, seed=seed + 100 + q, sd=1.0) for q, n in enumerate(ns)]
    return Xs, Y0s


def _slices(ns, n_nu, R):
    """Offsets of fit (q, v, r) in the batched Y output."""
    off, out = 0, {}
    for q, n in enumerate(ns):
        for v in range(n_nu):
            for r in range(R):
                out[q, v, r] = (off, off + 2 * n)
                off += 2 * n
    return out


def test_batched_matches_single_fits(G):
    ns, ps, nus, R, T = [150, 300, 77], [5, 12, 30], [1.5, 2.0, 3.0], 3, 20
    Xs, Y0s = _batch(500, ns, ps, R)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, T, Y0, eta0=1.0, history=True)
    Yb = out["Y"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    for q, n in enumerate(ns):
        mats, _ = G.gini_dist(Xd[q], nus, layout="full")
        for v, nu in enumerate(nus):
            D = G.gini_pack(mats[v], "f32")
            eta = G.default_step(n, 2, nu, D.sum_delta2, 1.0)
            for r in range(R):
                y0 = torch.from_numpy(Y0s[q][r * n:(r + 1) * n]).cuda()
                Ys, hs, fs = G.gini_mds_fit(y0, nu, D, eta, T)
                h = out["history"][:, q, v, r].cpu().numpy()
                hr = hs.cpu().numpy()
                assert np.max(np.abs(h - hr) / hr) <= 1e-4, (q, v, r)
                a, b = sl[q, v, r]
                Yq = Yb[a:b].reshape(n, 2)
                assert np.max(np.abs(Yq - Ys.cpu().numpy())) <= 1e-4 * np.abs(Yq).max()
                assert out["final"][q, v, r].item() == pytest.approx(float(fs), rel=1e-4)
    assert out["tuned"] in (1601, 1602, 1603, 801, 802)


def test_batched_one_step_against_oracle(G):
    ns, ps, nus, R = [130, 260], [7, 9], [1.3, 2.5], 2
    Xs, Y0s = _batch(600, ns, ps, R)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, 1, Y0, eta0=0.5, history=True)
    Yb = out["Y"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    for q, n in enumerate(ns):
        D, sd2 = orc.delta(Xs[q], nus)
        for v, nu in enumerate(nus):
            eta = G.default_step(n, 2, nu, sd2[v], 0.5)
            for r in range(R):
                y0 = Y0s[q][r * n:(r + 1) * n].astype(np.float64)
                y1, h = orc.fit(D[v], nu, sd2[v], y0, eta, 1)
                assert out["history"][0, q, v, r].item() == pytest.approx(h[0], rel=1e-5)
                a, b = sl[q, v, r]
                step = Yb[a:b].reshape(n, 2) - y0
                step_ref = y1 - y0
                assert np.max(np.abs(step - step_ref)) <= (1e-5 * np.abs(step_ref).max()
                                                          + 2e-7 * np.abs(y0).max())


def test_batched_graph_reuse_and_errors(G):
    from paper_2605_25124_gb300._lib import GiniError
    ns, ps, nus, R, T = [200, 90], [6, 4], [2.0], 2, 10
    Xs, Y0s = _batch(700, ns, ps, R)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    a = G.gini_fit_batched(Xd, nus, R, T, Y0)
    b = G.gini_fit_batched(Xd, nus, R, T, Y0)  # replays the cached graph from Y0
    np.testing.assert_allclose(a["final"].cpu().numpy(), b["final"].cpu().numpy(), rtol=1e-5)
    with pytest.raises(GiniError, match="EINVAL"):
        G.gini_fit_batched(Xd, nus, 17, T, torch.zeros(17 * 290 * 2, device="cuda"))
    with pytest.raises(GiniError, match="EINVAL"):
        G.gini_fit_batched(Xd, [0.9], R, T, Y0)


def test_batched_benchmark_configuration_sampled(G):
    """The benchmark's batch (64 UCI-sized problems x 8 nu x 8 restarts, the
    autotuned launch) for one iteration; the oracle rebuilds Delta for the
    three smallest problems and the smallest integer-valued one and
    checks S(Y0) and the first step of every nu and restart of those."""
    w = wl.WORKLOADS["uci-batch-64"]
    Xs = wl.uci_like_batch(w["n_problems"], w["seed"])
    R, nus = w["restarts"], [float(v) for v in w["nu"]]
    ns = [X.shape[0] for X in Xs]
    Y0s = [wl.y_init(R * n, 2, seed=w["seed"] + 1000 + q) for q, n in enumerate(ns)]
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, 1, Y0, eta0=1.0, history=True)
    Yb = out["Y"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    order = np.argsort(ns)
    ints = [q for q in order if q % 4 == 3]
    picks = sorted({int(q) for q in order[:3]} | {int(ints[0])})
    for q in picks:
        n = ns[q]
        D, sd2 = orc.delta(Xs[q], nus)
        for v, nu in enumerate(nus):
            eta = orc.default_step(n, 2, nu, sd2[v], 1.0)
            for r in range(R):
                y0 = Y0s[q][r * n:(r + 1) * n].astype(np.float64)
                y1, h = orc.fit(D[v], nu, sd2[v], y0, eta, 1)
                assert out["history"][0, q, v, r].item() == pytest.approx(h[0], rel=1e-5)
                a, b = sl[q, v, r]
                step = Yb[a:b].reshape(n, 2) - y0
                step_ref = y1 - y0
                assert np.max(np.abs(step - step_ref)) <= (1e-5 * np.abs(step_ref).max()
                                                          + 2e-7 * np.abs(y0).max()), (q, v, r)


def test_batched_ten_steps_against_the_oracle(G):
    """Ten iterations of the benchmark's batch shape (64 UCI-sized problems x 8
    nu x 8 restarts) for the three smallest problems and the smallest
    integer-valued one: the stress history of every fit against the oracle's
    fixed-step iterations, and Y_10.  The residual r = d - delta is formed in
    FP32, so once a small problem's stress has dropped by orders of magnitude
    its last digits go (an error of about 1e-7 of delta in r); the history is
    therefore bounded against S(Y_0), the scale of those errors, and Y_10
    against the distance the points moved."""
    w = wl.WORKLOADS["uci-batch-64"]
    Xs = wl.uci_like_batch(w["n_problems"], w["seed"])
    R, nus, T = w["restarts"], [float(v) for v in w["nu"]], 10
    ns = [X.shape[0] for X in Xs]
    Y0s = [wl.y_init(R * n, 2, seed=w["seed"] + 1000 + q) for q, n in enumerate(ns)]
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, T, Y0, eta0=1.0, history=True)
    Yb = out["Y"].cpu().numpy()
    hist = out["history"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    order = np.argsort(ns)
    ints = [q for q in order if q % 4 == 3]
    picks = sorted({int(q) for q in order[:3]} | {int(ints[0])})
    worst_h, worst_y = 0.0, 0.0
    for q in picks:
        n = ns[q]
        D, sd2 = orc.delta(Xs[q], nus)
        for v, nu in enumerate(nus):
            eta = orc.default_step(n, 2, nu, sd2[v], 1.0)
            for r in range(R):
                y0 = Y0s[q][r * n:(r + 1) * n].astype(np.float64)
                yT, h = orc.fit(D[v], nu, sd2[v], y0, eta, T)
                worst_h = max(worst_h, np.max(np.abs(hist[:, q, v, r] - h)) / h[0])
                a, b = sl[q, v, r]
                moved = np.abs(yT - y0).max()
                worst_y = max(worst_y, np.abs(Yb[a:b].reshape(n, 2) - yT).max() / moved)
    print(f"10 batched steps: history max err / S(Y_0) {worst_h:.3e}, "
          f"Y_10 max err / total move {worst_y:.3e}")
    assert worst_h <= 1e-5
    assert worst_y <= 1e-4


@pytest.mark.parametrize("tile", [None, (8, 2)])
def test_batched_bf16_pool_one_step_against_the_oracle(G, tile):
    """The Delta pool in BF16 (half the memory): S(Y0) and the first step of
    every fit against the oracle run on the same dissimilarities rounded to
    bf16 on the host; also with the tile shape given instead of autotuned."""
    ns, ps, nus, R = [150, 300, 77], [5, 12, 30], [1.5, 2.0, 3.0], 3
    Xs = [wl.gaussian_outliers(n, p, seed=7300 + q) for q, (n, p) in enumerate(zip(ns, ps))]
    Y0s = [wl.y_init(R * n, 2, seed=7310 + q) for q, n in enumerate(ns)]
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, 1, Y0, eta0=1.0, history=True, delta_dtype="bf16",
                             tile=tile)
    if tile:
        assert out["tuned"] == tile[0] * 100 + tile[1]
    Yb = out["Y"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    for q, n in enumerate(ns):
        D, sd2 = orc.delta(Xs[q], nus)
        for v, nu in enumerate(nus):
            Dq = quantize(D[v], "bf16")  # the stored values; the step keeps the FP32 sum
            eta = orc.default_step(n, 2, nu, sd2[v], 1.0)
            for r in range(R):
                y0 = Y0s[q][r * n:(r + 1) * n].astype(np.float64)
                y1, h = orc.fit(Dq, nu, sd2[v], y0, eta, 1)
                assert out["history"][0, q, v, r].item() == pytest.approx(h[0], rel=1e-5)
                a, b = sl[q, v, r]
                step = Yb[a:b].reshape(n, 2) - y0
                assert np.max(np.abs(step - (y1 - y0))) <= (1e-5 * np.abs(y1 - y0).max()
                                                           + 2e-7 * np.abs(y0).max()), (q, v, r)


@pytest.mark.parametrize("tile", [None, (8, 2)])
def test_batched_tiny_problems_against_the_oracle(G, tile):
    """Problems of 2, 3, 5 and 129 points (one tile, mostly padding, and a
    ragged second tile) with 2 to 7 features: three steps of every fit against
    the oracle's fixed-step iterations; then a one-feature problem, whose
    pseudo-distances are all zero (W_{1,nu} = 0), is refused as degenerate."""
    from paper_2605_25124_gb300._lib import GiniError
    ns, ps, nus, R, T = [2, 3, 5, 129], [2, 3, 2, 7], [1.5, 2.0], 2, 3
    Xs, Y0s = _batch(800, ns, ps, R)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    out = G.gini_fit_batched(Xd, nus, R, T, Y0, eta0=1.0, history=True, tile=tile)
    hist = out["history"].cpu().numpy()
    Yb = out["Y"].cpu().numpy()
    sl = _slices(ns, len(nus), R)
    for q, n in enumerate(ns):
        D, sd2 = orc.delta(Xs[q], nus)
        for v, nu in enumerate(nus):
            eta = orc.default_step(n, 2, nu, sd2[v], 1.0)
            for r in range(R):
                y0 = Y0s[q][r * n:(r + 1) * n].astype(np.float64)
                yT, h = orc.fit(D[v], nu, sd2[v], y0, eta, T)
                assert np.max(np.abs(hist[:, q, v, r] - h)) <= 1e-5 * h[0] + 1e-12, (q, v, r)
                a, b = sl[q, v, r]
                moved = max(np.abs(yT - y0).max(), 1e-30)
                assert np.abs(Yb[a:b].reshape(n, 2) - yT).max() <= 1e-4 * moved + 1e-6, (q, v, r)
    X1 = [torch.from_numpy(wl.gaussian_outliers(40, 1, seed=801)).cuda()]
    Y1 = torch.from_numpy(wl.y_init(R * 40, 2, seed=802).reshape(-1)).cuda()
    with pytest.raises(GiniError, match="EDEGENERATE"):
        G.gini_fit_batched(X1, nus, R, T, Y1)
