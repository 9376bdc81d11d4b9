"""gini_stress_grad (plain FULL form and fused TILED form) and the GiniStress
autograd op on the GPU against the FP64 oracle.

Tolerances: stress relative 1e-5; gradient max-abs error <= 1e-5 x max |grad|
(an FP32 sum of n terms with cancellation is only accurate relative to the
scale of its terms); finite differences relative 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl
from util import host_col_scale, quantize, tile_pack

pytestmark = pytest.mark.gpu


def _dis(G, full_ref, n, dtype, sd2):
    """Upload a host matrix as the library's Dissimilarity in layout/dtype."""
    if dtype == "full":
        t = torch.from_numpy(np.asarray(full_ref, dtype=np.float32)).cuda()
        return G.Dissimilarity(t, n, "full", "f32", sd2)
    sc = host_col_scale(full_ref) if dtype == "fp8" else None
    flat = tile_pack(full_ref, n, dtype, sc)
    t = torch.from_numpy(flat).cuda()
    return G.Dissimilarity(t, n, "tiled", dtype, sd2,
                           torch.from_numpy(sc).cuda() if sc is not None else None)


def _ref_delta(n, p, nu, seed):
    X = wl.gaussian_outliers(n, p, seed=seed)
    D, s = orc.delta(X, [nu])
    return X, D[0], float(s[0])


@pytest.mark.parametrize("dtype", ["full", "f32", "bf16", "bf16x2", "fp8"])
@pytest.mark.parametrize("k,nu", [(2, 2.0), (2, 1.5), (3, 3.0), (3, 1.6), (4, 1.3), (8, 2.0)])
def test_stress_grad_parity(G, dtype, k, nu):
    n = 300  # 3 tiles per edge, ragged tail
    X, D, sd2 = _ref_delta(n, 8, nu, seed=200 + k)
    sc = host_col_scale(D) if dtype == "fp8" else None
    Dq = quantize(D, "f32" if dtype == "full" else dtype, sc)
    Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
    Y = wl.y_init(n, k, seed=201 + k, sd=1.0)
    Sref, gref = orc.stress_grad(Y.astype(np.float64), nu, Dq, sd2)
    S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, _dis(G, D, n, dtype, sd2))
    assert float(S) == pytest.approx(Sref, rel=1e-5)
    assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max()
    S2, g2 = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, _dis(G, D, n, dtype, sd2),
                                grad=False)
    assert g2 is None and float(S2) == pytest.approx(Sref, rel=1e-5)


@pytest.mark.parametrize("k,nu", [(2, 2.0), (3, 1.6)])
def test_planted_embedding_zero_stress(G, k, nu):
    n = 200
    Ys = wl.y_init(n, k, seed=210, sd=1.0)
    I, J = np.triu_indices(n, 1)
    d = orc.embed_dist_pairs(Ys.astype(np.float64), nu, I, J)
    D = np.zeros((n, n)); D[I, J] = d; D[J, I] = d
    sd2 = float(np.sum(d ** 2))
    for dtype in ("full", "f32"):
        S, g = G.gini_stress_grad(torch.from_numpy(Ys).cuda(), nu, _dis(G, D, n, dtype, sd2))
        Yp = Ys + 0.05 * wl.y_init(n, k, seed=211, sd=1.0)
        Sp, gp = G.gini_stress_grad(torch.from_numpy(Yp).cuda(), nu, _dis(G, D, n, dtype, sd2))
        assert float(S) < 1e-11 and float(Sp) > 1e-5
        assert g.abs().max().item() < 1e-4 * gp.abs().max().item()


@pytest.mark.parametrize("k", [2, 3])
def test_gradient_against_central_differences(G, k):
    # Differences of the stress are taken through the plain form, whose forward
    # pass rounds each r^2 once and sums in FP64, so unchanged pairs cancel
    # exactly; the fused gradient must match the plain one.
    n, nu = 64, 1.8
    X, D, sd2 = _ref_delta(n, 6, nu, seed=220 + k)
    Dd = _dis(G, D, n, "full", sd2)
    Y = wl.y_init(n, k, seed=221, sd=1.0)
    _, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dd)
    _, gt = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, _dis(G, D, n, "f32", sd2))
    assert (g - gt).abs().max().item() <= 1e-5 * g.abs().max().item()
    g = g.cpu().numpy()
    rng = np.random.default_rng(222)
    pairs = [(a, b) for a in range(k) for b in range(a + 1, k)]
    for _ in range(24):
        i, c = int(rng.integers(n)), int(rng.integers(k))
        # distance to the nearest kink along y_ic: a tie of z_a and z_b for a
        # pair (a, b) containing c moves when y_ic moves
        gap = np.inf
        for (a, b) in pairs:
            if c in (a, b):
                v = (Y[:, a].astype(np.float64) - Y[:, b])
                dv = np.abs(v[i] - np.delete(v, i))
                gap = min(gap, dv.min())
        h = float(min(1e-3, 0.3 * gap))
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, c] += np.float32(h)
        Ym[i, c] -= np.float32(h)
        hp, hm = float(Yp[i, c]) - float(Y[i, c]), float(Y[i, c]) - float(Ym[i, c])
        Sp, _ = G.gini_stress_grad(torch.from_numpy(Yp).cuda(), nu, Dd, grad=False)
        Sm, _ = G.gini_stress_grad(torch.from_numpy(Ym).cuda(), nu, Dd, grad=False)
        fd = (float(Sp) - float(Sm)) / (hp + hm)
        assert g[i, c] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(g).max())


@pytest.mark.parametrize("k,dtype", [(2, "full"), (2, "f32"), (2, "bf16"), (2, "bf16x2"),
                                     (3, "full"), (3, "f32")])
def test_adjoint_at_mixture_scale_sampled_rows(G, k, dtype):
    """n = 5000, p = 50 Gaussian mixture with heavy-tailed rows (many tiles per
    CTA): GPU gradient rows against oracle rows computed from the oracle's
    Delta rounded on the host to the same storage type."""
    n, p, nu = 5000, 50, 2.0
    X = wl.gaussian_mixture(n, p, seed=wl.SEED_BASE + 3)
    Y = wl.y_init(n, k, seed=230 + k, sd=1.0)
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="full")
    Dg = G.Dissimilarity(mats[0].data, n, "full", "f32", 1.0)  # sum_delta2 = 1 on both sides
    Dd = Dg if dtype == "full" else G.gini_pack(Dg, dtype)
    _, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dd)
    rows = np.random.default_rng(231).choice(n, 12, replace=False)
    I = np.repeat(rows, n)
    J = np.tile(np.arange(n), len(rows))
    Drows = orc.delta_pairs(X, [nu], I, J)[:, 0].reshape(len(rows), n)
    if dtype in ("bf16", "bf16x2"):
        Drows = quantize(Drows, dtype)
    gref = orc.grad_rows(Y.astype(np.float64), nu, Drows, rows, 1.0)
    scale = np.abs(gref).max()
    err = np.max(np.abs(g.cpu().numpy()[rows] - gref))
    assert err <= 1e-5 * scale, (dtype, err / scale)


def test_autograd_function(G):
    n, k, nu = 150, 2, 2.0
    X, D, sd2 = _ref_delta(n, 5, nu, seed=240)
    Y = wl.y_init(n, k, seed=241, sd=1.0)
    Dd = _dis(G, D, n, "bf16x2", sd2)
    Yt = torch.from_numpy(Y).cuda().requires_grad_(True)
    S = G.gini_stress(Yt, nu, Dd)
    (3.0 * S).backward()
    Sref, gref = orc.stress_grad(Y.astype(np.float64), nu,
                                 np.triu(quantize(D, "bf16x2"), 1) + np.triu(quantize(D, "bf16x2"), 1).T,
                                 sd2)
    assert float(S) == pytest.approx(Sref, rel=1e-5)
    assert np.max(np.abs(Yt.grad.cpu().numpy() - 3.0 * gref)) <= 1e-5 * 3.0 * np.abs(gref).max()
    with torch.no_grad():
        S0 = G.gini_stress(torch.from_numpy(Y).cuda(), nu, Dd)
    assert float(S0) == pytest.approx(Sref, rel=1e-5)


def test_nonfinite_embedding_reported(G):
    from paper_2605_25124_gb300._lib import GiniError
    n = 40
    _, D, sd2 = _ref_delta(n, 4, 2.0, seed=250)
    Y = wl.y_init(n, 2, seed=251)
    Y[5, 1] = np.nan
    with pytest.raises(GiniError, match="ENONFINITE"):
        G.gini_stress_grad(torch.from_numpy(Y).cuda(), 2.0, _dis(G, D, n, "f32", sd2))


def test_bounded_wait_expires_and_context_survives(G):
    # the pipelined kernels' bounded wait, on a barrier nothing completes: it
    # must give up after its limit, report ETIMEOUT through gini_check, and
    # leave the GPU usable for the next call
    import time
    from paper_2605_25124_gb300 import _lib
    L = _lib.lib()
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert L.gini_selftest_wait_timeout(20_000_000, ws.data_ptr(), ws.numel(), None) == 0
    st = L.gini_check(ws.data_ptr(), None)
    dt = time.perf_counter() - t0
    assert st == _lib.GINI_ETIMEOUT
    assert 0.015 <= dt < 5.0
    assert L.gini_check(ws.data_ptr(), None) == 0  # the check cleared it
    assert L.gini_selftest_wait_timeout(10, ws.data_ptr(), ws.numel(), None) == _lib.GINI_EINVAL
    n = 60
    _, D, sd2 = _ref_delta(n, 5, 2.0, seed=260)
    Y = wl.y_init(n, 2, seed=261)
    S, _ = G.gini_stress_grad(torch.from_numpy(Y).cuda(), 2.0, _dis(G, D, n, "f32", sd2))
    Dq = quantize(D, "f32")
    Sref, _ = orc.stress_grad(Y.astype(np.float64), 2.0, np.triu(Dq, 1) + np.triu(Dq, 1).T, sd2)
    assert float(S) == pytest.approx(Sref, rel=1e-5)


def _tiny_lo_points(k):
    """Points whose pair differences u = y_a - y_b share their FP32 part and
    differ only below it (lo parts 2^-30, 2^-140 and subnormal 2^-149 apart),
    plus exact duplicates: the rank comparisons are decided by lo, or tie."""
    n = 64
    Y = np.zeros((n, k), np.float64)
    for g, (c, eps) in enumerate(((1.0, 2.0 ** -30), (2.0 ** -100, 2.0 ** -140),
                                  (2.0 ** -120, 2.0 ** -149))):
        for m in range(16):
            row = [c, m * eps] if k == 2 else [c, m * eps, (15 - m + 3 * g) * eps]
            Y[16 * g + m] = row
    Y[48:] = Y[:16]
    assert np.array_equal(Y.astype(np.float32).astype(np.float64), Y)  # exact in FP32
    return Y.astype(np.float32)


@pytest.mark.parametrize("k,nu", [(2, 1.7), (3, 1.7), (3, 2.0)])  # 2.0: k = 3's affine body
def test_exact_sign_decided_by_tiny_lo_parts(G, k, nu):
    # The fused and plain kernels order u_i - u_j through TwoSum pairs whose lo
    # parts carry the sign when the FP32 parts are equal.  Here 3/4 of the
    # within-group pairs differ only in lo (down to the subnormal step) and a
    # quarter of the points are exact duplicates (sign 0): a wrong or missing
    # sign moves h_i by about one delta, about 1/n of the largest gradient.
    n = 64
    X, D, sd2 = _ref_delta(n, 6, nu, seed=270 + k)
    Y = _tiny_lo_points(k)
    Dq = quantize(D, "f32")
    Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
    Sref, gref = orc.stress_grad(Y.astype(np.float64), nu, Dq, sd2)
    for form in ("f32", "full"):
        S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, _dis(G, D, n, form, sd2))
        assert float(S) == pytest.approx(Sref, rel=1e-5), form
        assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max(), form
    if k == 2:  # the batched kernel's own copy of the pair arithmetic: one step
        eta = orc.default_step(n, 2, nu, sd2, 1.0)
        y1, h = orc.fit(D, nu, sd2, Y.astype(np.float64), eta, 1)
        out = G.gini_fit_batched([torch.from_numpy(X).cuda()], [nu], 1, 1,
                                 torch.from_numpy(Y.reshape(-1)).cuda(), eta0=1.0, history=True)
        assert out["history"][0, 0, 0, 0].item() == pytest.approx(h[0], rel=1e-5)
        step = out["Y"].cpu().numpy().reshape(n, 2).astype(np.float64) - Y
        assert np.max(np.abs(step - (y1 - Y))) <= 1e-5 * np.abs(y1 - Y).max() + 2e-7 * np.abs(Y).max()
