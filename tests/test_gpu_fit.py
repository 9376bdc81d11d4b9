"""gini_mds_fit on the GPU against the oracle's fixed-step gradient descent.

One GD step from a common Y_t must match to 1e-5 (relative to the step).
Over many steps FP32 and FP64 iterates drift apart slowly (a pair whose
embedding gap is within rounding of zero can take the other side of a kink),
so whole trajectories are compared with a looser, stated bound.
"""
import numpy as np
import pytest
import torch

from oracle import gini_oracle as orc
from paper_2605_25124_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NAME = "gauss-outliers-n200-p10"


def _problem(G, nu=2.0):
    w = wl.WORKLOADS[NAME]
    X = wl.make_X(NAME)
    Dref, sref = orc.delta(X, [nu])
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="full")
    Y0 = wl.y_init(w["n"], w["k"], seed=w["seed"] + 1000)
    return w, X, Dref[0], float(sref[0]), mats[0], Y0


@pytest.mark.parametrize("form", ["full", "f32", "bf16x2"])
def test_fit_trajectory_gauss_outliers(G, form):
    w, X, Dref, sref, Dfull, Y0 = _problem(G)
    n, k, nu, T = w["n"], w["k"], 2.0, w["iters"]
    eta = G.default_step(n, k, nu, sref, 1.0)
    Yr, href = orc.fit(Dref, nu, sref, Y0.astype(np.float64), eta, T)
    D = Dfull if form == "full" else G.gini_pack(Dfull, form)
    Y, hist, final = G.gini_mds_fit(torch.from_numpy(Y0).cuda(), nu, D, eta, T, polish_iters=T)
    h = hist.cpu().numpy()
    rel = np.abs(h - href) / href
    print(f"{form}: max rel history error {rel.max():.3e}, "
          f"max |Y - Y_ref| / max|Y_ref| {np.abs(Y.cpu().numpy() - Yr).max() / np.abs(Yr).max():.3e}")
    assert rel[:10].max() <= 1e-5
    assert rel.max() <= 1e-3
    assert float(final) == pytest.approx(h[-1], rel=0, abs=0)
    assert h[-1] < h[0]


@pytest.mark.parametrize("form,k", [("full", 2), ("f32", 2), ("full", 3), ("f32", 3)])
def test_fit_one_step_from_common_iterate(G, form, k):
    w, X, Dref, sref, Dfull, _ = _problem(G, nu=1.7)
    n, nu = w["n"], 1.7
    Y0 = wl.y_init(n, k, seed=300 + k)
    eta = G.default_step(n, k, nu, sref, 1.0)
    Ymid, _ = orc.fit(Dref, nu, sref, Y0.astype(np.float64), eta, 20)
    Yt = Ymid.astype(np.float32)
    Y1r, h1 = orc.fit(Dref, nu, sref, Yt.astype(np.float64), eta, 1)
    D = Dfull if form == "full" else G.gini_pack(Dfull, form)
    Y1, hist, _ = G.gini_mds_fit(torch.from_numpy(Yt).cuda(), nu, D, eta, 1)
    step_ref = Y1r - Yt
    step = Y1.cpu().numpy().astype(np.float64) - Yt
    assert np.max(np.abs(step - step_ref)) <= 1e-5 * np.abs(step_ref).max() + 2e-7 * np.abs(Yt).max()
    assert hist.cpu().numpy()[0] == pytest.approx(h1[0], rel=1e-5)


def test_split_bf16_reaches_fp32_final_stress(G):
    # BF16 hi + lo storage (split-precision correction) in every iteration
    # lands on the same stationary point as FP32.  A hi-only phase may not:
    # the k = 2 stress is piecewise quadratic with many kinks, and an early
    # BF16 gradient (relative error up to 2^-8 per entry) can steer the
    # descent into a neighbouring local minimum that later hi + lo
    # iterations do not leave (here about 0.4% higher); that schedule is
    # only reported.
    w, X, Dref, sref, Dfull, Y0 = _problem(G)
    n, k, nu, T = w["n"], w["k"], 2.0, 200
    eta = G.default_step(n, k, nu, Dfull.sum_delta2, 1.0)
    Yd = torch.from_numpy(Y0).cuda()
    _, hf, f32 = G.gini_mds_fit(Yd, nu, G.gini_pack(Dfull, "f32"), eta, T)
    Dhl = G.gini_pack(Dfull, "bf16x2")
    _, _, hl = G.gini_mds_fit(Yd, nu, Dhl, eta, T, polish_iters=T)
    assert abs(float(hl) - float(f32)) <= 1e-4 * float(f32)
    _, hs, sched = G.gini_mds_fit(Yd, nu, Dhl, eta, T, polish_iters=40)
    h = hs.cpu().numpy()
    print(f"hi-only 160 + hi+lo 40: final stress {float(sched):.6g} vs FP32 {float(f32):.6g} "
          f"(rel {abs(float(sched) - float(f32)) / float(f32):.2e})")
    assert np.all(np.diff(h) <= 1e-7 * h[0]) and h[-1] < 0.1 * h[0]  # FP32 wobble at rest


def test_fit_resume_and_zero_iterations(G):
    w, X, Dref, sref, Dfull, Y0 = _problem(G)
    n, k, nu = w["n"], w["k"], 2.0
    eta = G.default_step(n, k, nu, Dfull.sum_delta2, 1.0)
    Yd = torch.from_numpy(Y0).cuda()
    D = G.gini_pack(Dfull, "f32")
    Ya, ha, _ = G.gini_mds_fit(Yd, nu, D, eta, 30)
    Yb, _, _ = G.gini_mds_fit(Yd, nu, D, eta, 15)
    Yc, hc, _ = G.gini_mds_fit(Yb, nu, D, eta, 15)
    assert (Ya - Yc).abs().max().item() <= 1e-5 * Ya.abs().max().item()
    Y0r, h0, f0 = G.gini_mds_fit(Yd, nu, D, eta, 0)
    assert torch.equal(Y0r, Yd)
    S, _ = G.gini_stress_grad(Yd, nu, D, grad=False)
    assert h0.cpu().numpy()[0] == pytest.approx(float(S), rel=1e-12)
    assert float(f0) == pytest.approx(float(S), rel=1e-12)
