"""gini_stress_grad_noalloc: the stress/gradient entry point for callers that
may not allocate device memory (plugins whose host application owns every byte
of device memory, real-time loops that cannot afford the synchronisation of
cudaMalloc and cudaFree), whose scratch space is a fixed array inside the
library.

It is checked through the C ABI against gini_stress_grad with a caller
workspace, on two calls in a row with different problems, at the tolerances
of the other stress tests (stress 1e-5 relative, gradient 1e-5 of its max).
Named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_25124_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _both(G, Y, nu, D):
    from paper_2605_25124_gb300._lib import LAYOUTS, DTYPES, lib
    L = lib()
    n, k = Y.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (_p(Y), n, k, float(nu), _p(D.data), LAYOUTS[D.layout], DTYPES[D.dtype], D.ldd,
            _p(D.col_scale), D.sum_delta2)
    ws = torch.zeros(G.workspace_size("stress", n, 0, k), dtype=torch.uint8, device="cuda")
    s_ref = torch.empty((), dtype=torch.float64, device="cuda")
    g_ref = torch.empty_like(Y)
    assert L.gini_stress_grad(*args, _p(s_ref), _p(g_ref), _p(ws), ws.numel(), stream) == 0
    s_new = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    g_new = torch.full_like(Y, float("nan"))
    assert L.gini_stress_grad_noalloc(*args, _p(s_new), _p(g_new), stream) == 0
    torch.cuda.synchronize()
    return float(s_ref), g_ref.cpu().numpy(), float(s_new), g_new.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_two_calls(G):
    nu = 1.8
    # call 1: k = 2, tiled BF16 hi + lo (bulk-copy pipeline, many tiles)
    X = wl.gaussian_mixture(3000, 20, seed=401)
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="full")
    Dt = G.gini_pack(mats[0], "bf16x2")
    Y = torch.from_numpy(wl.y_init(3000, 2, seed=402, sd=1.0)).cuda()
    s_ref, g_ref, s_new, g_new = _both(G, Y, nu, Dt)
    assert s_new == pytest.approx(s_ref, rel=1e-5)
    assert np.max(np.abs(g_new - g_ref)) <= 1e-5 * np.abs(g_ref).max()
    # call 2: k = 3, full FP32 matrix of another problem (plain kernels); the
    # array still holds call 1's contents
    X2 = wl.gaussian_outliers(700, 9, seed=403)
    mats2, _ = G.gini_dist(torch.from_numpy(X2).cuda(), [nu], layout="full")
    Y2 = torch.from_numpy(wl.y_init(700, 3, seed=404, sd=1.0)).cuda()
    s_ref, g_ref, s_new, g_new = _both(G, Y2, nu, mats2[0])
    assert s_new == pytest.approx(s_ref, rel=1e-5)
    assert np.max(np.abs(g_new - g_ref)) <= 1e-5 * np.abs(g_ref).max()


def test_noalloc_rejects_sizes_beyond_its_array(G):
    from paper_2605_25124_gb300._lib import GINI_ENOMEM, lib
    L = lib()
    fake = ctypes.c_void_p(0x1000)  # never touched: the size check comes first
    assert L.gini_stress_grad_noalloc(fake, 2_000_000, 2, 2.0, fake, 1, 1, 0, None, 1.0,
                                      fake, fake, None) == GINI_ENOMEM


def test_noalloc_reports_a_device_error_then_recovers(G):
    # A NaN in Y is caught by the kernels (no fault) and reported as a NaN
    # stress; the next call on the same array starts from a cleared error word
    # and matches the workspace entry point.
    nu = 2.0
    X = wl.gaussian_outliers(400, 7, seed=405)
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="tiled", dtype="f32")
    Y = torch.from_numpy(wl.y_init(400, 2, seed=406, sd=1.0)).cuda()
    Ybad = Y.clone()
    Ybad[17, 1] = float("nan")
    s_ref, g_ref, s_bad, _ = _both(G, Ybad, nu, mats[0])
    assert np.isnan(s_bad)
    s_ref, g_ref, s_new, g_new = _both(G, Y, nu, mats[0])
    assert np.isfinite(s_new) and s_new == pytest.approx(s_ref, rel=1e-5)
    assert np.max(np.abs(g_new - g_ref)) <= 1e-5 * np.abs(g_ref).max()
