"""Runs the hot paths on the debug library (device-side index checks) and
compares them with the FP64 oracle; prints one JSON line and exits 1 on any
failure.  tests/test_gpu_debug_checks.py starts it in a child process with
GINI_DEBUG=1 (the binding loads one library per process).

Cases: the index check's self-test (a planted store past its checked bound);
the Delta build in every kernel family (positional-weight, cell-key, 64-bit
exact through wide-range data, long vectors; FULL, tiled FP32 / BF16 hi+lo /
FP8 strips); the ranks (short and chunked segments); the stress and gradient
in every iteration kernel (k = 2 fused, generic k, plain form; atomics and the
deterministic partials); a fit; a batched fit with FP32 and BF16 pools.  Every
call's gini_check must return GINI_OK: a failed index check would return
GINI_EINDEX.
"""
import json
import os
import sys
import traceback

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import ctypes  # noqa: E402

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import gini_oracle as orc  # noqa: E402
import paper_2605_25124_gb300 as G  # noqa: E402
from paper_2605_25124_gb300 import _lib  # noqa: E402
from paper_2605_25124_gb300 import workloads as wl  # noqa: E402
from util import host_col_scale, quantize, rel_err, tile_pack, untile  # noqa: E402

RESULTS = {}


def case(fn):
    try:
        fn()
        RESULTS[fn.__name__] = "ok"
    except Exception:  # noqa: BLE001 -- reported, then the run fails
        RESULTS[fn.__name__] = traceback.format_exc(limit=3)
    return fn


def _close(got, ref, tol=1e-5):
    floor = 1e-6 * np.abs(ref).max()
    e = rel_err(got, ref, floor)
    assert e <= tol, e


def selftest_index_check():
    L = _lib.lib()
    assert L.gini_debug_checks() == 1, "not the debug library"
    ws = G.workspace()
    buf = ws.ensure(512)
    ptr = buf.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.gini_selftest_index_check(ptr, buf.numel(), stream) == _lib.GINI_OK
    assert L.gini_check(ptr, stream) == _lib.GINI_EINDEX
    site, cnt = ctypes.c_uint32(), ctypes.c_uint32()
    idx, bound = ctypes.c_int64(), ctypes.c_int64()
    assert L.gini_debug_index_record(ptr, ctypes.byref(site), ctypes.byref(idx),
                                     ctypes.byref(bound), ctypes.byref(cnt)) == _lib.GINI_OK
    assert site.value // 100000 == 6 and site.value % 100000 > 0, site.value  # selftest.cu
    assert bound.value == 32 and idx.value in range(32, 61, 4) and cnt.value == 8
    # the stores that passed landed, the others were skipped
    vals = buf[256:512].view(torch.float32).cpu().numpy()
    want = np.zeros(64, np.float32)
    want[8:32:4] = np.arange(8, 32, 4)
    np.testing.assert_array_equal(vals, want)
    # the word and the record are clear again
    assert L.gini_check(ptr, stream) == _lib.GINI_OK
    assert L.gini_debug_index_record(ptr, ctypes.byref(site), ctypes.byref(idx),
                                     ctypes.byref(bound), ctypes.byref(cnt)) == _lib.GINI_OK
    assert site.value == 0 and cnt.value == 0


def delta_full_every_family():
    # 784: 25 registers per lane; 600, 700, 850: 20, 24, 28 (the other 32-lane shapes)
    for n, p, nus in ((41, 784, [2.0]), (41, 784, [1.5, 2.5]), (33, 50, [1.5, 2.0, 3.0]),
                      (29, 7, [3.0]), (23, 600, [2.0]), (23, 700, [1.5]),
                      (23, 850, [2.0, 3.5])):
        X = wl.gaussian_outliers(n, p, seed=900 + p + len(nus))
        ref, sref = orc.delta(X, nus)
        mats, sd2 = G.gini_dist(torch.from_numpy(X).cuda(), nus, layout="full")
        for q in range(len(nus)):
            _close(mats[q].data.double().cpu().numpy(), ref[q])
            assert abs(float(sd2[q]) - sref[q]) <= 1e-5 * sref[q]
    # a range of 1e4 with nonzero values near 1e-38: the cell keys' pre-pass
    # sends the build to the 64-bit network
    rng = np.random.default_rng(905)
    X = (rng.standard_normal((30, 40)) * 3000).astype(np.float32)
    X[rng.integers(0, 30, 8), rng.integers(0, 40, 8)] = np.float32(3e-38)
    ref, _ = orc.delta(X, [1.5])
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [1.5], layout="full")
    _close(mats[0].data.double().cpu().numpy(), ref[0])


def delta_tiled_fp8_and_long():
    n = 300  # three tiles per edge, ragged tail
    X = wl.gaussian_outliers(n, 30, seed=910)
    ref, _ = orc.delta(X, [2.0, 1.5, 3.0])
    Xd = torch.from_numpy(X).cuda()
    m32, _ = G.gini_dist(Xd, [2.0], layout="tiled", dtype="f32")
    _close(untile(m32[0].data.cpu().numpy(), n)[:n, :n], np.triu(ref[0], 1))
    mx2, _ = G.gini_dist(Xd, [1.5, 3.0], layout="tiled", dtype="bf16x2")
    for q in range(2):
        flat = mx2[q].data.view(torch.int16).cpu().numpy().astype(np.uint16).astype(np.uint32)
        vals = (flat << 16).view(np.float32)
        got = untile(vals, n, planes=2)[:n, :n]
        _close(got, np.triu(ref[q + 1], 1), tol=2.0 ** -15)
    m8, _ = G.gini_dist(Xd, [2.0], layout="tiled", dtype="fp8")
    P8 = G.gini_pack(G.gini_dist(Xd, [2.0], layout="full")[0][0], "fp8")
    assert torch.equal(m8[0].data, P8.data) and torch.equal(m8[0].col_scale, P8.col_scale)
    # vectors longer than one warp's registers: chunked sort + search
    Xl = wl.gaussian_outliers(24, 2048, seed=911)
    refl, _ = orc.delta(Xl, [1.5, 2.0])
    ml, _ = G.gini_dist(torch.from_numpy(Xl).cuda(), [1.5, 2.0], layout="full")
    for q in range(2):
        _close(ml[q].data.double().cpu().numpy(), refl[q])


def ranks_short_and_long():
    rng = np.random.default_rng(920)
    for m, nseg in ((100, 50), (1000, 9), (3000, 3)):
        v = (rng.integers(-3, 4, (nseg, m)) * 0.5).astype(np.float32)  # heavy ties
        got = G.gini_rank(torch.from_numpy(v).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, np.stack([orc.midrank2(r) for r in v]))


def stress_every_iteration_kernel():
    n = 300
    for k, nu, dtype, det in ((2, 2.0, "f32", False), (2, 1.5, "bf16x2", False),
                              (2, 2.0, "fp8", False), (2, 2.0, "f32", True),
                              (3, 3.0, "f32", False), (3, 3.0, "f32", True),
                              (4, 1.3, "bf16", False), (2, 1.7, "full", False),
                              (3, 1.7, "full", False)):
        X = wl.gaussian_outliers(n, 8, seed=930 + k)
        D, s = orc.delta(X, [nu])
        D, sd2 = D[0], float(s[0])
        sc = host_col_scale(D) if dtype == "fp8" else None
        Dq = quantize(D, "f32" if dtype == "full" else dtype, sc)
        Dq = np.triu(Dq, 1) + np.triu(Dq, 1).T
        Y = wl.y_init(n, k, seed=931 + k, sd=1.0)
        Sref, gref = orc.stress_grad(Y.astype(np.float64), nu, Dq, sd2)
        if dtype == "full":
            Dd = G.Dissimilarity(torch.from_numpy(D.astype(np.float32)).cuda(), n, "full", "f32", sd2)
        else:
            Dd = G.Dissimilarity(torch.from_numpy(tile_pack(D, n, dtype, sc)).cuda(), n, "tiled",
                                 dtype, sd2, torch.from_numpy(sc).cuda() if sc is not None else None)
        with G.deterministic(det):
            S, g = G.gini_stress_grad(torch.from_numpy(Y).cuda(), nu, Dd)
        assert abs(float(S) - Sref) <= 1e-5 * Sref, (k, dtype, det)
        assert np.max(np.abs(g.cpu().numpy() - gref)) <= 1e-5 * np.abs(gref).max(), (k, dtype, det)


def fit_and_batched():
    n, nu, T = 300, 2.0, 20
    X = wl.gaussian_outliers(n, 10, seed=940)
    D, s = orc.delta(X, [nu])
    sd2 = float(s[0])
    mats, _ = G.gini_dist(torch.from_numpy(X).cuda(), [nu], layout="tiled", dtype="f32")
    Y0 = wl.y_init(n, 2, seed=941)
    eta = G.default_step(n, 2, nu, sd2, 1.0)
    _, href = orc.fit(D[0], nu, sd2, Y0.astype(np.float64), eta, T)
    for det in (False, True):
        _, hist, _ = G.gini_mds_fit(torch.from_numpy(Y0).cuda(), nu, mats[0], eta, T,
                                    deterministic=det)
        h = hist.cpu().numpy()
        assert np.max(np.abs(h - href) / href) <= 1e-4, det
    ns, ps, nus, R, T = [150, 260, 77], [5, 12, 9], [1.5, 2.0], 2, 3
    Xs = [wl.gaussian_outliers(a, b, seed=950 + q) for q, (a, b) in enumerate(zip(ns, ps))]
    Y0s = [wl.y_init(R * a, 2, seed=960 + q) for q, a in enumerate(ns)]
    Y0 = torch.from_numpy(np.concatenate([y.reshape(-1) for y in Y0s])).cuda()
    Xd = [torch.from_numpy(a).cuda() for a in Xs]
    for dt, det in (("f32", False), ("bf16", False), ("f32", True)):
        out = G.gini_fit_batched(Xd, nus, R, T, Y0, eta0=1.0, history=True, delta_dtype=dt,
                                 deterministic=det)
        hist = out["history"].cpu().numpy()
        for q, a in enumerate(ns):
            Dr, sd = orc.delta(Xs[q], nus)
            for v, nuv in enumerate(nus):
                Dv = quantize(Dr[v], "bf16") if dt == "bf16" else Dr[v]
                eta_v = orc.default_step(a, 2, nuv, sd[v], 1.0)
                for r in range(R):
                    y0 = Y0s[q][r * a:(r + 1) * a].astype(np.float64)
                    _, h = orc.fit(Dv, nuv, sd[v], y0, eta_v, T)
                    assert np.max(np.abs(hist[:, q, v, r] - h)) <= 1e-5 * h[0], (dt, det, q, v, r)


def main():
    torch.cuda.set_device(0)
    for fn in (selftest_index_check, delta_full_every_family, delta_tiled_fp8_and_long,
               ranks_short_and_long, stress_every_iteration_kernel, fit_and_batched):
        case(fn)
    ok = all(v == "ok" for v in RESULTS.values())
    print(json.dumps({"debug_library": _lib.LIB_PATH, "ok": ok, "cases": RESULTS}))
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
