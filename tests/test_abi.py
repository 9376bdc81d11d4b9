"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol include/gini_mds.h declares, and rejects bad arguments on the host
before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gini_mds.h")


@pytest.fixture(scope="module")
def L():
    from paper_2605_25124_gb300 import build
    build.build()
    from paper_2605_25124_gb300 import _lib
    return _lib.lib()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gini_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("gini_rank", "gini_dist", "gini_stress_grad", "gini_mds_fit", "gini_pack",
                 "gini_workspace_size", "gini_check"):
        assert want in names


def test_library_exports_every_declared_symbol(L):
    from paper_2605_25124_gb300 import _lib
    for name in _declared():
        assert hasattr(L, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_constants(L):
    assert L.gini_version() == 2
    B = L.gini_tile_size()
    assert B == 128
    for n in (2, 127, 128, 129, 20000):
        T = -(-n // B)
        assert L.gini_tiled_elems(n) == T * (T + 1) // 2 * B * B
    assert L.gini_workspace_size(0, 10, 5, 0, 0) >= 256
    assert L.gini_workspace_size(3, 1000, 0, 2, 50) > L.gini_workspace_size(2, 1000, 0, 2, 0)
    assert L.gini_workspace_size(99, 1, 1, 1, 1) == 0
    # deterministic mode: per-tile gradient partials, 2 x 128 x k floats per tile
    for n, k in ((1000, 2), (300, 3)):
        T = -(-n // B)
        extra = L.gini_workspace_size(5, n, 0, k, 50) - L.gini_workspace_size(3, n, 0, k, 50)
        assert extra >= T * (T + 1) // 2 * 2 * B * k * 4
        assert L.gini_workspace_size(4, n, 0, k, 0) > L.gini_workspace_size(2, n, 0, k, 0)
    assert b"EINVAL" in L.gini_status_str(1)


def test_default_step(L):
    # eta0 * S / (2 (n-1) k ((k/2) ((k-1)/k)^(nu-1))^2)
    n, k, nu, s = 200, 2, 2.0, 1000.0
    want = s / (2 * (n - 1) * k * (0.5 * k * 0.5 ** (nu - 1)) ** 2)
    assert L.gini_default_step(n, k, nu, s, 1.0) == pytest.approx(want, rel=1e-15)
    assert L.gini_default_step(1, 2, 2.0, 1.0, 1.0) == 0.0


def test_host_side_validation(L):
    from paper_2605_25124_gb300 import _lib
    fake = ctypes.c_void_p(0x1000)      # never dereferenced: validation fails first
    ws = ctypes.c_void_p(0x2000)
    nu = (ctypes.c_double * 1)(2.0)
    bad_nu = (ctypes.c_double * 1)(1.0)
    EINVAL, EDEG, ENOMEM = _lib.GINI_EINVAL, _lib.GINI_EDEGENERATE, _lib.GINI_ENOMEM
    # gini_rank: m out of range, ld < m, missing pointers
    assert L.gini_rank(fake, 4, 0, 4, fake, ws, 1 << 20, None) == EINVAL
    assert L.gini_rank(fake, 4, 8193, 9000, fake, ws, 1 << 20, None) == EINVAL
    assert L.gini_rank(fake, 4, 8, 4, fake, ws, 1 << 20, None) == EINVAL
    assert L.gini_rank(None, 4, 8, 8, fake, ws, 1 << 20, None) == EINVAL
    # gini_dist: nu <= 1, n < 2, p > 1024, FULL needs F32, small workspace
    assert L.gini_dist(fake, 10, 5, 5, bad_nu, 1, 0, 0, fake, 10, 100, None, None, ws, 1 << 20, None) == EINVAL
    assert L.gini_dist(fake, 1, 5, 5, nu, 1, 0, 0, fake, 10, 100, None, None, ws, 1 << 20, None) == EINVAL
    assert L.gini_dist(fake, 10, 8193, 8193, nu, 1, 0, 0, fake, 10, 100, None, None, ws, 1 << 20, None) == EINVAL
    assert L.gini_dist(fake, 10, 5, 5, nu, 1, 0, 1, fake, 10, 100, None, None, ws, 1 << 20, None) == EINVAL
    assert L.gini_dist(fake, 10, 5, 5, nu, 1, 1, 3, fake, 10, 100, None, None, ws, 1 << 20, None) == EINVAL
    assert L.gini_dist(fake, 10, 5, 5, nu, 1, 0, 0, fake, 10, 100, None, None, ws, 8, None) == ENOMEM
    # gini_stress_grad: k = 1 and k > 8, nu <= 1, zero sum_delta2, unaligned tiled data
    args = lambda k, nu_, sd2, delta=fake, layout=0: (fake, 10, k, nu_, delta, layout, 0, 10, None,
                                                      sd2, fake, None, ws, 1 << 20, None)
    assert L.gini_stress_grad(*args(1, 2.0, 1.0)) == EINVAL
    assert L.gini_stress_grad(*args(9, 2.0, 1.0)) == EINVAL
    assert L.gini_stress_grad(*args(2, 0.5, 1.0)) == EINVAL
    assert L.gini_stress_grad(*args(2, 2.0, 0.0)) == EDEG
    assert L.gini_stress_grad(*args(2, 2.0, 1.0, delta=ctypes.c_void_p(0x1004), layout=1)) == EINVAL
    # gini_mds_fit: negative iterations, non-positive step
    a = _lib.FitArgs(n=10, k=2, nu=2.0, delta_dev=0x1000, layout=0, dtype=0, ldd=10,
                     sum_delta2=1.0, eta=0.0, iters=5, Y_dev=0x3000)
    assert L.gini_mds_fit(ctypes.byref(a), ws, 1 << 20, None) == EINVAL
    a.eta, a.iters = 1.0, -1
    assert L.gini_mds_fit(ctypes.byref(a), ws, 1 << 20, None) == EINVAL
    a.iters, a.sum_delta2 = 5, 0.0
    assert L.gini_mds_fit(ctypes.byref(a), ws, 1 << 20, None) == EDEG


def test_misaligned_workspace_is_rejected_on_the_host(L):
    # fake device addresses: every call must return EINVAL before it touches them
    from paper_2605_25124_gb300 import _lib
    EINVAL = _lib.GINI_EINVAL
    data, ws = 0x10000000, 0x20000010  # ws 16-byte but not 256-byte aligned
    big = 1 << 40
    nu = (ctypes.c_double * 1)(2.0)
    assert L.gini_dist(data, 100, 8, 8, nu, 1, 1, 0, data, 0, 0, None, None, ws, big, None) == EINVAL
    assert L.gini_rank(data, 10, 8, 8, data, ws, big, None) == EINVAL
    assert L.gini_stress_grad(data, 100, 2, 2.0, data, 1, 0, 0, None, 1.0, data, data, ws, big,
                              None) == EINVAL
    args = _lib.FitArgs()
    args.n, args.k, args.nu, args.delta_dev = 100, 2, 2.0, data
    args.layout, args.dtype, args.sum_delta2, args.eta, args.iters = 1, 0, 1.0, 0.1, 5
    args.Y_dev = data
    assert L.gini_mds_fit(ctypes.byref(args), ws, big, None) == EINVAL
    assert L.gini_classical_mds(data, 100, 1, 0, 0, None, 2, 5, 0, data, data, ws, big,
                                None) == EINVAL
    assert L.gini_distance_correlations(data, 100, 4, 4, data, 2, 1, data, ws, big,
                                        None) == EINVAL
    assert L.gini_silhouette(data, 100, 2, data, 2, data, ws, big, None) == EINVAL


def test_deterministic_mode_is_per_thread(L):
    import threading
    assert L.gini_get_deterministic() == 0
    L.gini_set_deterministic(1)
    seen = []
    t = threading.Thread(target=lambda: seen.append(L.gini_get_deterministic()))
    t.start()
    t.join()
    assert L.gini_get_deterministic() == 1 and seen == [0]
    L.gini_set_deterministic(0)
    assert L.gini_get_deterministic() == 0
