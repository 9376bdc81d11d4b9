"""The compile-time sorting networks of csrc/sortnet.cuh, checked on the CPU.

The odd-length in-lane merge tables (BitonicLeaf<N>) are read from the header
and checked by the 0-1 principle; then a lane-level model of the whole
alternating-layout sort is run on random keys for every shape the Delta build
dispatches: 32 lanes x E registers (E = 20, 24, 25, 28, 32), so that the
non-power-of-two register counts of the cross-lane stages and the recursive
in-lane merge are covered, and the segments of 1 to 16 lanes."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2605_25124_gb300", "csrc",
                   "sortnet.cuh")


def _leaves():
    src = open(HDR).read()
    out = {}
    for N, body in re.findall(r"struct BitonicLeaf<(\d+)> \{(.*?)\n\};", src, re.S):
        n = int(re.search(r"int n = (\d+);", body).group(1))
        a = [int(x) for x in re.search(r"a\[\d+\] = \{(.*?)\}", body, re.S).group(1).split(",")]
        b = [int(x) for x in re.search(r"b\[\d+\] = \{(.*?)\}", body, re.S).group(1).split(",")]
        assert len(a) == len(b) == n
        out[int(N)] = list(zip(a, b))
    return out


def _inlane_bitonic(E, leaves, off=0):
    """Compare-exchanges of bitonic_window<off, E>: half-cleaners down to odd leaves."""
    if E % 2 == 0 and E >= 2:
        h = E // 2
        return ([(off + t, off + t + h) for t in range(h)] + _inlane_bitonic(h, leaves, off) +
                _inlane_bitonic(h, leaves, off + h))
    if E > 1:
        return [(off + i, off + j) for i, j in leaves[E]]
    return []


def _cyclic_bitonic_01(n):
    out = set()
    for k in range(n + 1):
        base = [1] * k + [0] * (n - k)
        for r in range(n):
            out.add(tuple(base[r:] + base[:r]))
    return sorted(out)


def _batcher_merge_exchange(n):
    """Batcher's odd-even merge sort for any n (Knuth, TAOCP 3, 5.2.2 M)."""
    net, p = [], 1
    while p < n:
        k = p
        while k >= 1:
            j = k % p
            while j < n - k:
                for i in range(k):
                    if i + j + k < n and (i + j) // (2 * p) == (i + j + k) // (2 * p):
                        net.append((i + j, i + j + k))
                j += 2 * k
            k //= 2
        p *= 2
    return net


def test_leaf_tables_sort_every_cyclic_bitonic_input():
    leaves = _leaves()
    assert sorted(leaves) == [3, 5, 7, 25]
    assert {N: len(net) for N, net in leaves.items()} == {3: 3, 5: 8, 7: 12, 25: 72}
    for N, net in leaves.items():
        assert all(0 <= i < j < N for i, j in net)
        inputs = _cyclic_bitonic_01(N)
        assert len(inputs) == N * (N - 1) + 2
        for v in inputs:
            w = list(v)
            for i, j in net:
                if w[i] > w[j]:
                    w[i], w[j] = w[j], w[i]
            assert w == sorted(w), (N, v)


@pytest.mark.parametrize("E", [20, 24, 25, 28, 32])
def test_inlane_merge_sorts_every_cyclic_bitonic_input(E):
    net = _inlane_bitonic(E, _leaves())
    for v in _cyclic_bitonic_01(E):
        w = list(v)
        for i, j in net:
            if w[i] > w[j]:
                w[i], w[j] = w[j], w[i]
        assert w == sorted(w), v


def _alternating_sort(u, insort, bisort):
    """The merge levels of seg_sort_alternating on (L, E) keys, lane by lane."""
    L, E = u.shape
    ls = np.arange(L)
    s0 = np.where(ls & 1, -1.0, 1.0).astype(np.float32)

    def cas_all(u, net):
        for a, b in net:
            lo, hi = np.minimum(u[:, a], u[:, b]), np.maximum(u[:, a], u[:, b])
            u[:, a], u[:, b] = lo, hi

    cas_all(u, insort)
    K = 2
    while K <= L:
        s = s0.copy()
        if K >= 4:
            sn = np.where(ls & (K // 2), -1.0, 1.0).astype(np.float32)
            u *= (sn * s)[:, None]
            s = sn
        u = np.minimum(u, -u[ls ^ (K - 1)])
        D = K // 4
        while D >= 1:
            sn = np.where(ls & D, -1.0, 1.0).astype(np.float32)
            u *= (sn * s)[:, None]
            s = sn
            if D >= 2:
                u = np.minimum(u, -u[ls ^ D])
            else:  # opposite orientations: register t meets E-1-t
                u = np.minimum(u, -u[ls ^ 1][:, ::-1])
            D //= 2
        assert np.all(s == s0)
        cas_all(u, bisort)
        K *= 2
    return u


@pytest.mark.parametrize("E,ms", [(20, (513, 600, 640)), (24, (641, 700, 768)),
                                  (25, (769, 784, 800)), (28, (801, 850, 896)),
                                  (32, (897, 1000, 1024))])
def test_alternating_sort_32_lanes(E, ms):
    L = 32
    rng = np.random.default_rng(E)
    insort, bisort = _batcher_merge_exchange(E), _inlane_bitonic(E, _leaves())
    for m in ms:
        for kind in range(3):
            if kind == 0:
                x = rng.standard_normal(m)
            elif kind == 1:
                x = rng.integers(-2, 3, m).astype(np.float64)  # many ties
            else:
                x = np.clip(rng.normal(0.0, 0.1, m), 0.0, 1.0)
            x = x.astype(np.float32)
            u = np.full((L, E), np.finfo(np.float32).max, dtype=np.float32)
            for l in range(L):
                for t in range(E):
                    e = t * L + l
                    if e < m:
                        u[l, t] = -x[e] if l & 1 else x[e]
            u = _alternating_sort(u, insort, bisort)
            z = np.empty(L * E, dtype=np.float32)
            for l in range(L):
                for t in range(E):
                    odd = l & 1
                    z[E * l + (E - 1 - t if odd else t)] = -u[l, t] if odd else u[l, t]
            # padding of odd lanes sits at the bottom, of even lanes at the top
            n_lo = sum(E - min(E, (m - l + L - 1) // L) for l in range(1, L, 2))
            assert np.all(np.diff(z) >= 0)
            np.testing.assert_array_equal(z[n_lo:n_lo + m], np.sort(x))


def test_bench_counts_the_network_the_header_defines():
    # bench.py's network_frac counts the minima of the tables above
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
    import bench
    leaves = _leaves()
    assert {N: len(net) for N, net in leaves.items()} == \
        {N: c for N, c in bench.BITONIC_LEAF_STEPS.items() if N > 1}
    for E in (20, 24, 25, 28, 32):
        assert bench._inlane_merge_steps(E) == len(_inlane_bitonic(E, leaves))
    # p = 784: 32 lanes x (2 x 140 odd-even + 15 x 25 cross-lane + 5 x 2 x 72 in-lane)
    assert bench._network_minima(784) == 32 * (280 + 375 + 720)


@pytest.mark.parametrize("E,L,ms", [(4, 1, (1, 3, 4)), (8, 1, (5, 8)), (16, 1, (9, 16)),
                                    (32, 1, (17, 32)), (32, 2, (33, 50, 64)),
                                    (32, 4, (65, 100, 128)), (32, 8, (129, 200, 256)),
                                    (32, 16, (257, 300, 512))])
def test_alternating_sort_narrow_segments(E, L, ms):
    # segments of 1 to 16 lanes (the shapes below 513 components): one segment
    rng = np.random.default_rng(100 * L + E)
    insort, bisort = _batcher_merge_exchange(E), _inlane_bitonic(E, _leaves())
    for m in ms:
        x = rng.integers(-3, 4, m).astype(np.float32) * np.float32(0.5)
        u = np.full((L, E), np.finfo(np.float32).max, dtype=np.float32)
        for l in range(L):
            for t in range(E):
                e = t * L + l
                if e < m:
                    u[l, t] = -x[e] if (L >= 2 and l & 1) else x[e]
        u = _alternating_sort(u, insort, bisort)
        z = np.empty(L * E, dtype=np.float32)
        for l in range(L):
            for t in range(E):
                odd = L >= 2 and (l & 1)
                z[E * l + (E - 1 - t if odd else t)] = -u[l, t] if odd else u[l, t]
        n_lo = sum(E - min(E, (m - l + L - 1) // L) for l in range(1, L, 2)) if L >= 2 else 0
        assert np.all(np.diff(z) >= 0)
        np.testing.assert_array_equal(z[n_lo:n_lo + m], np.sort(x))
