"""Host-side checks of the Delta build's segment shapes, read from csrc/dist.cu.

dispatch_dist picks, by vector length m, E registers x L lanes per pair and
the bounds TL, TR: registers t < TL are loaded without a bounds test (every
lane holds a real element there for the smallest m of the bucket) and
registers t >= TR hold nothing.  A TL too large would read past the end of
a row of X, so the bounds are checked here for every bucket, together with
bench.py's copy of the table (its count of the network's minima)."""
import os
import re
import sys

import pytest

ROOT = os.path.join(os.path.dirname(__file__), "..")
SRC = os.path.join(ROOT, "paper_2605_25124_gb300", "csrc", "dist.cu")


def _shapes():
    src = open(SRC).read()
    body = src[src.index("static cudaError_t dispatch_dist("):]
    body = body[body.index("} else {"):body.index("\n}\n")]
    rows = [(int(m), int(E), int(L), int(TL), int(TR)) for m, E, L, TL, TR in re.findall(
        r"if \(m <= (\d+)\) return launch_dist<(\d+), (\d+), KIND, (\d+), (\d+)>", body)]
    last = re.search(r"\n    return launch_dist<(\d+), (\d+), KIND, (\d+), (\d+)>", body)
    E, L, TL, TR = (int(v) for v in last.groups())
    rows.append((E * L, E, L, TL, TR))
    return rows


def test_every_bucket_bounds_its_registers():
    rows = _shapes()
    assert rows[-1][0] == 1024 and len(rows) == 13
    m_min = 1
    for m_max, E, L, TL, TR in rows:
        assert L & (L - 1) == 0 and L <= 32
        assert E * L >= m_max, (m_max, E, L)          # room for every element
        assert TL * L <= m_min, (m_max, TL, L)        # t < TL: e = t L + ls < m, every lane
        assert TR * L >= m_max and TR <= E            # t >= TR: e >= m, no lane
        # element e = t L + ls of a lane never passes m for t < TL
        for t in range(TL):
            assert t * L + (L - 1) < m_min
        m_min = m_max + 1


def test_bench_uses_the_same_shapes():
    sys.path.insert(0, ROOT)
    import bench
    from inspect import getsource
    src = getsource(bench._network_minima)
    table = eval(re.search(r"table = (\[.*?\])\n", src, re.S).group(1))
    assert [(m, E, L, TR) for m, E, L, _, TR in _shapes()] == table


@pytest.mark.parametrize("p,E", [(513, 20), (640, 20), (641, 24), (768, 24), (769, 25), (784, 25),
                                 (800, 25), (801, 28), (896, 28), (897, 32), (1024, 32)])
def test_32_lane_register_counts(p, E):
    for m_max, e, L, TL, TR in _shapes():
        if p <= m_max:
            assert (e, L) == (E, 32)
            return
    raise AssertionError(p)
