"""The replicas path of bench.py (one process per GPU, no data-path
collective) on CPU: two gloo ranks, the barrier, the max over ranks and the
whole-job rate; the reference arm's non-zero ranks return without work."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, local, w = bench._dist_init(None)
    bench._barrier(w)
    # rank 1 is the slow replica: 2 s for the same 100 units
    secs = 1.0 + rank
    rate = bench._replica_rate(100, secs, w)
    mx = bench._max_over_ranks(secs, w)
    ref = bench.run_reference(None, r, w) if r != 0 else "rank0"
    q.put((r, w, rate, mx, ref))
    torch.distributed.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, rate, mx, ref in out:
        assert w == 2
        assert mx == 2.0                    # the slowest rank sets the time
        assert rate == pytest.approx(100.0)  # 2 ranks x 100 units / 2 s
    assert out[1][4] is None                 # reference arm: rank 1 does no work


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._replica_rate(200, 0.5, 1) == 400.0
