"""bench.py's multi-rank path without a GPU: two gloo ranks on the CPU
(127.0.0.1) reduce their timings the way the GPU replicas do -- the slowest
rank's time and the sum of the iterations -- and read their rank from the
launcher's environment."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    ws, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    try:
        # rank k: (k + 1) * 10 ms for (k + 1) * 100 iterations
        out = bench.reduce_timing(10.0 * (r + 1), 100 * (r + 1), dist, torch.device("cpu"))
        q.put((r, ws, local, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_like_the_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, (ms, units) in got:
        assert ms == 20.0 and units == 300   # max time, summed work


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(12.5, 7, None, None) == (12.5, 7)
