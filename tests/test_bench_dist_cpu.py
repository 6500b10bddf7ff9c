"""bench.py's multi-rank path on CPU: two gloo ranks (127.0.0.1) agree on the slowest
rank's time and on the whole-job throughput of independent replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank            # rank 1 is slower
        dist.barrier()
        slowest = bench.max_over_ranks(dist, mine, "cpu")
        value = bench.replica_throughput(1000.0, world, slowest)
        q.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [2.5, 2.5]
    assert [g[2] for g in got] == [pytest.approx(800.0)] * 2


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(None, 3.25) == 3.25
    assert bench.replica_throughput(10.0, 1, 2.0) == 5.0
