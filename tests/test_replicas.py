"""Multi-GPU runs of bench.py are independent replicas (no data-path
exchange): each rank times the same workload and the job reports the units of
all ranks over the slowest rank's time. The aggregation is checked here with
two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r processed 1000 * (r + 1) units in 10 * (r + 1) ms
        value, ms = bench.replica_throughput(1000 * (rank + 1), 10.0 * (rank + 1), world)
        out.put((rank, value, ms, bench.max_over_ranks(float(rank), world), bench.sum_over_ranks(1.0, world)))
        bench.barrier_and_sync(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_aggregate():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, mx, sm in res:
        assert ms == pytest.approx(20.0)               # the slowest rank
        assert value == pytest.approx(3000 / 0.020)    # all units over that time
        assert mx == 1.0 and sm == 2.0


def test_single_rank_is_identity():
    import bench
    assert bench.replica_throughput(500, 250.0, 1) == (2000.0, 250.0)
