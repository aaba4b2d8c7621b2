"""The N > 1 bench path: independent replicas, one per rank, whose whole-job
figures are the slowest rank's time and the sum of the ranks' work.  Runs as
two gloo ranks on the CPU (no GPU, no collective in the data path)."""

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, work = bench.aggregate_replicas(10.0 + 5.0 * rank, 1e12 * (rank + 1), "cpu")
        q.put((rank, ms, work))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, work in out:
        assert ms == pytest.approx(15.0)      # the slowest rank
        assert work == pytest.approx(3e12)    # all ranks' work


def test_single_process_is_identity():
    assert bench.aggregate_replicas(12.5, 7.0, "cpu") == (12.5, 7.0)
