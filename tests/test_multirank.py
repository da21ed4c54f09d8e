"""The benchmark's multi-rank form on CPU: world_size 2 over gloo (127.0.0.1).  Each rank
labels its own replica of the work (no data-path collective); the timing is the max over
ranks and the throughput counts every rank's pixels."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 1.0 + r seconds for its replica
        t = bench.max_over_ranks(1.0 + rank, world)
        v = bench.aggregate_gpx_s(6 * 8192 * 8192, world, t)
        # the replica split: every rank labels the full workload (weak scaling)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_aggregate_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in res:
        assert t == pytest.approx(2.0)  # the slowest rank
        assert v == pytest.approx(2 * 6 * 8192 * 8192 / 2.0 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_gpx_s(10**9, 1, 0.5) == pytest.approx(2.0)
