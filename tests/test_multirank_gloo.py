"""The bench's multi-GPU path runs independent replicas (weak scaling, no
data-path collective); its only cross-rank steps are a barrier and the max of
the per-rank timed totals.  This checks that logic with two gloo ranks on the
host."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    rate = bench.whole_job_rate(1000.0, world, mx)
    q.put((rank, mx, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, rate in got:
        assert mx == 15.0                       # the slowest rank's total
        assert abs(rate - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5000.0
