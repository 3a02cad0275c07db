"""Host logic of bench.py's multi-GPU mode (independent replicas, one per
rank), run as two gloo ranks on the CPU: the job time is the slowest rank's,
and the job throughput counts every rank's updates."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 3.0][rank]
    slowest = bench.max_over_ranks(seconds, dist)
    mlups = bench.job_throughput(6e6, seconds, world, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, mlups))


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, mlups in res:
        assert slowest == 3.0
        assert mlups == pytest.approx(2 * 6e6 / 3.0 / 1e6)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_throughput(1e6, 0.5, 1) == pytest.approx(2.0)
