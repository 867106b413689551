"""The benchmark's multi-rank reduction (one process per GPU, replicas of the workload): the job's
step time is the slowest rank's and its value counts every rank's units.  Exercised with two gloo
ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        t = bench.slowest_rank_ms(dist, 10.0 + 5.0 * rank, "cpu")
        out[rank] = (t, bench.job_value(world, 1000.0, t))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_value_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29000 + os.getpid() % 1000
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            t, v = out[r]
            assert t == pytest.approx(15.0)
            assert v == pytest.approx(2 * 1000.0 / 0.015)
