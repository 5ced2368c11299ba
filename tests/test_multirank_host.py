"""Host logic of the N > 1 benchmark path on the CPU: two `gloo` ranks (the GPU runs use one
NCCL rank per GPU) each time their own replica; the job's time is the slowest rank's, every rank
sees it, and the whole-job rate counts every rank's units."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_seconds = 1.5 + rank          # rank 1 is the slower replica
        t = bench.max_over_ranks(local_seconds, dist, torch.device("cpu"))
        rate = bench.whole_job_rate(world, 128, 3, t)
        out[rank] = (t, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == 2.5
    assert abs(rate - 2 * 128 * 3 / 2.5) < 1e-12


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.75, None, None) == 0.75
    assert bench.whole_job_rate(1, 128, 3, 1.5) == 256.0
