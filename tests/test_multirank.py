"""The N > 1 host logic of the benchmark (replicas: every rank solves its own copy; the
job time is the slowest rank's), on two CPU processes over gloo."""
import os
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.max_over_ranks(1.5 + rank, torch.device("cpu"), world)
        w = bench.max_over_ranks(3.0 - rank, torch.device("cpu"), world)
        out[rank] = (v, w)
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + (os.getpid() % 1000)
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
        assert dict(out) == {0: (2.5, 3.0), 1: (2.5, 3.0)}


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25, torch.device("cpu"), 1) == 4.25
