"""The N > 1 path of bench.py on the CPU: two gloo ranks, each with its own
independent problem (no data-path collective), the step time reduced to the
maximum over ranks, and the whole-job rate counting the work of every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # rank r "took" 10 (r + 1) ms: every rank must see the slowest one
        t_max = bench.max_over_ranks(10.0 * (rank + 1), w, torch.device("cpu"))
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(r))
        out[rank] = (t_max, seeds)
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_independent_seeds():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t_max, seeds = res[rank]
        assert t_max == pytest.approx(10.0 * world)
        assert len(set(seeds)) == world  # every rank has its own problem


def test_job_rate_counts_every_rank():
    ops = 2.0 * 8192 ** 3
    one = bench.job_gflops(ops, 1, 3, 1737.0 * 3)
    two = bench.job_gflops(ops, 2, 3, 1737.0 * 3)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(ops / 1.737 / 1e9)
    # a slower rank lowers the job rate through the max-over-ranks time
    assert bench.job_gflops(ops, 2, 3, 2000.0 * 3) < two


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(5.0, 1, torch.device("cpu")) == 5.0
