"""Multi-rank host logic of bench.py on CPU with gloo ranks (world size 2):
each rank walks its own replica (distinct seeds), the timings are combined by
max over ranks and the work by sum, with no data-path collective."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        assert (w, r) == (world, rank)
        total_ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
        e2e = 1.0 + rank
        moves = 1000 * (rank + 1)
        res = bench.combine_ranks(dist, total_ms, e2e, moves, 2 * moves)
        out[rank] = (bench.rank_seed(rank),) + res
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_sum_work():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][1:] == out[1][1:] == (150.0, 2.0, 3000.0, 6000.0)
    assert out[0][0] != out[1][0]                  # distinct replicas


def test_single_rank_passthrough():
    assert bench.combine_ranks(None, 10.0, 2.0, 5, 6) == (10.0, 2.0, 5.0, 6.0)
