"""Line sharding of one surface across ranks, on CPU with gloo ranks (world
size 2): the LPT split covers every line exactly once, and the surface gathered
on rank 0 equals the surface computed by one rank.  The per-line walks here are
the CPU oracle's (the library is not needed to test the split and the gather);
tests/test_gpu_parity.py runs the same split through the library on a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1302_2320_gb300 import shard

L, SEED, U, C, BUDGET = 6, 3, 1e-6, 500, 40_000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _walk_lines(ells):
    out = {}
    for ell in ells:
        st = oracle.run_line(oracle.SQUARE, L, ell, SEED, U, C, 800, BUDGET, 0)
        out[ell] = oracle.assemble(L * L, ell, st.lng, st.visited, U)
    return out


def _costs():
    N = L * L
    return shard.line_costs(N, 2 * N, 4, 2)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shares = shard.lpt_partition(_costs(), world)
        local = _walk_lines(shares[rank])
        merged = shard.gather_lines(dist, local)
        if rank == 0:
            vals, offs = shard.ragged_surface(merged, L * L // 2 + 1)
            out["vals"], out["offs"] = vals, offs
            out["shares"] = shares
        else:
            assert merged is None
    finally:
        dist.destroy_process_group()


def test_lpt_partition_covers_every_line_once_and_balances():
    costs = shard.line_costs(64 * 64, 2 * 64 * 64, 4, 2)
    for n in (1, 2, 3, 8):
        shares = shard.lpt_partition(costs, n)
        flat = sorted(l for s in shares for l in s)
        assert flat == list(range(2049))
        loads = [sum(costs[l] for l in s) for s in shares]
        # LPT is within 4/3 of optimal; here the largest line is small against the total
        assert max(loads) <= 1.02 * (sum(loads) / n) + max(costs.values())
    assert shard.lpt_partition({0: 1, 1: 5, 2: 3}, 2) == [[1], [0, 2]]
    with pytest.raises(ValueError):
        shard.lpt_partition(costs, 0)


def test_gather_rejects_duplicates_and_missing_lines():
    assert shard.gather_lines(None, {1: [0.0]}) == {1: [0.0]}
    with pytest.raises(ValueError):
        shard.ragged_surface({0: [0.0], 2: [1.0]}, 3)


def test_two_gloo_ranks_gather_the_single_rank_surface():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    shares = out["shares"]
    assert sorted(shares[0] + shares[1]) == list(range(L * L // 2 + 1))
    assert not set(shares[0]) & set(shares[1])
    ref_vals, ref_offs = shard.ragged_surface(_walk_lines(range(L * L // 2 + 1)), L * L // 2 + 1)
    assert np.array_equal(out["offs"], ref_offs)
    assert np.array_equal(out["vals"], ref_vals)          # -inf where unvisited, on both
