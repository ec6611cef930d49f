"""Multi-rank host logic on CPU (gloo, world size 2).

The solves shard by contiguous mode ranges with no data-path collective; these tests
check the shard partition, that sharded solves (the O(N) oracle standing in for each
rank's GPU) gathered across ranks equal the unsharded solve, the bench's max-over-ranks
timing reduction, and that a failing rank is detected by the others on the host (a
short process-group timeout), without any GPU.
"""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=30):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def _run(fn, world=2, *args):
    import torch.multiprocessing as mp
    mp.spawn(fn, args=(world, _free_port()) + args, nprocs=world, join=True)


def test_shard_range_partitions_the_modes():
    from paper_1701_03787_gb300.sharding import shard_range
    for n in (0, 1, 2, 7, 544, 8320, 525312):
        for world in (1, 2, 3, 4, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0
            for (b0, c0), (b1, _) in zip(got, got[1:]):
                assert b0 + c0 == b1
            assert sum(c for _, c in got) == n
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _sharded_oracle_worker(rank, world, port):
    import torch
    dist = _init(rank, world, port)
    from oracle import on
    from oracle import solve as so
    from paper_1701_03787_gb300 import inputs
    from paper_1701_03787_gb300.sharding import shard_range
    N, Nx, Nz, nu, dt = 40, 8, 6, 1 / 180, 1e-3
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=7)
    begin, count = shard_range(z2.size, rank, world)
    for problem in ("helmholtz", "biharmonic"):
        mine = on.solve_modes(problem, N, z2[begin:begin + count], so.c_of(nu, dt), F[begin:begin + count])
        parts = [None] * world
        dist.all_gather_object(parts, (begin, mine))
        if rank == 0:
            full = np.concatenate([p for _, p in sorted(parts, key=lambda t: t[0])])
            ref = on.solve_modes(problem, N, z2, so.c_of(nu, dt), F)
            assert np.array_equal(full, ref)
    dist.barrier()
    dist.destroy_process_group()
    del torch


def test_sharded_solves_gather_to_the_full_solve():
    _run(_sharded_oracle_worker)


def _max_worker(rank, world, port):
    dist = _init(rank, world, port)
    import bench
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
    assert got == [10.0 + world - 1, 5.0]
    assert bench.max_over_ranks([1.5], None, "cpu") == [1.5]
    dist.barrier()
    dist.destroy_process_group()


def test_bench_takes_the_max_over_ranks():
    _run(_max_worker)


def _failing_worker(rank, world, port):
    dist = _init(rank, world, port, timeout_s=5)
    if rank == 1:
        raise RuntimeError("rank 1 fails before the collective")
    import torch
    t = torch.ones(1)
    dist.all_reduce(t)              # never completed by rank 1: times out on rank 0


def test_a_failing_rank_is_detected_on_the_host():
    import torch.multiprocessing as mp
    with pytest.raises(mp.ProcessRaisedException):
        _run(_failing_worker)
