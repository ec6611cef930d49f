"""The product's shard path across processes: two ranks (gloo process group, both on
cuda:0 of this one-GPU machine) each solve their contiguous mode range of one field with
shen_solve_modes (``sharding.solve_shard``), and the ranges gathered on rank 0 equal the
whole-plan solve bit for bit.  The ranks' kernels are independent (no data-path
collective, no rank waits on another rank's kernel); only the host gathers."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    torch.cuda.set_device(0)
    from paper_1701_03787_gb300 import Plan, inputs
    from paper_1701_03787_gb300.sharding import shard_range, solve_shard
    N, Nx, Nz, nu, dt = 128, 32, 24, 1 / 180, 5e-4
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=23)
        begin, count = shard_range(plan.n_modes, rank, world)
        for problem in ("helmholtz", "biharmonic"):
            for precision in ("fp64", "df"):
                mine = solve_shard(plan, problem, f[begin:begin + count].contiguous(), rank=rank, world=world,
                                   precision=precision)
                torch.cuda.synchronize()
                parts = [None] * world
                dist.all_gather_object(parts, (begin, mine.cpu().numpy()))
                if rank == 0:
                    full = np.concatenate([p for _, p in sorted(parts, key=lambda t: t[0])])
                    whole = plan.solve(problem, f, precision=precision).cpu().numpy()
                    assert np.array_equal(full, whole), (problem, precision)
    dist.barrier()
    dist.destroy_process_group()


def test_shards_on_two_ranks_gather_to_the_whole_solve():
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
