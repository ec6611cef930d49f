"""Sharded solves on one GPU: each emulated rank solves its contiguous mode range
(shen_solve_modes via sharding.solve_shard), one after the other (no rank waits on
another); the concatenated shards must equal the whole-plan solve bit for bit."""
import pytest

from paper_1701_03787_gb300 import Plan, inputs
from paper_1701_03787_gb300.sharding import shard_range, solve_shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 8])
@pytest.mark.parametrize("problem,precision", [("helmholtz", "df"), ("biharmonic", "df"),
                                               ("biharmonic", "fp64"), ("helmholtz", "df_r1")])
def test_shards_concatenate_to_the_full_solve(world, problem, precision):
    import torch
    with Plan(200, 20, 18, 1 / 2000, 1e-4) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=51)
        full = plan.solve(problem, f, precision=precision)
        parts = []
        for rank in range(world):
            b, c = shard_range(plan.n_modes, rank, world)
            parts.append(solve_shard(plan, problem, f[b:b + c].contiguous(), rank=rank, world=world,
                                     precision=precision))
        torch.cuda.synchronize()
        assert torch.equal(torch.cat(parts), full)


def test_empty_shards_do_nothing():
    """More ranks than modes: the ranks past the last mode hold no columns (empty tensors,
    possibly NULL data pointers); their solve and transform calls succeed and launch nothing."""
    import torch
    with Plan(64, 2, 2, 1 / 180, 1e-3) as plan:                     # 2 x 2 = 4 modes
        assert plan.n_modes == 4
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=52)
        for problem in ("helmholtz", "biharmonic"):
            full = plan.solve(problem, f, precision="df")
            parts = []
            for rank in range(6):
                b, c = shard_range(plan.n_modes, rank, 6)
                parts.append(solve_shard(plan, problem, f[b:b + c].contiguous(), rank=rank, world=6, precision="df"))
            torch.cuda.synchronize()
            assert [p.shape[0] for p in parts] == [1, 1, 1, 1, 0, 0]
            assert torch.equal(torch.cat(parts), full)
        empty = torch.empty((0, plan.N), dtype=torch.complex128, device="cuda")
        for kind in ("inverse", "scalar", "forward"):
            for space in ("chebyshev", "dirichlet", "biharmonic"):
                assert plan.transform_modes(kind, space, plan.n_modes, empty).shape == (0, plan.N)
        torch.cuda.synchronize()
        plan.check_device()
