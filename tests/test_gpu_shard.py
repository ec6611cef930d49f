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
