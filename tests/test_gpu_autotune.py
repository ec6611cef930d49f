"""GPU tests of the autotuner and of precision "auto".

The autotuner picks among paths that all meet the 1e-10 bar; so after tuning, an "auto"
solve must equal the solve with the chosen precision bit for bit.  Shapes 0 and 1 of the
float-float sweeps run the same arithmetic (same bits); shapes 2 and 3 renormalise once per
row instead of once per term, so a float-float result after tuning equals the one before
it bit for bit when the tuner kept shape 0 or 1, and to the float-float rounding otherwise.
"""
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import BatchPlan, Plan, ShenError, inputs

pytestmark = pytest.mark.gpu

CANDIDATES = {"helmholtz": {"fp64", "df", "df_r1", "fp32_r1"}, "biharmonic": {"fp64", "df"}}


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_plan_autotune_and_auto_precision(problem):
    import torch
    with Plan(384, 48, 32, 1 / 2000, 1e-4) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=41)
        before = plan.solve(problem, f, precision="df")
        u_default = plan.solve(problem, f, precision="auto")          # SHEN_DF until tuned
        torch.cuda.synchronize()
        assert torch.equal(u_default, before)
        name, ms = plan.autotune(problem, f)
        assert name in CANDIDATES[problem] and ms > 0
        u_auto = plan.solve(problem, f, precision="auto")
        u_named = plan.solve(problem, f, precision=name)
        after = plan.solve(problem, f, precision="df")
        torch.cuda.synchronize()
        assert torch.equal(u_auto, u_named)
        if plan.shape(problem) in (0, 1):
            assert torch.equal(after, before)                          # shapes 0, 1 keep the bits
        else:
            d = torch.linalg.vector_norm(after - before, dim=1) / torch.linalg.vector_norm(before, dim=1)
            assert float(d.max()) < 1e-11
        # the tuned result still meets the bar against the O(N) oracle
        z2 = so.mode_z2(48, 32)
        modes = [0, 5, plan.n_modes // 2, plan.n_modes - 1]
        F = f[modes].cpu().numpy()
        R = on.solve_modes(problem, 384, z2[modes], so.c_of(1 / 2000, 1e-4), F)
        U = u_auto[modes].cpu().numpy()
        n = so.n_unknowns(problem, 384)
        assert max(so.rel_l2(U[i, :n], R[i, :n]) for i in range(len(modes))) < 1e-10


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_batch_autotune_and_auto_precision(problem):
    import torch
    insts = inputs.batch_instances(64, seed=13)
    with BatchPlan(insts) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=42)
        before = bp.solve(problem, f, precision="df")
        name, ms = bp.autotune(problem, f)
        assert name in {"fp64", "df"} and ms > 0
        u_auto = bp.solve(problem, f, precision="auto")
        u_named = bp.solve(problem, f, precision=name)
        after = bp.solve(problem, f, precision="df")
        torch.cuda.synchronize()
        bp.check_device()
        assert torch.equal(u_auto, u_named)
        assert torch.equal(after, before)


@pytest.mark.parametrize("N", [8, 33, 130, 1024])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_every_shape_gives_the_same_bits(problem, N):
    """Shapes 0 and 1 (rows prefetched in registers, blocks of different depth) run the same
    arithmetic: identical bits, out of place, in place and on a mode range, and the oracle's
    bar."""
    import torch
    Nx, Nz = (16, 12) if N < 1024 else (64, 64)
    with Plan(N, Nx, Nz, 1 / 2000, 1e-4) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=N)
        outs = []
        for shape in (0, 1):
            plan.set_shape(problem, shape)
            assert plan.shape(problem) == shape
            a = plan.solve(problem, f, precision="df")
            g = f.clone()
            plan.solve(problem, g, u=g, precision="df")
            h = plan.solve_modes(problem, 3, f[3:plan.n_modes - 2].contiguous(), precision="df")
            torch.cuda.synchronize()
            assert torch.equal(a, g)
            assert torch.equal(a[3:plan.n_modes - 2], h)
            outs.append(a)
        assert torch.equal(outs[0], outs[1])
        z2 = so.mode_z2(Nx, Nz)
        modes = [0, 1, plan.n_modes // 2, int(z2.argmax()), plan.n_modes - 1]
        R = on.solve_modes(problem, N, z2[modes], so.c_of(1 / 2000, 1e-4), f[modes].cpu().numpy())
        U = outs[1][modes].cpu().numpy()
        n = so.n_unknowns(problem, N)
        assert max(so.rel_l2(U[i, :n], R[i, :n]) for i in range(len(modes))) < 1e-10
        with pytest.raises(ShenError):
            plan.set_shape(problem, 4)


def test_autotune_rejects_in_place_and_bad_problem():
    with Plan(64, 8, 8, 1 / 180, 1e-3) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=43)
        with pytest.raises(ShenError):
            plan.autotune("helmholtz", f, f)
        with pytest.raises(KeyError):
            plan.autotune("poisson", f)
