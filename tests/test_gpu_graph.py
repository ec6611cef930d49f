"""Solves captured into CUDA graphs (stream capture) and replayed.

The solve entry points only enqueue kernels (and, for batched plans, a memset of the
plan's queue counter) on the caller's stream, so they can be captured.  A replay with
new data in the captured input buffers must give the eager result bit for bit.
"""
import pytest

from paper_1701_03787_gb300 import BatchPlan, Plan, inputs

pytestmark = pytest.mark.gpu


def _capture(fn):
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                                   # warm-up outside the graph
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_plan_solves_replay_in_a_graph(precision):
    import torch
    with Plan(257, 24, 16, 1 / 2000, 1e-4) as plan:
        fh = torch.empty((plan.n_modes, plan.N), dtype=torch.complex128, device="cuda")
        fb = torch.empty_like(fh)
        uh, ub = torch.empty_like(fh), torch.empty_like(fh)

        def step():
            plan.helmholtz_solve(fh, uh, precision=precision)
            plan.biharmonic_solve(fb, ub, precision=precision)
        fh.copy_(inputs.rhs_torch(plan.n_modes, plan.N, seed=1))
        fb.copy_(inputs.rhs_torch(plan.n_modes, plan.N, seed=2))
        g = _capture(step)
        for seed in (3, 4):
            fh.copy_(inputs.rhs_torch(plan.n_modes, plan.N, seed=seed))
            fb.copy_(inputs.rhs_torch(plan.n_modes, plan.N, seed=seed + 10))
            uh.zero_()
            ub.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(uh, plan.helmholtz_solve(fh, precision=precision))
            assert torch.equal(ub, plan.biharmonic_solve(fb, precision=precision))


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_batch_solves_replay_in_a_graph(precision):
    import torch
    insts = inputs.batch_instances(48, seed=9)
    with BatchPlan(insts) as bp:
        fh = inputs.batch_rhs_torch(bp.offsets, insts, seed=1)
        fb = inputs.batch_rhs_torch(bp.offsets, insts, seed=2)
        uh, ub = torch.empty_like(fh), torch.empty_like(fh)

        def step():
            bp.solve("helmholtz", fh, uh, precision=precision)
            bp.solve("biharmonic", fb, ub, precision=precision)
        g = _capture(step)
        for seed in (3, 4, 5):
            fh.copy_(inputs.batch_rhs_torch(bp.offsets, insts, seed=seed))
            fb.copy_(inputs.batch_rhs_torch(bp.offsets, insts, seed=seed + 10))
            uh.zero_()
            ub.zero_()
            g.replay()
            torch.cuda.synchronize()
            bp.check_device()
            assert torch.equal(uh, bp.solve("helmholtz", fh, precision=precision))
            assert torch.equal(ub, bp.solve("biharmonic", fb, precision=precision))
