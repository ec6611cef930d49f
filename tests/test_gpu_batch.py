"""GPU parity of batched plans (many channels with uneven N in one persistent launch).

Each instance's block must equal the single-channel plan's result bit for bit (the
same chain code and factors run in both) and match the O(N) oracle (float64 1e-12,
float-float 1e-10 per mode column).
"""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import BatchPlan, Plan, ShenError, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df": 1e-10}


def _uneven_instances():
    return [dict(N=8, Nx=2, Nz=2, nu=1e-2, dt=1e-2), dict(N=130, Nx=8, Nz=6, nu=1 / 180, dt=1e-3),
            dict(N=9, Nx=4, Nz=4, nu=1e-3, dt=5e-3), dict(N=64, Nx=16, Nz=16, nu=1 / 180, dt=1e-3),
            dict(N=257, Nx=4, Nz=8, nu=1 / 2000, dt=1e-4), dict(N=64, Nx=6, Nz=4, nu=3e-3, dt=2e-3),
            dict(N=96, Nx=32, Nz=16, nu=1e-4, dt=1e-2, Lx=4.0, Lz=1.5)]


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_batch_matches_single_plans_and_oracle(problem, precision):
    import torch
    insts = _uneven_instances()
    with BatchPlan(insts) as bp:
        assert bp.n_instances == len(insts)
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=3)
        u = bp.solve(problem, f, precision=precision)
        torch.cuda.synchronize()
        bp.check_device()
        for i, inst in enumerate(insts):
            N = inst["N"]
            fi = f[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N).contiguous()
            ui = u[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N)
            with Plan(N, inst["Nx"], inst["Nz"], inst["nu"], inst["dt"], Lx=inst.get("Lx"), Lz=inst.get("Lz")) as p:
                us = p.solve(problem, fi, precision=precision)
                torch.cuda.synchronize()
            assert torch.equal(ui, us), i
            kw = {k: inst[k] for k in ("Lx", "Lz") if k in inst}
            z2 = so.mode_z2(inst["Nx"], inst["Nz"], **kw)
            F, U = fi.cpu().numpy(), ui.cpu().numpy()
            R = on.solve_modes(problem, N, z2, so.c_of(inst["nu"], inst["dt"]), F)
            n = so.n_unknowns(problem, N)
            for m in range(z2.size):
                assert so.rel_l2(U[m, :n], R[m, :n]) <= TOL[precision], (i, m)
                assert np.all(U[m, n:] == 0)


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_batching_workload_sampled(problem):
    """The batching workload: 4096 instances, N in {64, 96, 128, 256, 512}, grids 16..64,
    nu log-uniform [1e-4, 1e-2], dt uniform [1e-4, 1e-2]; float-float sweeps; sampled
    columns vs the O(N) oracle."""
    import torch
    insts = inputs.batch_instances(4096, seed=5)
    with BatchPlan(insts) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=6)
        u = bp.solve(problem, f, precision="df")
        torch.cuda.synchronize()
        rng = np.random.default_rng(7)
        for i in rng.choice(len(insts), size=24, replace=False):
            inst = insts[i]
            N = inst["N"]
            fi = f[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N).cpu().numpy()
            ui = u[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N).cpu().numpy()
            z2 = so.mode_z2(inst["Nx"], inst["Nz"])
            pick = rng.choice(z2.size, size=min(8, z2.size), replace=False)
            R = on.solve_modes(problem, N, z2[pick], so.c_of(inst["nu"], inst["dt"]), fi[pick])
            n = so.n_unknowns(problem, N)
            for j, m in enumerate(pick):
                assert so.rel_l2(ui[m, :n], R[j, :n]) <= TOL["df"], (i, m)


def test_batch_rejects_bad_descriptors_and_precisions():
    import torch
    with pytest.raises(ShenError):
        BatchPlan([dict(N=7, Nx=4, Nz=4, nu=1e-2, dt=1e-2)])
    with pytest.raises(ShenError):
        BatchPlan([dict(N=64, Nx=3, Nz=4, nu=1e-2, dt=1e-2)])
    with BatchPlan([dict(N=64, Nx=4, Nz=4, nu=1e-2, dt=1e-2)]) as bp:
        f = torch.zeros(bp.field_elems, dtype=torch.complex128, device="cuda")
        with pytest.raises(ShenError) as e:
            bp.solve("helmholtz", f, precision="df_r1")
        assert e.value.status == 5


def test_batch_helmholtz_and_biharmonic_overlap_on_two_streams():
    """The two problems use separate work-queue counters, so their solves may run
    concurrently on two streams; each result equals its serial solve."""
    import torch
    insts = inputs.batch_instances(64, seed=9)
    with BatchPlan(insts) as bp:
        fh = inputs.batch_rhs_torch(bp.offsets, insts, seed=1)
        fb = inputs.batch_rhs_torch(bp.offsets, insts, seed=2)
        ref_h = bp.solve("helmholtz", fh, precision="df")
        ref_b = bp.solve("biharmonic", fb, precision="df")
        torch.cuda.synchronize()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        for _ in range(3):
            uh = torch.empty_like(fh)
            ub = torch.empty_like(fb)
            bp.solve("helmholtz", fh, uh, precision="df", stream=s1)
            bp.solve("biharmonic", fb, ub, precision="df", stream=s2)
            torch.cuda.synchronize()
            assert torch.equal(uh, ref_h)
            assert torch.equal(ub, ref_b)
