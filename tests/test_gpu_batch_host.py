"""GPU parity of the batched solve on host fields (shen_batch_solve_host).

The host pipeline runs the same persistent kernel as shen_batch_solve on staging slots,
one chunk of whole modes at a time, so its results must equal the device solve's bit for
bit; sampled columns are also checked against the O(N) oracle.  The large case spans
several 256 MB chunks with chunk boundaries inside instances.
"""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import BatchPlan, ShenError, inputs

pytestmark = pytest.mark.gpu


def _pinned(t):
    import torch
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


def _instances_small():
    return [dict(N=8, Nx=2, Nz=2, nu=1e-2, dt=1e-2), dict(N=130, Nx=8, Nz=6, nu=1 / 180, dt=1e-3),
            dict(N=64, Nx=16, Nz=16, nu=1 / 180, dt=1e-3), dict(N=257, Nx=4, Nz=8, nu=1 / 2000, dt=1e-4),
            dict(N=96, Nx=32, Nz=16, nu=1e-4, dt=1e-2, Lx=4.0, Lz=1.5)]


def _instances_large():
    # about 0.87 GB of complex128 field: four 256 MB chunks (a slot reused), ends inside instances
    out = []
    for i in range(48):
        N = (512, 1024, 96, 768)[i % 4]
        out.append(dict(N=N, Nx=64, Nz=48 if N == 1024 else 64, nu=1 / 2000, dt=1e-4 * (1 + i % 3)))
    return out


def _oracle_sample(bp, insts, f, u, problem, tol, seed):
    rng = np.random.default_rng(seed)
    for i in rng.choice(len(insts), size=min(6, len(insts)), replace=False):
        inst = insts[i]
        N = inst["N"]
        fi = f[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N).numpy()
        ui = u[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N).numpy()
        kw = {k: inst[k] for k in ("Lx", "Lz") if k in inst}
        z2 = so.mode_z2(inst["Nx"], inst["Nz"], **kw)
        pick = rng.choice(z2.size, size=min(6, z2.size), replace=False)
        R = on.solve_modes(problem, N, z2[pick], so.c_of(inst["nu"], inst["dt"]), fi[pick])
        n = so.n_unknowns(problem, N)
        for j, m in enumerate(pick):
            assert so.rel_l2(ui[m, :n], R[j, :n]) <= tol, (i, m)
            assert np.all(ui[m, n:] == 0)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_batch_host_equals_device_small(problem, precision):
    import torch
    insts = _instances_small()
    with BatchPlan(insts) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=11)
        ref = bp.solve(problem, f, precision=precision)
        torch.cuda.synchronize()
        hf = _pinned(f.cpu())
        hu = bp.solve_host(problem, hf, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(hu, ref.cpu())
        # in place: u_host == f_host
        hin = _pinned(f.cpu())
        bp.solve_host(problem, hin, hin, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(hin, ref.cpu())
        bp.check_device()
        _oracle_sample(bp, insts, hf, hu, problem, 1e-12 if precision == "fp64" else 1e-10, seed=3)


def test_batch_host_gauss_lobatto():
    """A Gauss-Lobatto batch (SHEN_PLAN_GL): host solve equals the device solve bit for bit."""
    import torch
    insts = _instances_small()
    with BatchPlan(insts, gl=True) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=13)
        for problem in ("helmholtz", "biharmonic"):
            ref = bp.solve(problem, f, precision="df")
            torch.cuda.synchronize()
            hu = bp.solve_host(problem, _pinned(f.cpu()), precision="df")
            torch.cuda.synchronize()
            assert torch.equal(hu, ref.cpu()), problem


def test_batch_host_several_chunks_two_problems_on_two_streams():
    """Both problems through the shared pipeline, issued on two caller streams: each
    result equals its device solve bit for bit; the staging is counted by the plan."""
    import torch
    insts = _instances_large()
    with BatchPlan(insts) as bp:
        assert bp.field_elems * 16 > 3 * (256 << 20)
        fh = inputs.batch_rhs_torch(bp.offsets, insts, seed=21)
        fb = inputs.batch_rhs_torch(bp.offsets, insts, seed=22)
        ref_h = bp.solve("helmholtz", fh, precision="df").cpu()
        ref_b = bp.solve("biharmonic", fb, precision="df").cpu()
        torch.cuda.synchronize()
        bytes0 = bp.info()["device_bytes"]
        hfh, hfb = _pinned(fh.cpu()), _pinned(fb.cpu())
        del fh, fb
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        for _ in range(2):
            huh = torch.empty_like(hfh).pin_memory()
            hub = torch.empty_like(hfb).pin_memory()
            bp.solve_host("helmholtz", hfh, huh, precision="df", stream=s1)
            bp.solve_host("biharmonic", hfb, hub, precision="df", stream=s2)
            torch.cuda.synchronize()
            assert torch.equal(huh, ref_h)
            assert torch.equal(hub, ref_b)
        assert bp.info()["device_bytes"] > bytes0 + 3 * (200 << 20)
        _oracle_sample(bp, insts, hfb, hub, "biharmonic", 1e-10, seed=5)


def test_batch_host_rejects_bad_arguments():
    import torch
    insts = _instances_small()
    with BatchPlan(insts) as bp:
        buf = torch.zeros(bp.field_elems + 1, dtype=torch.complex128).pin_memory()
        f, u = buf[:-1], buf[1:]
        with pytest.raises(ShenError) as e:             # partial overlap
            bp.solve_host("helmholtz", f, u, precision="df")
        assert e.value.status == 1
        with pytest.raises(ShenError) as e:
            bp.solve_host("helmholtz", f, precision="df_r1")
        assert e.value.status == 5
        with pytest.raises(ValueError):
            bp.solve_host("helmholtz", f.cuda(), precision="df")
