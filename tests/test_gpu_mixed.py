"""GPU parity of the reduced-precision paths against the oracle.

Bar: relative L2 error per mode column <= 1e-10.
  fp32_r1 / df_r1  float32 sweeps with float64-built factors and one refinement step
                   whose residual is float64 / float-float (Helmholtz)
  df               float-float sweeps (both problems), no refinement
"""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, ShenError, inputs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-10
PROBLEMS = ("helmholtz", "biharmonic")
CASES = [("helmholtz", "fp32_r1"), ("helmholtz", "df_r1"), ("helmholtz", "df"), ("biharmonic", "df")]


@pytest.mark.parametrize("problem,precision", CASES)
@pytest.mark.parametrize("wl", [dict(N=64, Nx=32, Nz=32, nu=1 / 180, dt=1e-3),
                                dict(N=128, Nx=128, Nz=128, nu=1 / 180, dt=5e-4),
                                dict(N=1024, Nx=16, Nz=16, nu=1 / 2000, dt=1e-4)])
def test_mixed_all_modes(problem, precision, wl):
    N = wl["N"]
    c = so.c_of(wl["nu"], wl["dt"])
    z2 = so.mode_z2(wl["Nx"], wl["Nz"])
    F = inputs.rhs_numpy(z2.size, N, seed=11)
    with Plan(N, wl["Nx"], wl["Nz"], wl["nu"], wl["dt"]) as plan:
        U = to_host(plan.solve(problem, to_dev(F), precision=precision))
    R = on.solve_modes(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    errs = np.array([so.rel_l2(U[m, :n], R[m, :n]) for m in range(z2.size)])
    assert errs.max() <= MIXED_TOL, (errs.max(), int(errs.argmax()))
    assert np.all(U[:, n:] == 0)
    for m in inputs.sample_modes(z2.size, 0.01, 5, must_include=[0, int(np.argmax(z2))]):
        r = so.solve_mode_ref(problem, N, float(z2[m]), c, F[m])
        assert so.rel_l2(U[m, :n], r) <= MIXED_TOL


@pytest.mark.parametrize("problem,precision", CASES)
@pytest.mark.parametrize("N", [8, 9, 12, 63, 65, 66, 130, 257, 300, 513, 1000, 1537, 2048])
def test_mixed_ragged_N(problem, precision, N):
    """Chains that do not fill the lanes evenly; N up to the largest supported size."""
    nu, dt = 1 / 2000, 5e-5
    c = so.c_of(nu, dt)
    z2 = np.array([0.0, 1.0, 4.0, 1846.0 ** 2, 300.0 ** 2])
    F = inputs.rhs_numpy(z2.size, N, seed=N)
    n = so.n_unknowns(problem, N)
    with Plan(N, z2=z2, nu=nu, dt=dt) as plan:
        U = to_host(plan.solve(problem, to_dev(F), precision=precision))
    for m in range(z2.size):
        r = so.solve_mode_ref(problem, N, float(z2[m]), c, F[m])
        assert so.rel_l2(U[m, :n], r) <= MIXED_TOL, (m, so.rel_l2(U[m, :n], r))
        assert np.all(U[m, n:] == 0)


@pytest.mark.parametrize("problem,precision", CASES)
def test_mixed_in_place_and_shards(problem, precision):
    N, Nx, Nz = 256, 16, 16
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=3)
    with Plan(N, Nx, Nz, 1 / 1000, 1e-3) as plan:
        full = to_host(plan.solve(problem, to_dev(F), precision=precision))
        f = to_dev(F)
        plan.solve(problem, f, u=f, precision=precision)
        assert np.array_equal(to_host(f), full)
        f = to_dev(F)
        part = to_host(plan.solve_modes(problem, 17, f[17:50].contiguous(), precision=precision))
        assert np.array_equal(part, full[17:50])


def test_unsupported_combinations_report_status():
    import torch
    with Plan(64, 8, 8, 1e-2, 1e-3) as plan:
        f = torch.zeros((plan.n_modes, 64), dtype=torch.complex128, device="cuda")
        for problem, prec in (("helmholtz", "fp32_r2"), ("helmholtz", "df_r2"), ("biharmonic", "fp32_r1"),
                              ("biharmonic", "df_r1"), ("biharmonic", "df_r2")):
            with pytest.raises(ShenError) as e:
                plan.solve(problem, f, precision=prec)
            assert e.value.status == 5


@pytest.mark.parametrize("problem", PROBLEMS)
def test_df_full_size_sampled(problem):
    """N=1024, 1024 x 1024 grid (525,312 modes), nu=1/2000, dt=1e-4, the launch the
    benchmark times: sampled columns (mean, Nyquists, max z2, random) vs the refined
    reference, and a 0.2 % sample vs the O(N) oracle."""
    import torch
    N, Nx, Nz, nu, dt = 1024, 1024, 1024, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=41)
        u = plan.solve(problem, f, precision="df")
        torch.cuda.synchronize()
        special = list(inputs.grid_modes(Nx, Nz).values()) + [int(np.argmax(z2))]
        sample = inputs.sample_modes(z2.size, 0.002, 17, must_include=special)
        idx = torch.as_tensor(sample, device="cuda")
        F = f[idx].cpu().numpy()
        U = u[idx].cpu().numpy()
        del f, u
    n = so.n_unknowns(problem, N)
    R = on.solve_modes(problem, N, z2[sample], c, F)
    for i, m in enumerate(sample):
        assert so.rel_l2(U[i, :n], R[i, :n]) <= MIXED_TOL, m
        assert np.all(U[i, n:] == 0)
    for i, m in enumerate(sample[:: max(1, len(sample) // 12)] + special[-1:]):
        j = sample.index(m)
        r = so.solve_mode_ref(problem, N, float(z2[m]), c, F[j])
        assert so.rel_l2(U[j, :n], r) <= MIXED_TOL, m
