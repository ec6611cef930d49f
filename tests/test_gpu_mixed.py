"""GPU parity of the float32-sweep + refinement paths against the oracle.

Bar: relative L2 error per mode column <= 1e-10 after refinement (float32 sweeps
with float64-built factors, one refinement step whose residual is float64
(fp32_r1) or float-float (df_r1)).
"""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, ShenError, inputs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-10
HELM_PRECISIONS = ("fp32_r1", "df_r1")


@pytest.mark.parametrize("precision", HELM_PRECISIONS)
@pytest.mark.parametrize("wl", [dict(N=64, Nx=32, Nz=32, nu=1 / 180, dt=1e-3),
                                dict(N=128, Nx=128, Nz=128, nu=1 / 180, dt=5e-4),
                                dict(N=1024, Nx=16, Nz=16, nu=1 / 2000, dt=1e-4)])
def test_helmholtz_mixed_all_modes(precision, wl):
    N = wl["N"]
    c = so.c_of(wl["nu"], wl["dt"])
    z2 = so.mode_z2(wl["Nx"], wl["Nz"])
    F = inputs.rhs_numpy(z2.size, N, seed=11)
    with Plan(N, wl["Nx"], wl["Nz"], wl["nu"], wl["dt"]) as plan:
        U = to_host(plan.helmholtz_solve(to_dev(F), precision=precision))
    R = on.solve_modes("helmholtz", N, z2, c, F)
    n = N - 2
    errs = np.array([so.rel_l2(U[m, :n], R[m, :n]) for m in range(z2.size)])
    assert errs.max() <= MIXED_TOL, (errs.max(), int(errs.argmax()))
    assert np.all(U[:, n:] == 0)
    for m in inputs.sample_modes(z2.size, 0.01, 5, must_include=[0, int(np.argmax(z2))]):
        r = so.solve_mode_ref("helmholtz", N, float(z2[m]), c, F[m])
        assert so.rel_l2(U[m, :n], r) <= MIXED_TOL


@pytest.mark.parametrize("precision", HELM_PRECISIONS)
@pytest.mark.parametrize("N", [8, 9, 63, 65, 66, 130, 257, 1000, 1537, 2048])
def test_helmholtz_mixed_ragged_N(precision, N):
    """Chains that do not fill the lanes evenly; N up to the largest supported size."""
    nu, dt = 1 / 2000, 5e-5
    c = so.c_of(nu, dt)
    z2 = np.array([0.0, 1.0, 4.0, 1846.0 ** 2, 300.0 ** 2])
    F = inputs.rhs_numpy(z2.size, N, seed=N)
    with Plan(N, z2=z2, nu=nu, dt=dt) as plan:
        U = to_host(plan.helmholtz_solve(to_dev(F), precision=precision))
    for m in range(z2.size):
        r = so.solve_mode_ref("helmholtz", N, float(z2[m]), c, F[m])
        assert so.rel_l2(U[m, :N - 2], r) <= MIXED_TOL, (m, so.rel_l2(U[m, :N - 2], r))
        assert np.all(U[m, N - 2:] == 0)


@pytest.mark.parametrize("precision", HELM_PRECISIONS)
def test_helmholtz_mixed_in_place_and_shards(precision):
    N, Nx, Nz = 256, 16, 16
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=3)
    with Plan(N, Nx, Nz, 1 / 1000, 1e-3) as plan:
        full = to_host(plan.helmholtz_solve(to_dev(F), precision=precision))
        f = to_dev(F)
        plan.helmholtz_solve(f, u=f, precision=precision)
        assert np.array_equal(to_host(f), full)
        f = to_dev(F)
        part = to_host(plan.solve_modes("helmholtz", 17, f[17:50].contiguous(), precision=precision))
        assert np.array_equal(part, full[17:50])


def test_unsupported_combinations_report_status():
    import torch
    with Plan(64, 8, 8, 1e-2, 1e-3) as plan:
        f = torch.zeros((plan.n_modes, 64), dtype=torch.complex128, device="cuda")
        for prec in ("fp32_r2", "df_r2"):
            with pytest.raises(ShenError) as e:
                plan.helmholtz_solve(f, precision=prec)
            assert e.value.status == 5
