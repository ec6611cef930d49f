"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by element.

Tolerances (relative L2 per mode column, complex):
  float64 path: 1e-12 against the O(N) C oracle and the dense / refined definitions.
The solves are exact algorithms (Sec. 4); differences are rounding only.
"""
import math

import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, ShenError, inputs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
PROBLEMS = ("helmholtz", "biharmonic")


def _check_columns(U, F, problem, N, z2, c, modes, tol, ref="dense"):
    n = so.n_unknowns(problem, N)
    worst = 0.0
    for m in modes:
        if ref == "refined":
            r = so.solve_mode_ref(problem, N, float(z2[m]), c, F[m])
        else:
            r = so.solve_mode(problem, N, float(z2[m]), c, F[m])
        e = so.rel_l2(U[m, :n], r)
        worst = max(worst, e)
        assert e <= tol, (problem, m, e)
        assert np.all(U[m, n:] == 0), (problem, m)
    return worst


@pytest.mark.parametrize("problem", PROBLEMS)
def test_config_small_all_modes(problem):
    """N=64, 32x32 grid (544 modes), nu=1/180, dt=1e-3: every mode vs the O(N) oracle and a
    sample vs dense LU."""
    N, Nx, Nz, nu, dt = 64, 32, 32, 1 / 180, 1e-3
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=1)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        assert plan.n_modes == 544
        U = to_host(plan.solve(problem, to_dev(F), precision="fp64"))
    R = on.solve_modes(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    for m in range(z2.size):
        assert so.rel_l2(U[m, :n], R[m, :n]) <= FP64_TOL, m
    sample = inputs.sample_modes(z2.size, 0.05, 1, must_include=inputs.grid_modes(Nx, Nz).values())
    _check_columns(U, F, problem, N, z2, c, sample, FP64_TOL)


@pytest.mark.parametrize("problem", PROBLEMS)
def test_config_re_tau_180(problem):
    """N=128, 128x128 grid (8320 modes), nu=1/180, dt=5e-4: every mode vs the O(N) oracle and a
    sample (incl. mean, Nyquists, max z2) vs the refined reference."""
    N, Nx, Nz, nu, dt = 128, 128, 128, 1 / 180, 5e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=2)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        U = to_host(plan.solve(problem, to_dev(F), precision="fp64"))
    R = on.solve_modes(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    errs = [so.rel_l2(U[m, :n], R[m, :n]) for m in range(z2.size)]
    assert max(errs) <= FP64_TOL
    sample = inputs.sample_modes(z2.size, 0.003, 2, must_include=list(inputs.grid_modes(Nx, Nz).values())
                                 + [int(np.argmax(z2))])
    _check_columns(U, F, problem, N, z2, c, sample, FP64_TOL, ref="refined")


@pytest.mark.parametrize("N", [8, 9, 10, 11, 33, 65, 130])
@pytest.mark.parametrize("problem", PROBLEMS)
def test_small_and_odd_N(N, problem):
    """Ragged chain lengths: odd and even N, the minimum N = 8, tiny grid."""
    Nx, Nz, nu, dt = 4, 6, 1e-2, 1e-2
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=N)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        U = to_host(plan.solve(problem, to_dev(F)))
    _check_columns(U, F, problem, N, z2, c, range(z2.size), FP64_TOL, ref="refined")


@pytest.mark.parametrize("problem", PROBLEMS)
def test_in_place_and_shards(problem):
    N, Nx, Nz, nu, dt = 96, 16, 16, 1 / 500, 2e-3
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=5)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        full = to_host(plan.solve(problem, to_dev(F)))
        f = to_dev(F)
        plan.solve(problem, f, u=f)                       # in place
        assert np.array_equal(to_host(f), full)
        f = to_dev(F)
        parts = []
        for m0, m1 in ((0, 1), (1, 40), (40, 40), (40, z2.size)):
            if m1 > m0:
                parts.append(to_host(plan.solve_modes(problem, m0, f[m0:m1].contiguous())))
        assert np.array_equal(np.concatenate(parts), full)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem", PROBLEMS)
@pytest.mark.parametrize("N,Nx,Nz,nu,dt", [(64, 16, 16, 1 / 180, 1e-3), (257, 12, 10, 1 / 2000, 1e-4),
                                          (9, 4, 4, 1e-2, 1e-2)])
def test_rhs_matvec(problem, precision, N, Nx, Nz, nu, dt):
    """out = R x + beta y against the dense right-hand-side operators of Eqs. gfin / ufin,
    in float64 and float-float arithmetic (inputs beyond the unknowns are ignored)."""
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    X = inputs.rhs_numpy(z2.size, N, seed=6)
    Y = inputs.rhs_numpy(z2.size, N, seed=7)
    n = so.n_unknowns(problem, N)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        O1 = to_host(plan.rhs_matvec(problem, to_dev(X), precision=precision))
        O2 = to_host(plan.rhs_matvec(problem, to_dev(X), to_dev(Y), beta=-0.75, precision=precision))
    for m in range(z2.size):
        r1 = so.matvec_mode(problem, N, z2[m], c, X[m])
        r2 = so.matvec_mode(problem, N, z2[m], c, X[m], Y[m], -0.75)
        assert so.rel_l2(O1[m, :n], r1) <= 1e-13, m
        assert so.rel_l2(O2[m, :n], r2) <= 1e-13, m
        assert np.all(O1[m, n:] == 0)


@pytest.mark.parametrize("problem", PROBLEMS)
def test_rhs_matvec_df_full_size_sampled(problem):
    """Float-float operator at N = 1024 against the float64 operator (all modes) and the
    dense oracle operator (sampled modes, including the largest z2)."""
    import torch
    N, Nx, Nz, nu, dt = 1024, 64, 64, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    n = so.n_unknowns(problem, N)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        x = inputs.rhs_torch(plan.n_modes, N, seed=71)
        y = inputs.rhs_torch(plan.n_modes, N, seed=72)
        a = plan.rhs_matvec(problem, x, y, beta=0.5, precision="df")
        b = plan.rhs_matvec(problem, x, y, beta=0.5, precision="fp64")
        torch.cuda.synchronize()
        d = torch.linalg.vector_norm(a - b, dim=1) / torch.linalg.vector_norm(b, dim=1)
        assert float(d.max()) < 1e-13
        modes = sorted({0, int(np.argmax(z2)), plan.n_modes // 3, plan.n_modes - 1})
        A, X, Y = a[modes].cpu().numpy(), x[modes].cpu().numpy(), y[modes].cpu().numpy()
    for i, m in enumerate(modes):
        r = so.matvec_mode(problem, N, z2[m], c, X[i], Y[i], 0.5)
        assert so.rel_l2(A[i, :n], r) <= 1e-13, m


@pytest.mark.parametrize("problem", PROBLEMS)
def test_explicit_z2_plan_and_extremes(problem):
    """shen_plan_create_z2 with repeated, zero and very large z2 (3 modes share one class).

    The parameters are those of the Sec. 5 roundoff study (nu = 1/5200, dt = 1e-5, z up to
    5400), where the unpivoted O(N) algorithm itself loses accuracy: its roundoff there is
    of order 1e-11 (Table tab:roundoff), so this case is held to 2e-11."""
    N, nu, dt = 128, 1 / 5200, 1e-5
    c = so.c_of(nu, dt)
    z2 = np.array([0.0, 5400.0 ** 2, 1.0, 1800.0 ** 2, 1.0, 1.0, 200.0 ** 2])
    F = inputs.rhs_numpy(z2.size, N, seed=9)
    with Plan(N, z2=z2, nu=nu, dt=dt) as plan:
        assert plan.n_classes == 5
        U = to_host(plan.solve(problem, to_dev(F)))
    _check_columns(U, F, problem, N, z2, c, range(z2.size), 2e-11, ref="refined")


def test_error_statuses():
    import torch
    N, Nx, Nz = 64, 8, 8
    with Plan(N, Nx, Nz, 1e-2, 1e-3) as plan:
        f = torch.zeros((plan.n_modes, N), dtype=torch.complex128, device="cuda")
        u = torch.zeros_like(f)
        with pytest.raises(ShenError) as e:
            plan.helmholtz_solve(f, u, precision=99)
        assert e.value.status == 1
        big = torch.zeros(plan.n_modes * N + 1, dtype=torch.complex128, device="cuda")
        with pytest.raises(ShenError) as e:                 # input and output overlap partially
            plan.helmholtz_solve(big[:-1].view(plan.n_modes, N), big[1:].view(plan.n_modes, N))
        assert e.value.status == 1
        raw = torch.zeros(2 * plan.n_modes * N + 1, dtype=torch.float64, device="cuda")
        from paper_1701_03787_gb300 import binding
        st = binding.lib().shen_helmholtz_solve(plan.handle, binding._ptr(raw.data_ptr() + 8),
                                                binding._ptr(u), 0, None)
        assert st == 1                                       # misaligned
        with pytest.raises(ShenError) as e:
            plan.rhs_matvec("helmholtz", f, out=f)           # out aliases x
        assert e.value.status == 1
        plan.check_device()


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_df_only_plan_gives_the_same_bits_with_less_memory(problem):
    """A SHEN_PLAN_DF_ONLY plan keeps only the float-float factors: same float-float
    result bit for bit, about half the device memory, other precisions unsupported."""
    import torch
    from paper_1701_03787_gb300 import Plan, ShenError, inputs
    with Plan(300, 24, 20, 1 / 2000, 1e-4) as full, Plan(300, 24, 20, 1 / 2000, 1e-4, df_only=True) as lean:
        f = inputs.rhs_torch(full.n_modes, full.N, seed=61)
        a = full.solve(problem, f, precision="df")
        b = lean.solve(problem, f, precision="df")
        c = lean.solve(problem, f, precision="auto")
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(a, c)
        assert lean.info()[3] < 0.7 * full.info()[3]      # float64 factors and float32 tables gone
        for prec in ("fp64", "df_r1", "fp32_r1"):
            with pytest.raises(ShenError) as e:
                lean.solve(problem, f, precision=prec)
            assert e.value.status == 5
        name, _ = lean.autotune(problem, f)
        assert name == "df"
