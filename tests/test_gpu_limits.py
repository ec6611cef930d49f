"""GPU cases at the size limits of a plan: the largest N (8192, the largest N_x of the
paper's timing table, Table tab:timings) and the smallest (8).

At N = 4096 and 8192 a dense exact oracle is out of reach, so the solves are held to the
paper's O(N) algorithms in the oracle's C code (float64) and the float-float operators to
the float64 ones; at N = 8 every mode is checked against the dense oracle.  Tolerances at
N = 8192: two float64 implementations of the same algorithm differ by their rounding,
which the paper's roundoff table (Table tab:roundoff) puts near 1.5e-11 for the
biharmonic solver at N_x = 4096; the float-float path keeps the reduced-precision bar."""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [4096, 8192])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_largest_N(problem, precision, N):
    import torch
    Nx, Nz, nu, dt = 6, 8, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=101)
        u = plan.solve(problem, f, precision=precision)
        F, U = f.cpu().numpy(), u.cpu().numpy()
        R = on.solve_modes(problem, N, z2, c, F)
        n = so.n_unknowns(problem, N)
        err = max(so.rel_l2(U[m, :n], R[m, :n]) for m in range(plan.n_modes))
        bar = 1e-10 if precision == "df" else (1e-12 if N <= 4096 else 5e-11)
        assert err <= bar, err
        assert np.all(U[:, n:] == 0)
        # float-float operator against the float64 one
        y = inputs.rhs_torch(plan.n_modes, N, seed=102)
        a = plan.rhs_matvec(problem, f, y, beta=0.25, precision="df")
        b = plan.rhs_matvec(problem, f, y, beta=0.25, precision="fp64")
        torch.cuda.synchronize()
        d = torch.linalg.vector_norm(a - b, dim=1) / torch.linalg.vector_norm(b, dim=1)
        assert float(d.max()) < 1e-13


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_smallest_N(problem, precision):
    N, Nx, Nz, nu, dt = 8, 4, 6, 1e-2, 1e-2
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=103)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        import torch
        U = plan.solve(problem, torch.as_tensor(F, device="cuda"), precision=precision).cpu().numpy()
    n = so.n_unknowns(problem, N)
    for m in range(z2.size):
        ref = so.solve_mode(problem, N, z2[m], c, F[m])
        assert so.rel_l2(U[m, :n], ref) <= 1e-12, (m, precision)
        assert np.all(U[m, n:] == 0)
