"""GPU cases at the size limits of a plan: the largest N (8192, the largest N_x of the
paper's timing table, Table tab:timings) and the smallest (8).

At N = 4096 and 8192 the dense exact oracle is out of reach; the reference is the refined
O(N) solution (``oracle.structured.solve_ref``: the paper's O(N) float64 solve refined with
a longdouble residual of the exactly evaluated matrices).  Bars per mode:
  float64 sweeps   within 10x of the same algorithm's own float64 error on the CPU
                   (``shen_on.c`` against the same reference), and <= 1e-12 wherever that
                   error is below 1e-13: the unpivoted algorithm's roundoff grows with N
                   (Table tab:roundoff), and the GPU runs the same algorithm;
  SHEN_FP64_R1     <= 1e-12 (the double-double residual removes that roundoff);
  float-float      <= 1e-10 (the reduced-precision bar).
At N = 8 every mode is checked against the dense oracle."""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from oracle import structured as st
from paper_1701_03787_gb300 import Plan, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [4096, 8192])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_largest_N(problem, N):
    import torch
    Nx, Nz, nu, dt = 6, 8, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=101)
        F = f.cpu().numpy()
        U = {prec: plan.solve(problem, f, precision=prec).cpu().numpy() for prec in ("fp64", "fp64_r1", "df")}
        # float-float operator against the float64 one
        y = inputs.rhs_torch(plan.n_modes, N, seed=102)
        a = plan.rhs_matvec(problem, f, y, beta=0.25, precision="df")
        b = plan.rhs_matvec(problem, f, y, beta=0.25, precision="fp64")
        torch.cuda.synchronize()
        d = torch.linalg.vector_norm(a - b, dim=1) / torch.linalg.vector_norm(b, dim=1)
        assert float(d.max()) < 1e-13
    R = st.solve_ref(problem, N, z2, c, F)
    C = on.solve_modes(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    for m in range(plan.n_modes):
        own = so.rel_l2(C[m, :n], R[m, :n])
        assert so.rel_l2(U["fp64"][m, :n], R[m, :n]) <= max(10 * own, 1e-12), (m, own)
        assert so.rel_l2(U["fp64_r1"][m, :n], R[m, :n]) <= 1e-12, m
        assert so.rel_l2(U["df"][m, :n], R[m, :n]) <= 1e-10, m
    for prec in U:
        assert np.all(U[prec][:, n:] == 0), prec


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
