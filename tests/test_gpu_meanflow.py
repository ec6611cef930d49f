"""GPU tests of the mass-matrix operator (shen_mass_matvec) and of the mean-flow step of
the m = n = 0 mode (Eqs. v00, w00) assembled from the library's entry points.

Eq. v00, scaled like the Helmholtz solve (times 2 / (nu dt)):
    H_h v_new = R_h v_old + (2 / nu) (B_D H_y - S(beta)),  S(beta)_k = (beta, phi_k) = pi beta [k = 0],
at z2 = 0, checked against the oracle's dense matrices."""
import numpy as np
import pytest

from oracle import matrices as mat
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("gl", [False, True])
def test_mass_matvec(problem, gl):
    import torch
    N, Nx, Nz = 45, 6, 4
    with Plan(N, Nx, Nz, 1 / 180, 1e-3, gl=gl) as plan:
        X = inputs.rhs_numpy(plan.n_modes, N, seed=121)
        Y = inputs.rhs_numpy(plan.n_modes, N, seed=122)
        O = plan.mass_matvec(problem, torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"),
                             beta=-2.0).cpu().numpy()
    n = so.n_unknowns(problem, N)
    B = mat.mass_dirichlet(N, gl) if problem == "helmholtz" else mat.mass_biharmonic(N, gl)
    for m in range(plan.n_modes):
        ref = B @ X[m, :n] - 2.0 * Y[m, :n]
        assert so.rel_l2(O[m, :n], ref) <= 1e-13, m
        assert np.all(O[m, n:] == 0)


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_mean_flow_step(precision):
    import torch
    N, nu, dt, beta = 96, 1 / 180, 1e-3, 0.75
    c = so.c_of(nu, dt)
    V_old = inputs.rhs_numpy(1, N, seed=123)
    Hy = inputs.rhs_numpy(1, N, seed=124)
    with Plan(N, z2=np.array([0.0]), nu=nu, dt=dt) as plan:
        v_old, hy = torch.as_tensor(V_old, device="cuda"), torch.as_tensor(Hy, device="cuda")
        load = plan.mass_matvec("helmholtz", hy)                  # B_D H_y
        load[0, 0] -= np.pi * beta                                  # - S(beta): only the k = 0 row
        rhs = plan.rhs_matvec("helmholtz", v_old, load, beta=2.0 / nu, precision=precision)
        v_new = plan.solve("helmholtz", rhs, precision=precision).cpu().numpy()[0]
    n = N - 2
    B, A = mat.mass_dirichlet(N), mat.stiff_dirichlet(N)
    S = np.zeros(n)
    S[0] = np.pi * beta
    rhs_ref = (c * B + A) @ V_old[0, :n] + (2.0 / nu) * (B @ Hy[0, :n] - S)
    v_ref = so.solve_dense(c * B - A, rhs_ref)
    assert so.rel_l2(v_new[:n], v_ref) <= (1e-12 if precision == "fp64" else 1e-10)
