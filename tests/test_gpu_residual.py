"""GPU tests of the a posteriori residual check (shen_residual) and the error detail.

The per-mode relative residual ||f - H u|| / ||f|| computed on the GPU is compared
with the same quantity from the oracle's exactly assembled system matrix in numpy
longdouble (a route independent of the library's row tables and float-float
arithmetic), for solved fields and for fields with a planted perturbation.
"""
import numpy as np
import pytest

from oracle import solve as so
from paper_1701_03787_gb300 import Plan, inputs

pytestmark = pytest.mark.gpu


def _oracle_rel(problem, N, z2, c, F, U):
    n = so.n_unknowns(problem, N)
    H = so._system_ld(problem, N, z2, c)
    Ul = U[:n].real.astype(np.longdouble) + 1j * U[:n].imag.astype(np.longdouble)
    r = F[:n] - (H @ Ul.real + 1j * (H @ Ul.imag))
    return float(np.sqrt(np.sum(np.abs(r) ** 2) / np.sum(np.abs(F[:n]) ** 2)))


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_residual_of_solutions_and_of_a_planted_error(problem, precision):
    import torch
    N, Nx, Nz, nu, dt = 96, 10, 8, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=81)
        u = plan.solve(problem, f, precision=precision)
        rel = plan.residual(problem, f, u)
        torch.cuda.synchronize()
        mx, ns = plan.error_detail()
        assert ns == 0
        assert mx == float(rel.max())
        F, U, R = f.cpu().numpy(), u.cpu().numpy(), rel.cpu().numpy()
        # solved fields: tiny residuals that agree with the oracle's to rounding
        assert R.max() < 1e-11
        # resolution of the float-float H u: ~1e-14 of ||f|| (Helmholtz); ~1e-12 for the
        # biharmonic, whose Q tail p_k q_j + r_k s_j cancels between its two terms
        res = 1e-13 if problem == "helmholtz" else 2e-12
        for m in (0, plan.n_modes // 2, plan.n_modes - 1):
            ref = _oracle_rel(problem, N, z2[m], c, F[m], U[m])
            assert abs(R[m] - ref) <= res, (m, R[m], ref)
        # planted error: 1e-6 of mode 3's leading coefficient added to its coefficient 2
        U2 = U.copy()
        U2[3, 2] += 1e-6 * abs(U[3, 0])
        rel2 = plan.residual(problem, f, torch.as_tensor(U2, device="cuda")).cpu().numpy()
        ref = _oracle_rel(problem, N, z2[3], c, F[3], U2[3])
        assert ref > 1e-9
        assert abs(rel2[3] - ref) <= 1e-3 * ref
        assert plan.error_detail()[0] == pytest.approx(rel2.max())


def test_residual_rejects_bad_arguments():
    import torch
    with Plan(64, 8, 8, 1 / 180, 1e-3) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=82)
        with pytest.raises(ValueError):
            plan.residual("helmholtz", f, f, rel=torch.empty(3, dtype=torch.float64, device="cuda"))
        with pytest.raises(KeyError):
            plan.residual("poisson", f, f)
