"""GPU tests of the wall-index-first field layout (SHEN_PLAN_WALL_FIRST, the paper's
uhat(l, m, n) order of Sec. 2): element (m, k) at k * n_modes + m.  Each chain runs the
same arithmetic as in the mode-major layout, so the solution is the transpose of the
mode-major one bit for bit; that solution is itself pinned to the oracle elsewhere, and
here again on a sample."""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, ShenError, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,Nx,Nz", [(8, 4, 6), (33, 12, 10), (130, 16, 16), (1024, 64, 64)])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_wall_first_is_transpose_of_mode_major(N, Nx, Nz, problem, precision):
    import torch
    nu, dt = 1 / 2000, 1e-4
    with Plan(N, Nx, Nz, nu, dt) as pm, Plan(N, Nx, Nz, nu, dt, wall_first=True) as pw:
        f = inputs.rhs_torch(pm.n_modes, N, seed=N + 1)
        u = pm.solve(problem, f, precision=precision)
        ft = f.t().contiguous()                              # (N, n_modes): row k holds every mode
        ut = pw.solve(problem, ft, precision=precision)
        gt = ft.clone()
        pw.solve(problem, gt, u=gt, precision=precision)    # in place
        torch.cuda.synchronize()
        assert torch.equal(ut.t(), u)
        assert torch.equal(gt, ut)
        z2 = so.mode_z2(Nx, Nz)
        modes = sorted({0, 1, pm.n_modes // 2, int(z2.argmax()), pm.n_modes - 1})
        R = on.solve_modes(problem, N, z2[modes], so.c_of(nu, dt), f[modes].cpu().numpy())
        U = ut.t()[modes].cpu().numpy()
        n = so.n_unknowns(problem, N)
        tol = 1e-12 if precision == "fp64" else 1e-10
        assert max(so.rel_l2(U[i, :n], R[i, :n]) for i in range(len(modes))) <= tol
        assert torch.all(ut[n:] == 0)


def test_wall_first_auto_and_unsupported_entry_points():
    import torch
    N = 64
    with Plan(N, 8, 8, 1 / 180, 1e-3, wall_first=True) as pw:
        f = inputs.rhs_torch(pw.n_modes, N, seed=5).t().contiguous()
        name, ms = pw.autotune("biharmonic", f)
        assert name in ("fp64", "df")
        pw.solve("biharmonic", f, precision="auto")
        for call in (lambda: pw.rhs_matvec("helmholtz", f), lambda: pw.transform("inverse", "dirichlet", f),
                     lambda: pw.velocity(f, f), lambda: pw.residual("helmholtz", f, f),
                     lambda: pw.solve("helmholtz", f, precision="df_r1")):
            with pytest.raises(ShenError) as e:
                call()
            assert e.value.status == 5
        torch.cuda.synchronize()
