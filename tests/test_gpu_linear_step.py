"""GPU test of the linear step (shen_linear_step) against the oracle, which takes the
paper's unscaled Eqs. ufin and gfin as printed (Hchk u_new = (2 Achk - 2 z2 Bchk - Hchk)
u_old + dt S(h_v), Hbar g_new = (2 Bbar - Hbar) g_old + dt S(h_g)) and then recovers
f, v, w (Eqs. ffin with the sign of Eq. f, f3, g3)."""
import numpy as np
import pytest

from oracle import matrices as mat
from oracle import solve as so
from oracle import velocity as vel
from paper_1701_03787_gb300 import Plan, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("df", 1e-10), ("auto", 1e-10)])
def test_linear_step_matches_the_paper_equations(precision, tol):
    import torch
    N, Nx, Nz, nu, dt = 48, 6, 4, 1 / 180, 1e-3
    z2s = so.mode_z2(Nx, Nz)
    m_, n_ = vel.mode_mn(Nx, Nz)
    nm = z2s.size
    Uo, Go = inputs.rhs_numpy(nm, N, 131), inputs.rhs_numpy(nm, N, 132)
    Lu, Lg = inputs.rhs_numpy(nm, N, 133), inputs.rhs_numpy(nm, N, 134)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        dev = [torch.as_tensor(a, device="cuda") for a in (Uo, Go, Lu, Lg)]
        un, gn, v, w = [t.cpu().numpy() for t in plan.linear_step(*dev, precision=precision)]
    nb, nd = N - 4, N - 2
    for k in range(nm):
        z2 = z2s[k]
        rhs_u = mat.paper_biharmonic_rhs(N, z2, nu, dt) @ Uo[k, :nb] + dt * Lu[k, :nb]
        u_ref = so.solve_dense(mat.paper_biharmonic(N, z2, nu, dt), rhs_u)
        rhs_g = mat.paper_helmholtz_rhs(N, z2, nu, dt) @ Go[k, :nd] + dt * Lg[k, :nd]
        g_ref = so.solve_dense(mat.paper_helmholtz(N, z2, nu, dt), rhs_g)
        assert so.rel_l2(un[k, :nb], u_ref) <= tol, ("u", k)
        assert so.rel_l2(gn[k, :nd], g_ref) <= tol, ("g", k)
        if z2 > 0:
            U = np.zeros(N, dtype=complex)
            U[:nb] = u_ref
            G = np.zeros(N, dtype=complex)
            G[:nd] = g_ref
            v_ref, w_ref = vel.velocity_from_fg(vel.f_from_u(N, U), G, m_[k], n_[k])
            assert so.rel_l2(v[k, :nd], v_ref[:nd]) <= tol, ("v", k)
            assert so.rel_l2(w[k, :nd], w_ref[:nd]) <= tol, ("w", k)
        else:
            assert np.all(v[k] == 0) and np.all(w[k] == 0)          # mean mode left as passed


def test_linear_step_rejects_aliasing():
    import torch
    from paper_1701_03787_gb300 import ShenError
    with Plan(32, 4, 4, 1 / 180, 1e-3) as plan:
        a = inputs.rhs_torch(plan.n_modes, plan.N, seed=135)
        b = inputs.rhs_torch(plan.n_modes, plan.N, seed=136)
        outs = tuple(torch.empty_like(a) for _ in range(4))
        with pytest.raises(ShenError):
            plan.linear_step(a, b, out=(a,) + outs[1:])
        with pytest.raises(ShenError):
            plan.linear_step(a, b, out=(outs[0], outs[0]) + outs[2:])


@pytest.mark.parametrize("with_loads", [True, False])
def test_step_at_n1024(with_loads):
    """The float-float step (float-float operators and solves) against the float64 one on
    N = 1024, 64 x 64 modes (z up to ~72), with and without loads, and the unscaled paper
    equations on a few modes."""
    import torch
    N, Nx, Nz, nu, dt = 1024, 64, 64, 1 / 2000, 1e-4
    z2s = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        dev = [inputs.rhs_torch(plan.n_modes, N, seed=s) for s in (141, 142, 143, 144)]
        if not with_loads:
            dev[2] = dev[3] = None
        fused = [t.cpu().numpy() for t in plan.linear_step(*dev, precision="df")]
        ref = [t.cpu().numpy() for t in plan.linear_step(*dev, precision="fp64")]
        Uo, Go = dev[0].cpu().numpy(), dev[1].cpu().numpy()
        Lu = dev[2].cpu().numpy() if with_loads else np.zeros_like(Uo)
        Lg = dev[3].cpu().numpy() if with_loads else np.zeros_like(Go)
    nb, nd = N - 4, N - 2
    for a, b, n in zip(fused, ref, (nb, nd, nd, nd)):
        assert np.all(a[:, n:] == 0)
        for k in range(plan.n_modes):
            if np.any(b[k]):
                assert so.rel_l2(a[k, :n], b[k, :n]) <= 1e-10, k
    for k in (1, plan.n_modes // 2, int(z2s.argmax())):
        z2 = z2s[k]
        rhs_u = mat.paper_biharmonic_rhs(N, z2, nu, dt) @ Uo[k, :nb] + dt * Lu[k, :nb]
        u_ref = so.solve_dense(mat.paper_biharmonic(N, z2, nu, dt), rhs_u)
        rhs_g = mat.paper_helmholtz_rhs(N, z2, nu, dt) @ Go[k, :nd] + dt * Lg[k, :nd]
        g_ref = so.solve_dense(mat.paper_helmholtz(N, z2, nu, dt), rhs_g)
        assert so.rel_l2(fused[0][k, :nb], u_ref) <= 1e-10, k
        assert so.rel_l2(fused[1][k, :nd], g_ref) <= 1e-10, k
