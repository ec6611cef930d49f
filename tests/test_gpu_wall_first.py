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
        for call in (lambda: pw.solve("helmholtz", f, precision="df_r1"),
                     lambda: pw.solve("helmholtz", f, precision="fp64_r1"),
                     lambda: pw.solve_refine("helmholtz", f)):
            with pytest.raises(ShenError) as e:
                call()
            assert e.value.status == 5
        torch.cuda.synchronize()


@pytest.mark.parametrize("N,Nx,Nz", [(16, 4, 6), (128, 16, 12), (1024, 32, 32)])
def test_wall_first_operators_velocity_transforms(N, Nx, Nz):
    """Every other entry point on a wall-first plan gives the transpose of the mode-major
    result bit for bit: the operators (float64 and float-float), the mass operator, the
    residual, the velocity recovery, the linear step and every transform (whole field and a
    mode range)."""
    import ctypes
    import torch
    from paper_1701_03787_gb300 import binding
    nu, dt = 1 / 2000, 1e-4
    T = lambda t: t.t().contiguous()
    with Plan(N, Nx, Nz, nu, dt) as pm, Plan(N, Nx, Nz, nu, dt, wall_first=True) as pw:
        x = inputs.rhs_torch(pm.n_modes, N, seed=N + 11)
        y = inputs.rhs_torch(pm.n_modes, N, seed=N + 12)
        for problem in ("helmholtz", "biharmonic"):
            for prec in ("fp64", "df"):
                a = pm.rhs_matvec(problem, x, y, beta=0.5, precision=prec)
                b = pw.rhs_matvec(problem, T(x), T(y), beta=0.5, precision=prec)
                assert torch.equal(T(b), a), (problem, prec)
            assert torch.equal(T(pw.mass_matvec(problem, T(x), T(y), 0.25)), pm.mass_matvec(problem, x, y, 0.25))
            u = pm.solve(problem, x, precision="df")
            assert torch.equal(pw.residual(problem, T(x), T(u)), pm.residual(problem, x, u))
        um, gm = pm.solve("biharmonic", x, precision="df"), pm.solve("helmholtz", y, precision="df")
        fm = torch.zeros_like(x)
        vm, wm = pm.velocity(um, gm, f=fm)
        fw = torch.zeros_like(T(x))
        vw, ww = pw.velocity(T(um), T(gm), f=fw)
        assert torch.equal(T(vw), vm) and torch.equal(T(ww), wm) and torch.equal(T(fw), fm)
        sm = pm.linear_step(x, y, um, gm, precision="df")
        sw = pw.linear_step(T(x), T(y), T(um), T(gm), precision="df")
        for a, b in zip(sm, sw):
            assert torch.equal(T(b), a)
        L = binding.lib()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for kind in ("inverse", "scalar", "forward"):
            for space in ("chebyshev", "dirichlet", "biharmonic"):
                src = x if kind == "inverse" else pm.transform("inverse", "chebyshev", x)
                a = pm.transform(kind, space, src)
                b = pw.transform(kind, space, T(src))
                assert torch.equal(T(b), a), (kind, space)
                g = T(src)
                pw.transform(kind, space, g, out=g)                       # in place
                assert torch.equal(T(g), a), (kind, space)
                # a mode range: pointers at element (mode_begin, 0) of the full wall-first field
                m0, cnt = 3, pm.n_modes - 5
                wsrc, wout = T(src), torch.zeros_like(T(src))
                st = L.shen_transform_modes(pw._h, binding.TRANSFORMS[kind], binding.SPACES[space], m0, cnt,
                                            ctypes.c_void_p(wsrc.data_ptr() + 16 * m0),
                                            ctypes.c_void_p(wout.data_ptr() + 16 * m0), stream)
                assert st == 0, binding.status_string(st)
                torch.cuda.synchronize()
                assert torch.equal(T(wout)[m0:m0 + cnt], a[m0:m0 + cnt]), (kind, space)
