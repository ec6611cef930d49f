"""GPU parity of plans on Chebyshev-Gauss-Lobatto points (SHEN_PLAN_GL) against the GL
oracle: solves (float64, float-float, float32 + refinement), the right-hand-side
operators, the velocity recovery, and batched GL plans against single GL plans."""
import math

import numpy as np
import pytest

from oracle import solve as so
from oracle import velocity as vel
from paper_1701_03787_gb300 import BatchPlan, Plan, inputs

pytestmark = pytest.mark.gpu

CASES = [("helmholtz", "fp64"), ("helmholtz", "df"), ("helmholtz", "df_r1"), ("biharmonic", "fp64"),
         ("biharmonic", "df")]


@pytest.mark.parametrize("problem,precision", CASES)
@pytest.mark.parametrize("N", [40, 129])
def test_gl_solves_match_the_gl_oracle(problem, precision, N):
    import torch
    Nx, Nz, nu, dt = 8, 6, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    F = inputs.rhs_numpy(z2.size, N, seed=111)
    with Plan(N, Nx, Nz, nu, dt, gl=True) as gl, Plan(N, Nx, Nz, nu, dt) as gc:
        f = torch.as_tensor(F, device="cuda")
        U = gl.solve(problem, f, precision=precision).cpu().numpy()
        Ugc = gc.solve(problem, f, precision=precision).cpu().numpy()
    n = so.n_unknowns(problem, N)
    tol = 1e-12 if precision == "fp64" else 1e-10
    for m in range(z2.size):
        ref = so.solve_mode(problem, N, z2[m], c, F[m], gl=True)
        assert so.rel_l2(U[m, :n], ref) <= tol, m
    # the two point sets give measurably different (Galerkin) solutions
    assert max(so.rel_l2(U[m, :n], Ugc[m, :n]) for m in range(z2.size)) > 1e-8


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_gl_rhs_matvec(problem, precision):
    N, Nx, Nz, nu, dt = 65, 6, 6, 1 / 180, 1e-3
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    X = inputs.rhs_numpy(z2.size, N, seed=112)
    Y = inputs.rhs_numpy(z2.size, N, seed=113)
    with Plan(N, Nx, Nz, nu, dt, gl=True) as plan:
        import torch
        O = plan.rhs_matvec(problem, torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"),
                            beta=0.5, precision=precision).cpu().numpy()
    n = so.n_unknowns(problem, N)
    for m in range(z2.size):
        ref = so.matvec_mode(problem, N, z2[m], c, X[m], Y[m], 0.5, gl=True)
        assert so.rel_l2(O[m, :n], ref) <= 1e-13, m


def test_gl_velocity():
    import torch
    N, Nx, Nz = 48, 6, 8
    rng = np.random.default_rng(114)
    nm = (Nx // 2 + 1) * Nz
    U = (rng.standard_normal((nm, N)) + 1j * rng.standard_normal((nm, N))) * inputs.spectrum(N)
    G = (rng.standard_normal((nm, N)) + 1j * rng.standard_normal((nm, N))) * inputs.spectrum(N)
    with Plan(N, Nx, Nz, 1 / 2000, 1e-4, gl=True) as plan:
        v, w = plan.velocity(torch.as_tensor(U, device="cuda"), torch.as_tensor(G, device="cuda"))
        V, W = v.cpu().numpy(), w.cpu().numpy()
    m, n = vel.mode_mn(Nx, Nz, 2 * math.pi, math.pi)
    Vr, Wr = vel.velocity_from_fg(vel.f_from_u(N, U, gl=True), G, m, n)
    for k in range(1, nm):
        assert so.rel_l2(V[k, : N - 2], Vr[k, : N - 2]) <= 1e-12
        assert so.rel_l2(W[k, : N - 2], Wr[k, : N - 2]) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_gl_batch_matches_single_gl_plans(precision):
    import torch
    insts = [dict(N=64, Nx=8, Nz=6, nu=1e-3, dt=1e-3), dict(N=33, Nx=4, Nz=4, nu=1 / 180, dt=1e-3),
             dict(N=130, Nx=6, Nz=8, nu=1e-4, dt=5e-3)]
    with BatchPlan(insts, gl=True) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=115)
        for problem in ("helmholtz", "biharmonic"):
            u = bp.solve(problem, f, precision=precision)
            for i, d in enumerate(insts):
                with Plan(d["N"], d["Nx"], d["Nz"], d["nu"], d["dt"], gl=True) as p1:
                    fi = f[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, d["N"]).contiguous()
                    ui = p1.solve(problem, fi, precision=precision)
                    torch.cuda.synchronize()
                    assert torch.equal(u[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, d["N"]), ui)
