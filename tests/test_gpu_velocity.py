"""GPU parity of the velocity recovery (shen_velocity) against the oracle: f = -du/dx
projected on the Dirichlet space (B_D f = -C u) and (v, w) from Eqs. f3, g3."""
import math

import numpy as np
import pytest

from oracle import solve as so
from oracle import velocity as vel
from paper_1701_03787_gb300 import Plan, ShenError, inputs

pytestmark = pytest.mark.gpu


def _fields(n_modes, N, seed):
    rng = np.random.default_rng(seed)
    w_ = inputs.spectrum(N)
    U = (rng.standard_normal((n_modes, N)) + 1j * rng.standard_normal((n_modes, N))) * w_
    G = (rng.standard_normal((n_modes, N)) + 1j * rng.standard_normal((n_modes, N))) * w_
    return U, G                                  # trailing entries nonzero: must be ignored


@pytest.mark.parametrize("N,Nx,Nz,Lx,Lz", [(40, 10, 8, 2 * math.pi, math.pi), (129, 12, 10, 4.0, 1.5),
                                          (8, 4, 4, 2 * math.pi, math.pi)])
def test_velocity_matches_oracle(N, Nx, Nz, Lx, Lz):
    import torch
    U, G = _fields((Nx // 2 + 1) * Nz, N, seed=N)
    m, n = vel.mode_mn(Nx, Nz, Lx, Lz)
    F_ref = vel.f_from_u(N, U)
    V_ref, W_ref = vel.velocity_from_fg(F_ref, G, m, n)
    with Plan(N, Nx, Nz, 1 / 2000, 1e-4, Lx=Lx, Lz=Lz) as plan:
        u, g = torch.as_tensor(U, device="cuda"), torch.as_tensor(G, device="cuda")
        v = torch.full_like(u, 7.0)
        w = torch.full_like(u, -3.0)
        f = torch.empty_like(u)
        plan.velocity(u, g, v, w, f)
        V, W, F = v.cpu().numpy(), w.cpu().numpy(), f.cpu().numpy()
    n_d = N - 2
    assert np.all(V[0] == 7.0) and np.all(W[0] == -3.0)       # mode (0, 0) untouched
    for k in range(1, plan.n_modes):
        assert so.rel_l2(F[k, :n_d], F_ref[k, :n_d]) <= 1e-12, k
        assert so.rel_l2(V[k, :n_d], V_ref[k, :n_d]) <= 1e-12, k
        assert so.rel_l2(W[k, :n_d], W_ref[k, :n_d]) <= 1e-12, k
        assert np.all(V[k, n_d:] == 0) and np.all(W[k, n_d:] == 0) and np.all(F[k, n_d:] == 0)


def test_velocity_full_size_sampled():
    import torch
    N, Nx, Nz = 1024, 64, 64
    with Plan(N, Nx, Nz, 1 / 2000, 1e-4) as plan:
        u = inputs.rhs_torch(plan.n_modes, N, seed=91)
        g = inputs.rhs_torch(plan.n_modes, N, seed=92)
        v, w = plan.velocity(u, g)
        z2 = so.mode_z2(Nx, Nz)
        modes = sorted({1, int(np.argmax(z2)), plan.n_modes // 2, plan.n_modes - 1})
        U, G = u[modes].cpu().numpy(), g[modes].cpu().numpy()
        V, W = v[modes].cpu().numpy(), w[modes].cpu().numpy()
    m, n = vel.mode_mn(Nx, Nz)
    # refined reference: B_D's per-parity condition number is about 0.4 (N/2)^2 = 1e5 at
    # N = 1024, so a plain float64 (or float-float) solve carries up to ~1e-11 relative
    F_ref = vel.f_from_u_ref(N, U)
    V_ref, W_ref = vel.velocity_from_fg(F_ref, G, m[modes], n[modes])
    for i in range(len(modes)):
        assert so.rel_l2(V[i, : N - 2], V_ref[i, : N - 2]) <= 1e-11
        assert so.rel_l2(W[i, : N - 2], W_ref[i, : N - 2]) <= 1e-11


def test_velocity_rejections():
    import torch
    with Plan(64, 8, 8, 1 / 180, 1e-3) as plan:
        u = inputs.rhs_torch(plan.n_modes, plan.N, seed=93)
        g = inputs.rhs_torch(plan.n_modes, plan.N, seed=94)
        for kw in ({"v": u}, {"w": g}, {"v": torch.empty_like(u), "w": None, "f": g}):
            with pytest.raises(ShenError) as e:
                plan.velocity(u, g, **{k: val for k, val in kw.items()})
            assert e.value.status == 1
        with pytest.raises(ShenError) as e:
            plan.velocity(u, g, precision="fp64")
        assert e.value.status == 5
    z2 = so.mode_z2(8, 8)
    with Plan(64, z2=z2, nu=1 / 180, dt=1e-3) as zp:                 # no (m, n) known
        with pytest.raises(ShenError) as e:
            zp.velocity(u, g)
        assert e.value.status == 5
