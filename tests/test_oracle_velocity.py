"""Pins of the velocity-recovery oracle (CPU): f = -du/dx projected on the Dirichlet
space (Eq. ffin with the sign of Eq. f), and v, w from Eqs. f3, g3.

Independent routes: numpy's Chebyshev routines (series evaluation and
differentiation) instead of the oracle's integer algebra and coupling matrix; a
closed form; direct substitution into Eqs. f3 / g3."""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import solve as so
from oracle import velocity as vel


def _psi_cheb(N):
    """Chebyshev coefficients (rows) of psi_k, k = 0..N-5 (Eq. phiN), float64."""
    P = np.zeros((N - 4, N))
    for k in range(N - 4):
        P[k, k] = 1.0
        P[k, k + 2] = -2.0 * (k + 2) / (k + 3)
        P[k, k + 4] = (k + 1) / (k + 3)
    return P


def _phi_cheb(N):
    D = np.zeros((N - 2, N))
    for k in range(N - 2):
        D[k, k], D[k, k + 2] = 1.0, -1.0
    return D


def test_f_of_psi0_is_eight_thirds_phi1():
    # psi_0 = T0 - 4/3 T2 + 1/3 T4, so -psi_0' = 8/3 (T1 - T3) = 8/3 phi_1
    N = 16
    U = np.zeros(N, dtype=complex)
    U[0] = 1.0
    F = vel.f_from_u(N, U)
    expect = np.zeros(N)
    expect[1] = 8.0 / 3.0
    assert np.allclose(F.real, expect, atol=1e-14) and np.all(F.imag == 0)


@pytest.mark.parametrize("N", [8, 24, 65])
def test_f_reproduces_minus_du_dx_pointwise(N):
    """-u' of a biharmonic-space u vanishes at +-1 and has degree <= N-2, so it lies in
    the Dirichlet space: the Galerkin f must equal it pointwise."""
    rng = np.random.default_rng(N)
    U = np.zeros((3, N), dtype=complex)
    U[:, : N - 4] = rng.standard_normal((3, N - 4)) + 1j * rng.standard_normal((3, N - 4))
    F = vel.f_from_u(N, U)
    x = np.cos(np.linspace(0.05, 3.1, 41))
    P, D = _psi_cheb(N), _phi_cheb(N)
    for i in range(3):
        u_cheb = U[i, : N - 4] @ P
        du = npc.chebval(x, npc.chebder(u_cheb))
        f = npc.chebval(x, F[i, : N - 2] @ D)
        scale = np.abs(du).max()
        assert np.abs(f + du).max() <= 1e-12 * scale
        assert np.all(F[i, N - 2:] == 0)


def test_velocity_satisfies_f3_and_g3():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((5, 12)) + 1j * rng.standard_normal((5, 12))
    G = rng.standard_normal((5, 12)) + 1j * rng.standard_normal((5, 12))
    m = np.array([0.0, 1.0, 3.0, 0.0, 7.0])
    n = np.array([2.0, -2.0, 0.0, -4.0, 12.0])
    V, W = vel.velocity_from_fg(F, G, m, n)
    assert np.allclose(1j * m[:, None] * V + 1j * n[:, None] * W, F, rtol=0, atol=1e-14)
    assert np.allclose(1j * m[:, None] * W - 1j * n[:, None] * V, G, rtol=0, atol=1e-14)
    V0, W0 = vel.velocity_from_fg(F[0], G[0], 0.0, 0.0)          # mean mode: left to Eqs. v00, w00
    assert np.all(V0 == 0) and np.all(W0 == 0)


def test_recovered_velocity_is_divergence_free():
    """du/dx + dv/dy + dw/dz = 0 at points, for the whole chain u -> f -> (v, w)."""
    N, m, n = 20, 2.0, -6.0
    rng = np.random.default_rng(5)
    U = np.zeros(N, dtype=complex)
    U[: N - 4] = rng.standard_normal(N - 4) + 1j * rng.standard_normal(N - 4)
    G = np.zeros(N, dtype=complex)
    G[: N - 2] = rng.standard_normal(N - 2)
    F = vel.f_from_u(N, U)
    V, W = vel.velocity_from_fg(F, G, m, n)
    x = np.linspace(-0.97, 0.97, 23)
    D = _phi_cheb(N)
    du = npc.chebval(x, npc.chebder(U[: N - 4] @ _psi_cheb(N)))
    div = du + 1j * m * npc.chebval(x, V[: N - 2] @ D) + 1j * n * npc.chebval(x, W[: N - 2] @ D)
    assert np.abs(div).max() <= 1e-12 * np.abs(du).max()


def test_mode_mn_matches_mode_z2():
    for Nx, Nz, Lx, Lz in [(8, 6, 2 * math.pi, math.pi), (16, 12, 4.0, 1.5)]:
        m, n = vel.mode_mn(Nx, Nz, Lx, Lz)
        assert np.allclose(m * m + n * n, so.mode_z2(Nx, Nz, Lx, Lz), rtol=1e-15, atol=0)
        assert m[0] == 0 and n[0] == 0


def test_refined_f_agrees_with_plain_solve_and_is_more_accurate():
    """At N = 256 the plain float64 solve and the refined one agree to B_D's
    conditioning times float64 rounding; the refined one reproduces -u' pointwise to
    a tighter bound."""
    N = 256
    rng = np.random.default_rng(11)
    U = np.zeros((2, N), dtype=complex)
    U[:, : N - 4] = (rng.standard_normal((2, N - 4)) + 1j * rng.standard_normal((2, N - 4))) / (1 + np.arange(N - 4))
    F0, F1 = vel.f_from_u(N, U), vel.f_from_u_ref(N, U)
    for i in range(2):
        assert so.rel_l2(F0[i, : N - 2], F1[i, : N - 2]) < 1e-11
    x = np.cos(np.linspace(0.05, 3.1, 31))
    P, D = _psi_cheb(N), _phi_cheb(N)
    du = npc.chebval(x, npc.chebder(U[0, : N - 4] @ P))
    err1 = np.abs(npc.chebval(x, F1[0, : N - 2] @ D) + du).max()
    assert err1 <= 1e-12 * np.abs(du).max()
