"""Velocity recovery of the linear step (oracle, test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; it
shares no code with the CUDA library.

Sec. 3: with the wall-normal velocity u (biharmonic space) and g (Dirichlet space) of
the new time level known, the remaining velocity components follow from
    f = dv/dy + dw/dz = -du/dx           (Eq. f: continuity)
projected on the Dirichlet space,
    B_D f_hat = -C u_hat,   C_kj = (psi_j', phi_k)_sigma   (Eq. ffin; Table tab:matrices),
and, for every mode except m = n = 0, from the algebraic Eqs. f3, g3
    i m v_hat + i n w_hat = f_hat,    i m w_hat - i n v_hat = g_hat,
whose solution is
    v_hat = i (n g_hat - m f_hat) / z2,   w_hat = -i (n f_hat + m g_hat) / z2,   z2 = m^2 + n^2.
The minus sign of B_D f = -C u follows Eq. f (and continuity); Eqs. f1 and ffin print
it without the sign.  m is the wavenumber of the first periodic direction (length Lx,
m = 2 pi ix / Lx, ix = 0..Nx/2), n of the second (length Lz, FFT order), as in the
mode layout of ``solve.mode_z2``.
"""
import math

import numpy as np
import scipy.linalg as sla

from . import matrices as mat


def mode_mn(Nx, Nz, Lx=2 * math.pi, Lz=math.pi):
    """(m, n) of every mode in mode-major order (m for the Nx direction, n for Nz)."""
    ix = np.arange(Nx // 2 + 1)
    iz = np.arange(Nz)
    kz = np.where(iz < Nz // 2, iz, iz - Nz)
    m = np.repeat(2 * math.pi * ix / Lx, Nz)
    n = np.tile(2 * math.pi * kz / Lz, Nx // 2 + 1)
    return m, n


def f_from_u(N, U, gl=False):
    """Dirichlet coefficients of f = -du/dx from biharmonic coefficients u_hat.

    U: complex (..., N) with entries 0..N-5 used; returns (..., N) with entries
    N-2.. zero.  Dense float64 solve of B_D f = -C u (Eq. ffin with the sign of Eq. f)."""
    U = np.asarray(U)
    B = mat.mass_dirichlet(N, gl)
    C = mat.coupling(N, "C_D", gl)                   # (N-2) x (N-4): (psi_j', phi_k)
    rhs = -(U[..., : N - 4] @ C.T)
    F = np.zeros(U.shape, dtype=complex)
    F[..., : N - 2] = sla.solve(B, rhs.reshape(-1, N - 2).T).T.reshape(rhs.shape)
    return F


def f_from_u_ref(N, U, steps=3, gl=False):
    """``f_from_u`` with iterative refinement: the residual -C u - B_D f is evaluated
    with the exactly assembled B_D and C in numpy longdouble and the correction solved
    in float64, removing the float64 rounding that B_D's conditioning (about 0.4 (N/2)^2,
    1e5 at N = 1024) amplifies in the plain dense solve."""
    U = np.atleast_2d(np.asarray(U))
    B = mat.mass_dirichlet(N, gl)
    Bl = mat._to_ld(*mat.mass_dirichlet_exact(N, gl))
    Cl = mat._to_ld(*mat.coupling_exact(N, "C_D", gl))
    lu = sla.lu_factor(B)
    out = np.zeros(U.shape, dtype=complex)
    for part in ("real", "imag"):
        u = getattr(U[:, : N - 4], part).astype(np.longdouble)
        rhs = -(u @ Cl.T)                                   # (modes, N-2) longdouble
        f = sla.lu_solve(lu, np.asarray(rhs, dtype=float).T).T.astype(np.longdouble)
        for _ in range(steps):
            r = rhs - f @ Bl.T
            f = f + sla.lu_solve(lu, np.asarray(r, dtype=float).T).T.astype(np.longdouble)
        if part == "real":
            out[:, : N - 2] += np.asarray(f, dtype=float)
        else:
            out[:, : N - 2] += 1j * np.asarray(f, dtype=float)
    return out


def velocity_from_fg(F, G, m, n):
    """(v_hat, w_hat) from f_hat, g_hat of modes with wavenumbers (m, n) (Eqs. f3, g3).

    F, G: (n_modes, N) or (N,); m, n: scalars or (n_modes,).  Modes with m = n = 0 get
    zeros (Eqs. f3, g3 do not hold there; the mean flow comes from Eqs. v00, w00)."""
    F, G = np.asarray(F), np.asarray(G)
    m = np.asarray(m, dtype=float)
    n = np.asarray(n, dtype=float)
    z2 = m * m + n * n
    safe = np.where(z2 > 0, z2, 1.0)
    if F.ndim == 2:
        m, n, safe, z2 = m[:, None], n[:, None], safe[:, None], z2[:, None]
    V = 1j * (n * G - m * F) / safe
    W = -1j * (n * F + m * G) / safe
    return np.where(z2 > 0, V, 0), np.where(z2 > 0, W, 0)
