"""Definition of the per-mode solves and of the Fourier mode layout (oracle, test infrastructure).

For every Fourier mode the result is the exact solution of the dense real
Galerkin system of Sec. 3 (Eqs. ufin, gfin) -- the paper's O(N) algorithms of
Sec. 4 reach that same solution, they do not approximate it.  Here it is
computed by dense LU with partial pivoting (LAPACK through numpy), Re and Im as
two right-hand sides of one real system.  ``solve_mp`` is a 50-digit mpmath
brute force on the exact rational matrices for small N.

Mode layout (Sec. 2, wavenumber mesh K^p; periodic axes named x and z here):
mode index m = ix * Nz + iz, ix = 0..Nx/2 (kx = ix), iz = 0..Nz-1 with
kz = iz for iz < Nz/2 else iz - Nz (FFT order);  z2 = (2 pi kx/Lx)^2 + (2 pi kz/Lz)^2.
Defaults Lx = 2 pi, Lz = pi (the Re_tau = 2000 box of Sec. 5).
"""
import math

import numpy as np

from . import matrices as mat


def c_of(nu, dt):
    """c = 2 / (nu dt): the Crank-Nicolson constant of the scaled systems."""
    return 2.0 / (nu * dt)


def mode_z2(Nx, Nz, Lx=2 * math.pi, Lz=math.pi):
    """Squared wavenumber z2 of every mode, in mode-major order (length (Nx/2+1)*Nz)."""
    ix = np.arange(Nx // 2 + 1)
    iz = np.arange(Nz)
    kz = np.where(iz < Nz // 2, iz, iz - Nz)
    kxw = 2 * math.pi * ix / Lx
    kzw = 2 * math.pi * kz / Lz
    return (kxw[:, None] ** 2 + kzw[None, :] ** 2).ravel()


def helmholtz_coeffs(z2, c):
    """alpha = z2 + c for (alpha B - A) u = f."""
    return z2 + c


def biharmonic_coeffs(z2, c):
    """(a, b) = (-(2 z2 + c), z2 (z2 + c)) for (Q + a A + b B) u = f."""
    return -(2.0 * z2 + c), z2 * (z2 + c)


def n_unknowns(problem, N):
    return N - 2 if problem == "helmholtz" else N - 4


def system_matrix(problem, N, z2, c, gl=False):
    if problem == "helmholtz":
        return mat.helmholtz_system(N, helmholtz_coeffs(z2, c), gl)
    if problem == "biharmonic":
        a, b = biharmonic_coeffs(z2, c)
        return mat.biharmonic_system(N, a, b, gl)
    raise ValueError(problem)


def rhs_operator(problem, N, z2, c, gl=False):
    if problem == "helmholtz":
        return mat.helmholtz_rhs_operator(N, z2, c, gl)
    if problem == "biharmonic":
        return mat.biharmonic_rhs_operator(N, z2, c, gl)
    raise ValueError(problem)


def solve_dense(H, f):
    """Solve H u = f for complex f (length n) with a real H: dense LU, partial pivoting."""
    f = np.asarray(f)
    rhs = np.stack([f.real, f.imag], axis=-1).astype(np.float64)
    sol = np.linalg.solve(H, rhs)
    return sol[:, 0] + 1j * sol[:, 1]


def solve_mode(problem, N, z2, c, f, gl=False):
    """Solution coefficients (length n_unknowns) of one mode's system for load f."""
    n = n_unknowns(problem, N)
    return solve_dense(system_matrix(problem, N, z2, c, gl), np.asarray(f)[:n])


def _system_ld(problem, N, z2, c, gl=False):
    z2l, cl = np.longdouble(z2), np.longdouble(c)
    if problem == "helmholtz":
        B, A = mat.ld_matrices(N, problem, gl)
        return (z2l + cl) * B - A
    B, A, Q = mat.ld_matrices(N, problem, gl)
    return Q - (2 * z2l + cl) * A + z2l * (z2l + cl) * B


def solve_mode_ref(problem, N, z2, c, f, max_iter=6, gl=False):
    """Reference solution for tight checks: dense LU, then iterative refinement whose
    residual f - H u uses the exactly assembled H in numpy longdouble, until the
    correction stops shrinking.  Removes the float64 assembly and LU roundoff of
    ``solve_mode`` (which is ~5e-13 relative at N = 1024, z = 1145)."""
    n = n_unknowns(problem, N)
    H = system_matrix(problem, N, z2, c, gl)
    Hl = _system_ld(problem, N, z2, c, gl)
    f = np.asarray(f)[:n]
    lu = __import__("scipy.linalg", fromlist=["lu_factor"])
    fac = lu.lu_factor(H)
    out = []
    for part in (f.real, f.imag):
        fl = part.astype(np.longdouble)
        x = lu.lu_solve(fac, part).astype(np.longdouble)
        prev = np.inf
        for _ in range(max_iter):
            r = fl - Hl @ x
            d = lu.lu_solve(fac, r.astype(np.float64))
            x = x + d.astype(np.longdouble)
            nd = float(np.max(np.abs(d)))
            if nd == 0.0 or nd >= prev:
                break
            prev = nd
        out.append(x.astype(np.float64))
    return out[0] + 1j * out[1]


def matvec_mode(problem, N, z2, c, x, y=None, beta=0.0, gl=False):
    """out = R x + beta y for one mode (R the right-hand-side operator of Eq. gfin / ufin)."""
    n = n_unknowns(problem, N)
    out = rhs_operator(problem, N, z2, c, gl) @ np.asarray(x)[:n]
    if y is not None:
        out = out + beta * np.asarray(y)[:n]
    return out


def solve_field(problem, N, z2s, c, F, modes=None):
    """Solve every listed mode of a field F (shape (n_modes, >= n_unknowns), complex)."""
    z2s = np.asarray(z2s)
    modes = range(len(z2s)) if modes is None else modes
    n = n_unknowns(problem, N)
    out = {}
    for m in modes:
        out[int(m)] = solve_mode(problem, N, float(z2s[m]), c, F[m, :n])
    return out


# ---------------------------------------------------------------------------
# Brute force: 50-digit mpmath LU on the exact rational matrices (small N only).
# ---------------------------------------------------------------------------

def _exact_system_mp(problem, N, z2, c, mp):
    pi = mp.pi
    if problem == "helmholtz":
        bn, bd = mat.mass_dirichlet_exact(N)
        an, ad = mat.stiff_dirichlet_exact(N)
        alpha = mp.mpf(z2) + mp.mpf(c)
        n = N - 2
        H = mp.matrix(n, n)
        for k in range(n):
            for j in range(n):
                H[k, j] = pi * (alpha * mp.mpf(bn[k, j]) / bd[k, j] - mp.mpf(an[k, j]) / ad[k, j])
        return H
    qn, qd = mat.bilaplace_biharmonic_exact(N)
    an, ad = mat.stiff_biharmonic_exact(N)
    bn, bd = mat.mass_biharmonic_exact(N)
    z2m, cm = mp.mpf(z2), mp.mpf(c)
    a = -(2 * z2m + cm)
    b = z2m * (z2m + cm)
    n = N - 4
    H = mp.matrix(n, n)
    for k in range(n):
        for j in range(n):
            H[k, j] = pi * (mp.mpf(qn[k, j]) / qd[k, j] + a * mp.mpf(an[k, j]) / ad[k, j]
                            + b * mp.mpf(bn[k, j]) / bd[k, j])
    return H


def solve_mp(problem, N, z2, c, f, dps=50):
    """Brute-force solve of one mode at ``dps`` digits; returns complex128 coefficients."""
    import mpmath
    with mpmath.workdps(dps):
        H = _exact_system_mp(problem, N, z2, c, mpmath.mp)
        n = H.rows
        f = np.asarray(f)[:n]
        re = mpmath.lu_solve(H, mpmath.matrix([mpmath.mpf(float(v)) for v in f.real]))
        im = mpmath.lu_solve(H, mpmath.matrix([mpmath.mpf(float(v)) for v in f.imag]))
        return np.array([complex(float(re[i]), float(im[i])) for i in range(n)])


# ---------------------------------------------------------------------------
# Error metrics
# ---------------------------------------------------------------------------

def rel_l2(u, ref):
    """Per-mode relative L2 error ||u - ref|| / ||ref|| over the complex column."""
    ref = np.asarray(ref)
    u = np.asarray(u)[: ref.shape[-1]]
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(u - ref) / den) if den > 0 else float(np.linalg.norm(u))


def field_errors(results, refs):
    """max / median per-mode relative L2 and the field-level relative L2."""
    errs, num, den = [], 0.0, 0.0
    for m, ref in refs.items():
        u = np.asarray(results[m])[: len(ref)]
        errs.append(rel_l2(u, ref))
        num += float(np.sum(np.abs(u - ref) ** 2))
        den += float(np.sum(np.abs(ref) ** 2))
    errs = np.array(errs)
    return {"max": float(errs.max()), "median": float(np.median(errs)),
            "field": math.sqrt(num / den) if den > 0 else 0.0, "n": int(errs.size)}
