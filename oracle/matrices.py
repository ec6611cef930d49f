"""Dense Galerkin matrices of Sec. 3, from exact inner products (oracle, test infrastructure).

Convention (Sec. 3, X_{lq} = (phi_q, phi_l)): row index = test function k,
column index = trial function j, entry X[k, j] = (D^d trial_j, test_k)_sigma.

Stiffness sign (reading of Sec. 3): the paper defines A = -(phi'', phi) but its
Eqs. ufin, gfin, Biharmonic_matrix and Helmholtz_matrix are the Crank-Nicolson
discretisation of Eqs. biharmonic / g only when A = +(phi'', phi).  Every
stiffness matrix here is therefore the plain inner product (phi_j'', phi_k).

Each entry is computed as an exact rational multiple of pi (``chebyshev``) and
rounded to float64 once (correctly rounded integer division), then multiplied
by pi in float64.

Points (Sec. 2): Chebyshev-Gauss (GC) by default.  With ``gl=True`` the scalar product
is the Chebyshev-Gauss-Lobatto point sum, which in coefficient space is the same sum
with c_{N_x} = c_{N-1} = 2 (Table tab:matrices caption; GL quadrature with N points is
exact to degree 2N-3, and only T_{N-1} T_{N-1} exceeds it): the mass-type matrices change
in their highest-mode entries, the derivative couplings (stiffness, Q, C) do not.
"""
import functools
import math

import numpy as np

from . import chebyshev as cb


def _exact_matrix(N, trial, test, nderiv, n_trial, n_test, gl=False):
    """Exact matrix X[k, j] = (D^nderiv trial_j, test_k)_sigma / pi as (num, den) ints.

    trial(j, M) / test(k, M) return (integer coefficient list, integer scale):
    the basis function equals coeffs / scale.  gl: GL scalar product (c_{N-1} = 2).
    """
    M = N  # N Chebyshev modes: coefficient indices 0..N-1
    num = np.zeros((n_test, n_trial), dtype=object)
    den = np.ones((n_test, n_trial), dtype=object)
    tests = []
    for k in range(n_test):
        cv, sc = test(k, M)
        nz = [(n, v) for n, v in enumerate(cv) if v]
        tests.append((nz, sc))
    for j in range(n_trial):
        cv, sj = trial(j, M)
        g = cb.cscale(cv)
        for _ in range(nderiv):
            g = cb.derivative_scaled(g)
        if gl and len(g) >= M:
            g = list(g)
            g[M - 1] = 2 * g[M - 1]                  # c_{N-1} = 2 at GL points
        for k in range(n_test):
            nz, sk = tests[k]
            s = 0
            for n, v in nz:
                if g[n]:
                    s += g[n] * v
            # (D^d trial_j, test_k)/pi = (1/2) sum_n g_n v_n / (sj * sk)
            num[k, j] = s
            den[k, j] = 2 * sj * sk
    return num, den


def _to_f64(num, den):
    out = np.empty(num.shape, dtype=np.float64)
    flat_n, flat_d, flat_o = num.ravel(), den.ravel(), out.ravel()
    for i in range(flat_n.size):
        n = flat_n[i]
        flat_o[i] = 0.0 if n == 0 else n / flat_d[i]  # int/int: correctly rounded
    return out * math.pi


def _dirichlet(k, M):
    return cb.dirichlet_int(k, M), 1


def _biharmonic(k, M):
    return cb.biharmonic_int(k, M), cb.biharmonic_scale(k)


def _chebyshev(k, M):
    c = [0] * M
    c[k] = 1
    return c, 1


def _check_N(N, minimum):
    if N < minimum:
        raise ValueError(f"N={N} too small (need N >= {minimum})")


# ---------------------------------------------------------------------------
# Dirichlet space (phi_k = T_k - T_{k+2}, k = 0..N-3)
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def mass_dirichlet_exact(N, gl=False):
    """B_D[k, j] = (phi_j, phi_k)_sigma / pi, exact (num, den) (Table tab:matrices)."""
    _check_N(N, 4)
    return _exact_matrix(N, _dirichlet, _dirichlet, 0, N - 2, N - 2, gl)


@functools.lru_cache(maxsize=None)
def stiff_dirichlet_exact(N):
    """A_D[k, j] = (phi_j'', phi_k)_sigma / pi, exact (Sec. 3, sign per the reading above)."""
    _check_N(N, 4)
    return _exact_matrix(N, _dirichlet, _dirichlet, 2, N - 2, N - 2)


@functools.lru_cache(maxsize=None)
def mass_dirichlet(N, gl=False):
    return _to_f64(*mass_dirichlet_exact(N, gl))


@functools.lru_cache(maxsize=None)
def stiff_dirichlet(N):
    return _to_f64(*stiff_dirichlet_exact(N))


# ---------------------------------------------------------------------------
# Biharmonic space (psi_k, k = 0..N-5)
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def mass_biharmonic_exact(N, gl=False):
    """B_B[k, j] = (psi_j, psi_k)_sigma / pi, exact (Table tab:matrices)."""
    _check_N(N, 6)
    return _exact_matrix(N, _biharmonic, _biharmonic, 0, N - 4, N - 4, gl)


@functools.lru_cache(maxsize=None)
def stiff_biharmonic_exact(N):
    """A_B[k, j] = (psi_j'', psi_k)_sigma / pi, exact."""
    _check_N(N, 6)
    return _exact_matrix(N, _biharmonic, _biharmonic, 2, N - 4, N - 4)


@functools.lru_cache(maxsize=None)
def bilaplace_biharmonic_exact(N):
    """Q[k, j] = (psi_j'''', psi_k)_sigma / pi, exact (Eqs. N_Q, pk, rk)."""
    _check_N(N, 6)
    return _exact_matrix(N, _biharmonic, _biharmonic, 4, N - 4, N - 4)


@functools.lru_cache(maxsize=None)
def mass_biharmonic(N, gl=False):
    return _to_f64(*mass_biharmonic_exact(N, gl))


@functools.lru_cache(maxsize=None)
def stiff_biharmonic(N):
    return _to_f64(*stiff_biharmonic_exact(N))


@functools.lru_cache(maxsize=None)
def bilaplace_biharmonic(N):
    return _to_f64(*bilaplace_biharmonic_exact(N))


# ---------------------------------------------------------------------------
# Coupling matrices of Table tab:matrices (used here only as further pins of
# the inner-product machinery against printed closed forms).
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def coupling_exact(N, name, gl=False):
    """Exact (num, den) of a Table tab:matrices coupling matrix.

    'M_B'  (phi_j, psi_k)     k = 0..N-5, j = 0..N-3
    'C_B'  (phi_j', psi_k)    k = 0..N-5, j = 0..N-3
    'C_D'  (psi_j', phi_k)    k = 0..N-3, j = 0..N-5
    'C_T'  (phi_j', T_k)      k = 0..N-1, j = 0..N-3
    """
    _check_N(N, 6)
    if name == "M_B":
        return _exact_matrix(N, _dirichlet, _biharmonic, 0, N - 2, N - 4, gl)
    if name == "C_B":
        return _exact_matrix(N, _dirichlet, _biharmonic, 1, N - 2, N - 4, gl)
    if name == "C_D":
        return _exact_matrix(N, _biharmonic, _dirichlet, 1, N - 4, N - 2, gl)
    if name == "C_T":
        return _exact_matrix(N, _dirichlet, _chebyshev, 1, N - 2, N, gl)
    raise ValueError(name)


def coupling(N, name, gl=False):
    return _to_f64(*coupling_exact(N, name, gl))


# ---------------------------------------------------------------------------
# Systems.  Scaled forms (c = 2 / (nu dt), z2 = squared wavenumber):
#   Helmholtz   H_h = (z2 + c) B_D - A_D                      (alpha B - A)
#   biharmonic  H_b = Q - (2 z2 + c) A_B + z2 (z2 + c) B_B     (S + a A + b B)
# Paper forms (Eqs. Helmholtz_matrix, Biharmonic_matrix):
#   Hbar = -(nu dt/2) A_D + (1 + nu dt z2/2) B_D
#   Hchk = -(nu dt/2) Q + (1 + nu dt z2) A_B - (2 z2 + nu dt z2^2)/2 B_B
# Right-hand-side operators (Eqs. gfin, ufin):
#   paper:  2 B_D - Hbar ;  2 A_B - 2 z2 B_B - Hchk
#   scaled: R_h = (c - z2) B_D + A_D ;  R_b = Q + (c - 2 z2) A_B + z2 (z2 - c) B_B
# ---------------------------------------------------------------------------

def helmholtz_system(N, alpha, gl=False):
    """alpha B_D - A_D, the Helmholtz matrix in scaled form."""
    return alpha * mass_dirichlet(N, gl) - stiff_dirichlet(N)


def biharmonic_system(N, a, b, gl=False):
    """Q + a A_B + b B_B, the biharmonic matrix in scaled form."""
    return bilaplace_biharmonic(N) + a * stiff_biharmonic(N) + b * mass_biharmonic(N, gl)


def helmholtz_rhs_operator(N, z2, c, gl=False):
    """R_h = (c - z2) B_D + A_D  (Eq. gfin, scaled by 2/(nu dt))."""
    return (c - z2) * mass_dirichlet(N, gl) + stiff_dirichlet(N)


def biharmonic_rhs_operator(N, z2, c, gl=False):
    """R_b = Q + (c - 2 z2) A_B + z2 (z2 - c) B_B  (Eq. ufin, scaled by 2/(nu dt))."""
    return (bilaplace_biharmonic(N) + (c - 2.0 * z2) * stiff_biharmonic(N)
            + z2 * (z2 - c) * mass_biharmonic(N, gl))


def paper_helmholtz(N, z2, nu, dt):
    """Hbar of Eq. Helmholtz_matrix (with A = +(phi'', phi))."""
    return -(nu * dt / 2) * stiff_dirichlet(N) + (1 + nu * dt * z2 / 2) * mass_dirichlet(N)


def paper_biharmonic(N, z2, nu, dt):
    """Hchk of Eq. Biharmonic_matrix (with A = +(psi'', psi))."""
    return (-(nu * dt / 2) * bilaplace_biharmonic(N) + (1 + nu * dt * z2) * stiff_biharmonic(N)
            - (2 * z2 + nu * dt * z2 * z2) / 2 * mass_biharmonic(N))


def paper_helmholtz_rhs(N, z2, nu, dt):
    """2 B_D - Hbar  (Eq. gfin)."""
    return 2 * mass_dirichlet(N) - paper_helmholtz(N, z2, nu, dt)


def paper_biharmonic_rhs(N, z2, nu, dt):
    """2 A_B - 2 z2 B_B - Hchk  (Eq. ufin)."""
    return 2 * stiff_biharmonic(N) - 2 * z2 * mass_biharmonic(N) - paper_biharmonic(N, z2, nu, dt)


# ---------------------------------------------------------------------------
# Extended-precision copies (numpy longdouble) of the exact matrices, used only
# to compute residuals for the refined reference solution in ``solve``.
# ---------------------------------------------------------------------------

def _to_ld(num, den):
    out = np.empty(num.shape, dtype=np.longdouble)
    flat_n, flat_d, flat_o = num.ravel(), den.ravel(), out.ravel()
    for i in range(flat_n.size):
        n = flat_n[i]
        if n == 0:
            flat_o[i] = 0
        else:
            # split so that numerator and denominator each fit a longdouble exactly enough
            flat_o[i] = np.longdouble(n) / np.longdouble(flat_d[i])
    return out * PI_LD


PI_LD = np.longdouble("3.14159265358979323846264338327950288")


@functools.lru_cache(maxsize=None)
def ld_matrices(N, problem, gl=False):
    """(mass, stiffness[, bi-Laplacian]) in longdouble for 'helmholtz' / 'biharmonic'."""
    if problem == "helmholtz":
        return (_to_ld(*mass_dirichlet_exact(N, gl)), _to_ld(*stiff_dirichlet_exact(N)))
    return (_to_ld(*mass_biharmonic_exact(N, gl)), _to_ld(*stiff_biharmonic_exact(N)),
            _to_ld(*bilaplace_biharmonic_exact(N)))
