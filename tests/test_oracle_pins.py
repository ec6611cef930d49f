"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: an independent
evaluation of the paper's scalar product (sympy-exact derivatives at the
Chebyshev-Gauss points, Sec. 2 Eq. quadrature), printed closed forms
(Table tab:matrices, Eqs. N_Q, pk, rk), manufactured solutions with closed-form
loads, a 50-digit brute force, and invariants of the continuous problem.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import chebyshev as cb
from oracle import matrices as mat
from oracle import solve as so

PI = math.pi


def exact(num_den, k, j):
    n, d = num_den
    return Fraction(n[k, j], d[k, j])


# ---------------------------------------------------------------------------
# 1. The coefficient-space inner product equals the paper's GC point sum.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [8, 11])
def test_inner_product_equals_gc_point_sum_sympy(N):
    """(D^d trial_j, test_k) from exact coefficients == GC point sum of sympy-exact derivatives."""
    sp = pytest.importorskip("sympy")
    import mpmath
    x = sp.Symbol("x")

    def phi(k):
        return sp.chebyshevt(k, x) - sp.chebyshevt(k + 2, x)

    def psi(k):
        return (sp.chebyshevt(k, x) - sp.Rational(2 * (k + 2), k + 3) * sp.chebyshevt(k + 2, x)
                + sp.Rational(k + 1, k + 3) * sp.chebyshevt(k + 4, x))

    with mpmath.workdps(40):
        pts = [mpmath.cos((2 * i + 1) * mpmath.pi / (2 * N)) for i in range(N)]

        def gc(expr_u, expr_v):
            fu = sp.lambdify(x, sp.expand(expr_u), "mpmath")
            fv = sp.lambdify(x, sp.expand(expr_v), "mpmath")
            return mpmath.fsum(fu(p) * fv(p) for p in pts) * mpmath.pi / N

        cases = [
            (mat.mass_dirichlet_exact(N), phi, phi, 0),
            (mat.stiff_dirichlet_exact(N), phi, phi, 2),
            (mat.mass_biharmonic_exact(N), psi, psi, 0),
            (mat.stiff_biharmonic_exact(N), psi, psi, 2),
            (mat.bilaplace_biharmonic_exact(N), psi, psi, 4),
        ]
        for nd, trial, test, d in cases:
            n = nd[0].shape[0]
            for k in range(n):
                for j in range(n):
                    ref = gc(sp.diff(trial(j), x, d), test(k))
                    got = mpmath.mpf(exact(nd, k, j).numerator) / exact(nd, k, j).denominator * mpmath.pi
                    assert abs(ref - got) <= mpmath.mpf(10) ** -30 * (1 + abs(ref)), (d, k, j)


def test_inner_product_float_quadrature_moderate_N():
    """At N = 64 the float64 GC point sum agrees with the exact matrices (numpy chebder route)."""
    N = 64
    Q = mat.bilaplace_biharmonic(N)
    A = mat.stiff_biharmonic(N)
    rng = np.random.default_rng(1)
    for _ in range(20):
        k, j = rng.integers(0, N - 4, size=2)
        ck = np.zeros(N); ck[k] = 1; ck[k + 2] = -2 * (k + 2) / (k + 3); ck[k + 4] = (k + 1) / (k + 3)
        cj = np.zeros(N); cj[j] = 1; cj[j + 2] = -2 * (j + 2) / (j + 3); cj[j + 4] = (j + 1) / (j + 3)
        for deriv, M in ((4, Q), (2, A)):
            dj = np.polynomial.chebyshev.chebder(cj, deriv)
            ref = cb.gc_quadrature_f64(list(dj), list(ck), N)
            scale = max(1.0, np.abs(M).max() * 1e-3)
            assert abs(ref - M[k, j]) <= 1e-9 * scale


# ---------------------------------------------------------------------------
# 2. Printed closed forms (Table tab:matrices; GC points so c_{N_x} = 1).
# ---------------------------------------------------------------------------

def _ck(k):
    return 2 if k == 0 else 1


@pytest.mark.parametrize("N", [16, 33])
def test_table_mass_matrices(N):
    BD = mat.mass_dirichlet_exact(N)
    n = N - 2
    for k in range(n):
        for j in range(n):
            if j == k:
                ref = Fraction(_ck(k) + 1, 2)          # pi/2 (c_k + c_{k+2}), c_{k+2} = 1
            elif abs(j - k) == 2:
                ref = Fraction(-1, 2)
            else:
                ref = Fraction(0)
            assert exact(BD, k, j) == ref, (k, j)
    BB = mat.mass_biharmonic_exact(N)
    n = N - 4
    for k in range(n):
        for j in range(k, n):
            if j == k:
                ref = Fraction(1, 2) * (_ck(k) + 4 * Fraction(k + 2, k + 3) ** 2 + Fraction(k + 1, k + 3) ** 2)
            elif j == k + 2:
                ref = -(Fraction(k + 2, k + 3) + Fraction((k + 4) * (k + 1), (k + 5) * (k + 3)))
            elif j == k + 4:
                ref = Fraction(k + 1, 2 * (k + 3))
            else:
                ref = Fraction(0)
            assert exact(BB, k, j) == ref, (k, j)
            assert exact(BB, j, k) == ref  # symmetric


def test_table_coupling_matrices():
    N = 24
    CB = mat.coupling_exact(N, "C_B")       # (phi_j', psi_k)
    for k in range(N - 4):
        for j in range(N - 2):
            ref = {k - 1: -(k + 1), k + 1: 2 * (k + 1), k + 3: -(k + 1)}.get(j, 0)
            assert exact(CB, k, j) == ref, (k, j)
    CD = mat.coupling_exact(N, "C_D")       # (psi_j', phi_k)
    for k in range(N - 2):
        for j in range(N - 4):
            if j == k - 3:
                ref = Fraction((k - 2) * (k + 1), k)
            elif j == k - 1:
                ref = Fraction(-2 * (k + 1) ** 2, k + 2)
            elif j == k + 1:
                ref = Fraction(k + 1)
            else:
                ref = Fraction(0)
            assert exact(CD, k, j) == ref, (k, j)
    MB = mat.coupling_exact(N, "M_B")       # (phi_j, psi_k)
    for k in range(N - 4):
        for j in range(N - 2):
            if j == k - 2:
                ref = Fraction(-1, 2)
            elif j == k:
                ref = Fraction(1, 2) * (_ck(k) + 2 * Fraction(k + 2, k + 3))
            elif j == k + 2:
                ref = -Fraction(1, 2) * (2 * Fraction(k + 2, k + 3) + Fraction(k + 1, k + 3))
            elif j == k + 4:
                ref = Fraction(k + 1, 2 * (k + 3))
            else:
                ref = Fraction(0)
            assert exact(MB, k, j) == ref, (k, j)
    CT = mat.coupling_exact(N, "C_T")       # (phi_j', T_k), rows k >= 1 as printed
    for k in range(1, N):
        for j in range(N - 2):
            if j == k - 1:
                ref = -(k + 1)
            elif j >= k + 1 and (j - k) % 2 == 1:
                ref = -2
            else:
                ref = 0
            assert exact(CT, k, j) == ref, (k, j)


@pytest.mark.parametrize("N", [20, 64])
def test_bilaplace_closed_form(N):
    """Q off-diagonal p_k q_j + r_k s_j (Eqs. pk, rk); diagonal 8(k+1)^2(k+2)(k+4) (reading of Eq. N_Q)."""
    Q = mat.bilaplace_biharmonic_exact(N)
    n = N - 4
    for k in range(n):
        p = 8 * k * (k + 1) * (k + 2) * (k + 4)
        r = 24 * (k + 1) * (k + 2)
        for j in range(n):
            v = exact(Q, k, j)
            if j < k or (j - k) % 2:
                assert v == 0
            elif j == k:
                assert v == 8 * (k + 1) ** 2 * (k + 2) * (k + 4)
                # the diagonal as printed, -4(k+1)(k+2)^2, does not match (misprint)
                assert v != -4 * (k + 1) * (k + 2) ** 2
            else:
                assert v == p * Fraction(1, j + 3) + r * Fraction((j + 2) ** 2, j + 3)


def test_band_structure_claims():
    """Sec. 4: A_B has 3 diagonals (k-2, k, k+2), B_B has 5, the Dirichlet stiffness is upper
    triangular with one value per row beyond the diagonal."""
    N = 40
    A = mat.stiff_biharmonic(N)
    B = mat.mass_biharmonic(N)
    n = N - 4
    kk, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.all(A[np.abs(kk - jj) > 2] == 0)
    assert np.all(A[(np.abs(kk - jj) % 2) == 1] == 0)
    assert np.all(B[np.abs(kk - jj) > 4] == 0)
    AD = mat.stiff_dirichlet(N)
    for k in range(N - 2):
        assert np.all(AD[k, :k] == 0)
        tail = AD[k, k + 2::2]
        if tail.size:
            assert np.allclose(tail, tail[0], rtol=0, atol=0)
        assert np.all(AD[k, k + 1::2] == 0)


# ---------------------------------------------------------------------------
# 3. Manufactured solutions with closed-form loads.
# ---------------------------------------------------------------------------

def gc_load(g, test_coeffs, N):
    """(g, test)_sigma by the N-point GC sum in float64 (Sec. 2), g a callable."""
    i = np.arange(N)
    x = np.cos((2 * i + 1) * np.pi / (2 * N))
    return np.array([np.sum(g(x) * np.polynomial.chebyshev.chebval(x, tc)) * np.pi / N for tc in test_coeffs])


def dirichlet_tests(N):
    out = []
    for k in range(N - 2):
        c = np.zeros(N); c[k] = 1; c[k + 2] = -1
        out.append(c)
    return out


def biharmonic_tests(N):
    out = []
    for k in range(N - 4):
        c = np.zeros(N); c[k] = 1; c[k + 2] = -2 * (k + 2) / (k + 3); c[k + 4] = (k + 1) / (k + 3)
        out.append(c)
    return out


@pytest.mark.parametrize("N,z2,c", [(16, 0.0, 10.0), (64, 35.0 ** 2, 2 / (1 / 180 * 1e-3)), (128, 143.0 ** 2, 4e7)])
def test_manufactured_helmholtz_polynomial(N, z2, c):
    """u = 1 - x^2 = phi_0 / 2  solves  alpha u - u'' = alpha (1 - x^2) + 2."""
    alpha = z2 + c
    f = gc_load(lambda x: alpha * (1 - x ** 2) + 2.0, dirichlet_tests(N), N)
    u = so.solve_mode("helmholtz", N, z2, c, f.astype(complex))
    ref = np.zeros(N - 2); ref[0] = 0.5
    assert np.max(np.abs(u - ref)) <= 1e-13


@pytest.mark.parametrize("N,z2,c", [(16, 0.0, 10.0), (64, 35.0 ** 2, 2 / (1 / 180 * 1e-3)), (128, 143.0 ** 2, 4e7)])
def test_manufactured_biharmonic_polynomial(N, z2, c):
    """u = (1 - x^2)^2 = (3/8) psi_0 solves u'''' + a u'' + b u = f."""
    a, b = so.biharmonic_coeffs(z2, c)
    f = gc_load(lambda x: 24.0 + a * (12 * x ** 2 - 4) + b * (1 - x ** 2) ** 2, biharmonic_tests(N), N)
    u = so.solve_mode("biharmonic", N, z2, c, f.astype(complex))
    ref = np.zeros(N - 4); ref[0] = 3.0 / 8.0
    assert np.max(np.abs(u - ref)) <= 1e-12 * 3 / 8


def _eval_dirichlet(u, x):
    N = len(u) + 2
    t = np.zeros(N); t[: N - 2] += u; t[2:] -= u
    return np.polynomial.chebyshev.chebval(x, t)


def _eval_biharmonic(u, x):
    N = len(u) + 4
    k = np.arange(N - 4)
    t = np.zeros(N)
    t[: N - 4] += u
    t[2: N - 2] += -2 * (k + 2) / (k + 3) * u
    t[4:] += (k + 1) / (k + 3) * u
    return np.polynomial.chebyshev.chebval(x, t)


def test_manufactured_nonpolynomial_spectral_accuracy():
    """u = (1-x^2) e^x (Dirichlet) and (1-x^2)^2 cos 3x (biharmonic): spectral accuracy at N = 64."""
    N, z2, c = 64, 20.0 ** 2, 1e3
    alpha = z2 + c
    xs = np.linspace(-1, 1, 101)
    ue = lambda x: (1 - x ** 2) * np.exp(x)
    upp = lambda x: np.exp(x) * (-1 - 4 * x - x ** 2)          # ((1-x^2)e^x)''
    f = gc_load(lambda x: alpha * ue(x) - upp(x), dirichlet_tests(N), N)
    u = so.solve_mode("helmholtz", N, z2, c, f.astype(complex)).real
    assert np.max(np.abs(_eval_dirichlet(u, xs) - ue(xs))) <= 1e-13

    import sympy as sp
    x = sp.Symbol("x")
    expr = (1 - x ** 2) ** 2 * sp.cos(3 * x)
    a, b = so.biharmonic_coeffs(z2, c)
    g = sp.lambdify(x, sp.diff(expr, x, 4) + a * sp.diff(expr, x, 2) + b * expr, "numpy")
    ub = sp.lambdify(x, expr, "numpy")
    f = gc_load(g, biharmonic_tests(N), N)
    u = so.solve_mode("biharmonic", N, z2, c, f.astype(complex)).real
    assert np.max(np.abs(_eval_biharmonic(u, xs) - ub(xs))) <= 1e-13


# ---------------------------------------------------------------------------
# 4. The scaled systems are the paper's systems (Eqs. Helmholtz_matrix,
#    Biharmonic_matrix, gfin, ufin).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("z2", [0.0, 37.0, 1145.0 ** 2])
def test_scaled_forms_match_paper(z2):
    N, nu, dt = 48, 1 / 2000, 1e-4
    c = so.c_of(nu, dt)
    s = nu * dt / 2
    Hh = so.system_matrix("helmholtz", N, z2, c)
    Hb = so.system_matrix("biharmonic", N, z2, c)
    for got, ref in ((mat.paper_helmholtz(N, z2, nu, dt), s * Hh),
                     (mat.paper_biharmonic(N, z2, nu, dt), -s * Hb),
                     (mat.paper_helmholtz_rhs(N, z2, nu, dt), s * so.rhs_operator("helmholtz", N, z2, c)),
                     (mat.paper_biharmonic_rhs(N, z2, nu, dt), s * so.rhs_operator("biharmonic", N, z2, c))):
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# 5. Brute force, invariants, special cases.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [8, 16, 32])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_dense_lu_matches_50_digit_brute_force(N, problem):
    rng = np.random.default_rng(N)
    c = so.c_of(1 / 180, 1e-3)
    for z2 in (0.0, 300.0):
        f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        u = so.solve_mode(problem, N, z2, c, f)
        ub = so.solve_mp(problem, N, z2, c, f)
        assert so.rel_l2(u, ub) <= 1e-13


def _to_chebyshev(problem, u):
    n = len(u)
    if problem == "helmholtz":
        t = np.zeros(n + 2, dtype=complex); t[:n] += u; t[2:] -= u
        return t
    k = np.arange(n)
    t = np.zeros(n + 4, dtype=complex)
    t[:n] += u; t[2:n + 2] += -2 * (k + 2) / (k + 3) * u; t[4:] += (k + 1) / (k + 3) * u
    return t


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_wall_conditions_and_galerkin_residual(problem):
    N, c = 96, so.c_of(1 / 180, 5e-4)
    rng = np.random.default_rng(7)
    j = np.arange(N)
    f = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) / (1 + j) ** 2
    z2 = 50.0 ** 2
    H = so.system_matrix(problem, N, z2, c)
    u = so.solve_mode(problem, N, z2, c, f)
    n = len(u)
    res = H @ u - f[:n]
    assert np.linalg.norm(res) <= 50 * np.finfo(float).eps * np.linalg.norm(H, 2) * np.linalg.norm(u)
    t = _to_chebyshev(problem, u)
    n_ = np.arange(t.size)
    scale = np.sum(np.abs(t))
    assert abs(np.sum(t)) <= 1e-14 * scale                      # u(1) = 0
    assert abs(np.sum(t * (-1.0) ** n_)) <= 1e-14 * scale       # u(-1) = 0
    if problem == "biharmonic":
        d = np.sum(np.abs(t) * n_ ** 2)
        assert abs(np.sum(t * n_ ** 2)) <= 1e-13 * d            # u'(1) = 0
        assert abs(np.sum(t * n_ ** 2 * (-1.0) ** (n_ + 1))) <= 1e-13 * d


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_parity_decoupling_and_linearity(problem):
    N, c = 40, 1e3
    rng = np.random.default_rng(3)
    n = so.n_unknowns(problem, N)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    fe = f.copy(); fe[1::2] = 0
    ue = so.solve_mode(problem, N, 9.0, c, fe)
    assert np.all(ue[1::2] == 0) or np.max(np.abs(ue[1::2])) <= 1e-15 * np.max(np.abs(ue))
    u1 = so.solve_mode(problem, N, 9.0, c, f)
    ur = so.solve_mode(problem, N, 9.0, c, f.real.astype(complex))
    ui = so.solve_mode(problem, N, 9.0, c, (1j * f.imag))
    assert np.max(np.abs(u1 - ur - ui)) <= 1e-13 * np.max(np.abs(u1))


def test_large_alpha_limit_is_mass_solve():
    """alpha -> infinity: (alpha B - A) u = f  ->  u = B^{-1} f / alpha, B tridiagonal per parity."""
    import scipy.linalg as sl
    N, alpha = 64, 1e15
    rng = np.random.default_rng(5)
    f = rng.standard_normal(N - 2)
    u = so.solve_dense(mat.helmholtz_system(N, alpha), f.astype(complex)).real
    for p in (0, 1):
        idx = np.arange(p, N - 2, 2)
        d = np.array([PI * (1.5 if k == 0 else 1.0) for k in idx])
        off = -PI / 2 * np.ones(len(idx) - 1)
        ab = np.zeros((3, len(idx))); ab[0, 1:] = off; ab[1] = d; ab[2, :-1] = off
        ref = sl.solve_banded((1, 1), ab, f[idx]) / alpha
        assert np.max(np.abs(u[idx] - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_mode_layout():
    z2 = so.mode_z2(32, 32)
    assert z2.shape == (17 * 32,)
    Z = z2.reshape(17, 32)
    assert Z[0, 0] == 0.0
    assert Z[3, 0] == pytest.approx(9.0)                 # kx = 3 on a 2 pi box
    assert Z[0, 1] == pytest.approx(4.0)                 # kz = 1 on a pi box -> 2
    assert Z[0, 31] == pytest.approx(4.0)                # iz = 31 -> kz = -1
    assert Z[0, 16] == pytest.approx((2 * 16) ** 2)      # Nyquist kz = -16
    for iz in range(1, 32):
        assert Z[5, iz] == Z[5, 32 - iz] or iz == 16     # (kx, kz) and (kx, -kz): same system


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_refined_reference_matches_brute_force(problem):
    """The longdouble-refined reference agrees with the 50-digit brute force to ~1e-15."""
    N = 24
    c = so.c_of(1 / 2000, 1e-4)
    rng = np.random.default_rng(21)
    for z2 in (0.0, 1145.0 ** 2):
        f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        r = so.solve_mode_ref(problem, N, z2, c, f)
        ub = so.solve_mp(problem, N, z2, c, f)
        assert so.rel_l2(r, ub) <= 2e-15
