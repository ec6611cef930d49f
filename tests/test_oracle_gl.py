"""Pins of the Chebyshev-Gauss-Lobatto variant of the oracle (CPU).

With GL points the scalar product is the GL point sum (weights pi / (c_i N_x),
c_0 = c_{N_x} = 2, Sec. 2), exact to degree 2N - 3; in coefficient space that is the
GC form with c_{N-1} = 2 (Table tab:matrices caption).  Checked entry by entry against
the point sum itself in mpmath, and against the closed forms of the two entries that
change (the c_{k+2} term of B_D and the c_{k+4} term of B_B, Table tab:matrices)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import chebyshev as cb
from oracle import matrices as mat

mp = pytest.importorskip("mpmath").mp


def _basis(name, k, N):
    if name == "D":
        return [Fraction(x) for x in cb.dirichlet_int(k, N)]
    return [Fraction(x, cb.biharmonic_scale(k)) for x in cb.biharmonic_int(k, N)]


def _deriv(coeffs, d):
    a = [Fraction(x) for x in coeffs]
    for _ in range(d):
        a = [Fraction(x) for x in cb.unscale(cb.derivative_scaled(cb.cscale(a)))]
    return a


@pytest.mark.parametrize("N", [6, 9, 12])
def test_gl_matrices_equal_gl_point_sums(N):
    mp.dps = 40
    cases = [("D", "D", 0, mat.mass_dirichlet_exact(N, True)), ("D", "D", 2, mat.stiff_dirichlet_exact(N)),
             ("B", "B", 0, mat.mass_biharmonic_exact(N, True)), ("B", "B", 2, mat.stiff_biharmonic_exact(N)),
             ("B", "B", 4, mat.bilaplace_biharmonic_exact(N)), ("D", "B", 0, mat.coupling_exact(N, "M_B", True)),
             ("B", "D", 1, mat.coupling_exact(N, "C_D", True))]
    for trial, test, d, (num, den) in cases:
        n_test, n_trial = num.shape
        for k in range(n_test):
            v = _basis(test, k, N)
            for j in range(n_trial):
                u = _deriv(_basis(trial, j, N), d)
                q = cb.gl_quadrature_mp(u, v, N, mp)
                exact = mp.mpf(num[k, j]) / mp.mpf(den[k, j]) * mp.pi
                assert abs(q - exact) <= mp.mpf(10) ** -30 * max(1, abs(exact)), (trial, test, d, k, j)


@pytest.mark.parametrize("N", [8, 33, 64])
def test_gl_changes_only_the_highest_mode_entries(N):
    BD, BDg = mat.mass_dirichlet(N), mat.mass_dirichlet(N, True)
    BB, BBg = mat.mass_biharmonic(N), mat.mass_biharmonic(N, True)
    d1 = np.argwhere(BD != BDg)
    d2 = np.argwhere(BB != BBg)
    assert d1.tolist() == [[N - 3, N - 3]]
    assert d2.tolist() == [[N - 5, N - 5]]
    # B_D[k, k] = pi/2 (c_k + c_{k+2}) with c_{k+2} = c_{N-1} = 2 at k = N - 3
    assert BDg[N - 3, N - 3] == pytest.approx(3 * np.pi / 2, rel=1e-15)
    # B_B[k, k] = pi/2 (c_k + 4 ((k+2)/(k+3))^2 + c_{k+4} ((k+1)/(k+3))^2), c_{k+4} = 2 at k = N - 5
    k = N - 5
    expect = np.pi / 2 * (1 + 4 * ((k + 2) / (k + 3)) ** 2 + 2 * ((k + 1) / (k + 3)) ** 2)
    assert BBg[k, k] == pytest.approx(expect, rel=1e-15)
    # derivative couplings are the same for both point sets
    assert np.array_equal(mat.coupling(N, "C_D"), mat.coupling(N, "C_D", True))
