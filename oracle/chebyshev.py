"""Exact Chebyshev-coefficient algebra for the Shen bases (oracle, test infrastructure).

Everything here is exact: coefficients are Python integers (arbitrary precision),
so every inner product below is an exact rational multiple of pi.

Bases (Sec. 2, Eqs. Tk, phiD, phiN):
    T_k                                   Chebyshev polynomial of the first kind
    phi_k   = T_k - T_{k+2}               Shen Dirichlet basis, k = 0..N-3
    psi_k   = T_k - 2(k+2)/(k+3) T_{k+2} + (k+1)/(k+3) T_{k+4}
                                          Shen biharmonic basis, k = 0..N-5
with N the number of Chebyshev modes (N = N_x + 1 in the paper's notation).

Scalar product (Sec. 2, Eq. quadrature): the discrete Chebyshev-Gauss sum
    (u, v)_sigma = sum_{i=0}^{N-1} u(x_i) v(x_i) pi/N,  x_i = cos((2i+1) pi / (2N)).
N-point Gauss quadrature is exact for polynomials of degree <= 2N-1 and every
product formed here has degree <= 2N-2, so the sum equals the weighted integral
and, by Chebyshev orthogonality, the coefficient-space form
    (u, v)_sigma = (pi/2) sum_n c_n u_n v_n,   c_0 = 2, c_n = 1 otherwise
(for GC points c_{N_x} = 1, Table tab:matrices caption).  ``gc_quadrature_mp``
evaluates the point sum itself so tests can pin that identity.
"""
from fractions import Fraction

import numpy as np


def dirichlet_int(k, M):
    """Integer coefficient vector (length M) of phi_k = T_k - T_{k+2} (Eq. phiD)."""
    c = [0] * M
    c[k] = 1
    c[k + 2] = -1
    return c


def biharmonic_int(k, M):
    """Integer coefficient vector (length M) of (k+3) * psi_k (Eq. phiN).

    (k+3) psi_k = (k+3) T_k - 2(k+2) T_{k+2} + (k+1) T_{k+4}; the factor (k+3)
    is returned separately by ``biharmonic_scale`` so that all arithmetic stays
    integral.
    """
    c = [0] * M
    c[k] = k + 3
    c[k + 2] = -2 * (k + 2)
    c[k + 4] = k + 1
    return c


def biharmonic_scale(k):
    return k + 3


def derivative_scaled(a):
    """Derivative of a Chebyshev series, returned in 'c-scaled' form.

    For f = sum_n a_n T_n the derivative f' = sum_n b_n T_n satisfies the
    classical backward recurrence c_{n-1} b_{n-1} = b_{n+1} + 2 n a_n (n >= 1),
    b_n = 0 for n >= len(a).  This returns bt_n = c_n b_n (so bt_0 = 2 b_0),
    which keeps integer input integral.  Only entries n >= 1 of the input enter
    the recurrence, so c-scaled input can be differentiated again directly.
    """
    M = len(a)
    b = [0] * (M + 2)
    for n in range(M - 1, 0, -1):
        b[n - 1] = b[n + 1] + 2 * n * a[n]
    return b[:M]


def unscale(bt):
    """Convert c-scaled coefficients bt_n = c_n b_n back to b_n (exact Fractions)."""
    out = [Fraction(x) for x in bt]
    if out:
        out[0] = out[0] / 2
    return out


def inner_over_pi(u_scaled, v):
    """(u, v)_sigma / pi for u in c-scaled form (u_t[n] = c_n u_n) and plain v.

    (u, v)_sigma = (pi/2) sum_n c_n u_n v_n  =>  (u, v)/pi = (1/2) sum_n u_t[n] v_n.
    Returns an exact Fraction.
    """
    s = 0
    for x, y in zip(u_scaled, v):
        if x and y:
            s += x * y
    return Fraction(s, 2)


def cscale(a):
    """Plain coefficients -> c-scaled (multiply entry 0 by c_0 = 2)."""
    out = list(a)
    if out:
        out[0] = 2 * out[0]
    return out


# ---------------------------------------------------------------------------
# Independent evaluation of the scalar product as the paper defines it: the
# Chebyshev-Gauss point sum (Eq. quadrature, GC weights), in mpmath.
# ---------------------------------------------------------------------------

def cheb_eval_mp(coeffs, x, mp):
    """Evaluate sum_n coeffs[n] T_n(x) by the three-term recurrence, in mpmath."""
    t0, t1 = mp.mpf(1), x
    s = mp.mpf(0)
    for n, a in enumerate(coeffs):
        if n == 0:
            t = t0
        elif n == 1:
            t = t1
        else:
            t = 2 * x * t1 - t0
            t0, t1 = t1, t
        if a:
            s += mp.mpf(Fraction(a).numerator) / mp.mpf(Fraction(a).denominator) * t
    return s


def gc_points_mp(N, mp):
    """Chebyshev-Gauss points x_i = cos((2i+1) pi / (2N)), i = 0..N-1 (Sec. 2, h(i))."""
    return [mp.cos((2 * i + 1) * mp.pi / (2 * N)) for i in range(N)]


def gc_quadrature_mp(u_coeffs, v_coeffs, N, mp):
    """(u, v)_sigma by the N-point GC point sum with weight pi/N, in mpmath."""
    xs = gc_points_mp(N, mp)
    w = mp.pi / N
    return mp.fsum(cheb_eval_mp(u_coeffs, x, mp) * cheb_eval_mp(v_coeffs, x, mp) for x in xs) * w


def gc_quadrature_f64(u_coeffs, v_coeffs, N):
    """Same point sum in float64 (numpy's Chebyshev evaluation), for moderate N."""
    i = np.arange(N)
    x = np.cos((2 * i + 1) * np.pi / (2 * N))
    uu = np.polynomial.chebyshev.chebval(x, np.array([float(c) for c in u_coeffs]))
    vv = np.polynomial.chebyshev.chebval(x, np.array([float(c) for c in v_coeffs]))
    return float(np.sum(uu * vv) * np.pi / N)


def gl_points_weights_mp(N, mp):
    """Chebyshev-Gauss-Lobatto points x_i = cos(i pi / N_x), i = 0..N_x (N_x = N - 1),
    with weights pi / (c_i N_x), c_0 = c_{N_x} = 2 (Sec. 2)."""
    Nx = N - 1
    xs = [mp.cos(i * mp.pi / Nx) for i in range(N)]
    ws = [mp.pi / ((2 if i in (0, Nx) else 1) * Nx) for i in range(N)]
    return xs, ws


def gl_quadrature_mp(u_coeffs, v_coeffs, N, mp):
    """(u, v)_sigma by the N-point GL point sum, in mpmath."""
    xs, ws = gl_points_weights_mp(N, mp)
    return mp.fsum(cheb_eval_mp(u_coeffs, x, mp) * cheb_eval_mp(v_coeffs, x, mp) * w for x, w in zip(xs, ws))
