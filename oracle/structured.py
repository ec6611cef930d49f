"""Extended-precision residuals from the banded-plus-tail structure of the systems, and the
refined reference solution at any N (oracle, test infrastructure).

``solve.solve_mode_ref`` refines a dense LU solution with the exactly assembled dense
matrix, which is O(N^2) memory per mode and out of reach at N = 8192 or on thousands of
modes.  The same reference is reached here in O(N) per mode:

* the matrices are applied through their structure (Sec. 3, Table tab:matrices, Eqs. N_Q,
  pk, rk; stiffness with the + sign of the reading documented in ``matrices``), every entry
  evaluated from its closed form in numpy longdouble;
* starting from the paper's O(N) float64 solve (``shen_on.c``, Sec. 4), each step forms
  r = f - H u in longdouble and adds the O(N) float64 solution of H d = r.

Structure per parity chain (row k, columns of the same parity):
  Dirichlet  B_kk = pi/2 (c_k + c_{k+2}), B_{k,k+-2} = -pi/2;
             A_kk = -2 pi (k+1)(k+2), A_kj = -4 pi (k+1) for j = k+2, k+4, ...
  biharmonic B_kk = pi/2 (c_k + 4 ((k+2)/(k+3))^2 + c_{k+4} ((k+1)/(k+3))^2),
             B_{k,k+2} = B_{k+2,k} = -pi ((k+2)/(k+3) + (k+1)(k+4)/((k+3)(k+5))),
             B_{k,k+4} = B_{k+4,k} = pi/2 (k+1)/(k+3);
             A_kk = -4 pi (k+1)(k+2)^2/(k+3), A_{k,k+2} = 2 pi (k+1)(k+2),
             A_{k,k-2} = 2 pi (k-1)(k+2);
             Q_kk = 8 pi (k+1)^2 (k+2)(k+4) (the exact diagonal; Eq. N_Q misprints it),
             Q_kj = p_k q_j + r_k s_j for j = k+2, k+4, ... (Eqs. pk, rk):
             p_k = 8 pi k (k+1)(k+2)(k+4), r_k = 24 pi (k+1)(k+2), q_j = 1/(j+3),
             s_j = (j+2)^2/(j+3).
c_0 = 2; c_{N-1} = 2 for the Gauss-Lobatto scalar product, else 1.  Every closed form is
pinned entry by entry against the exact rational inner products of ``matrices``
(tests/test_oracle_structured.py).
"""
import numpy as np

from . import on
from . import solve as so

LD = np.longdouble
PI_LD = LD("3.14159265358979323846264338327950288")


def _c(kk, N, gl):
    c = np.ones(kk.shape, dtype=LD)
    c[kk == 0] = 2
    if gl:
        c[kk == N - 1] = 2
    return c


def tables(problem, N, gl=False):
    """Closed-form row entries (longdouble arrays indexed by the row k) of one problem."""
    if problem == "helmholtz":
        k = np.arange(N - 2).astype(LD)
        kk = np.arange(N - 2)
        return {
            "b0": PI_LD / 2 * (_c(kk, N, gl) + _c(kk + 2, N, gl)),
            "boff": np.full(N - 2, -PI_LD / 2, dtype=LD),
            "a0": -2 * PI_LD * (k + 1) * (k + 2),
            "at": -4 * PI_LD * (k + 1),
        }
    if problem != "biharmonic":
        raise ValueError(problem)
    k = np.arange(N - 4).astype(LD)
    kk = np.arange(N - 4)
    r2, r1 = (k + 2) / (k + 3), (k + 1) / (k + 3)
    return {
        "b0": PI_LD / 2 * (_c(kk, N, gl) + 4 * r2 * r2 + _c(kk + 4, N, gl) * r1 * r1),
        "b2": -PI_LD * (r2 + (k + 1) * (k + 4) / ((k + 3) * (k + 5))),
        "b4": PI_LD / 2 * r1,
        "a0": -4 * PI_LD * (k + 1) * (k + 2) * (k + 2) / (k + 3),
        "ap": 2 * PI_LD * (k + 1) * (k + 2),
        "am": 2 * PI_LD * (k - 1) * (k + 2),
        "q0": 8 * PI_LD * (k + 1) * (k + 1) * (k + 2) * (k + 4),
        "p": 8 * PI_LD * k * (k + 1) * (k + 2) * (k + 4),
        "r": 24 * PI_LD * (k + 1) * (k + 2),
        "q": 1 / (k + 3),
        "s": (k + 2) * (k + 2) / (k + 3),
    }


def _shift(X, d):
    """Y[:, k] = X[:, k + d] (zero outside the column)."""
    Y = np.zeros_like(X)
    n = X.shape[1]
    if d > 0:
        Y[:, : n - d] = X[:, d:]
    elif d < 0:
        Y[:, -d:] = X[:, : n + d]
    else:
        Y[:] = X
    return Y


def _tail(X):
    """T[:, k] = sum of X[:, j] over j = k+2, k+4, ... (same parity, strictly beyond k)."""
    T = np.zeros_like(X)
    for par in (0, 1):
        Xp = X[:, par::2]
        cs = np.cumsum(Xp[:, ::-1], axis=1)[:, ::-1]      # cs[:, i] = sum_{i' >= i}
        Tp = np.zeros_like(Xp)
        Tp[:, :-1] = cs[:, 1:]
        T[:, par::2] = Tp
    return T


def system_matvec(problem, N, z2, c, X, gl=False):
    """H X in longdouble for real X (n_modes, n), n = N-2 / N-4; z2 (n_modes,) float64.

    H is the scaled system of the problem (Helmholtz (z2 + c) B - A; biharmonic
    Q - (2 z2 + c) A + z2 (z2 + c) B) with a, b, alpha formed in longdouble from the
    float64 z2 and c."""
    T = tables(problem, N, gl)
    X = np.asarray(X, dtype=LD)
    z2 = np.asarray(z2, dtype=np.float64).astype(LD)[:, None]
    cl = LD(c)
    if problem == "helmholtz":
        BX = T["b0"] * X + T["boff"] * (_shift(X, -2) + _shift(X, 2))
        AX = T["a0"] * X + T["at"] * _tail(X)
        return (z2 + cl) * BX - AX
    BX = (T["b0"] * X + T["b2"] * _shift(X, 2) + _shift(T["b2"] * X, -2)
          + T["b4"] * _shift(X, 4) + _shift(T["b4"] * X, -4))
    AX = T["a0"] * X + T["ap"] * _shift(X, 2) + T["am"] * _shift(X, -2)
    QX = T["q0"] * X + T["p"] * _tail(T["q"] * X) + T["r"] * _tail(T["s"] * X)
    return QX - (2 * z2 + cl) * AX + z2 * (z2 + cl) * BX


def solve_ref(problem, N, z2, c, F, steps=3):
    """Refined reference of every mode (Chebyshev-Gauss): the O(N) float64 solve, then
    ``steps`` corrections with the residual in longdouble.  F complex (n_modes, >= n);
    returns complex128 (n_modes, N) with zeros beyond the unknowns."""
    n = so.n_unknowns(problem, N)
    z2 = np.ascontiguousarray(z2, dtype=np.float64)
    F = np.asarray(F)
    Fp = np.zeros((F.shape[0], N), dtype=np.complex128)
    Fp[:, :n] = F[:, :n]
    U = on.solve_modes(problem, N, z2, c, Fp)
    out = []
    for part in ("real", "imag"):
        f = getattr(Fp, part)[:, :n].astype(LD)
        x = getattr(U, part)[:, :n].astype(LD)
        for _ in range(steps):
            r = f - system_matvec(problem, N, z2, c, x)
            R = np.zeros((F.shape[0], N), dtype=np.complex128)
            R.real[:, :n] = r.astype(np.float64)
            x = x + on.solve_modes(problem, N, z2, c, R).real[:, :n].astype(LD)
        out.append(x.astype(np.float64))
    res = np.zeros((F.shape[0], N), dtype=np.complex128)
    res[:, :n] = out[0] + 1j * out[1]
    return res
