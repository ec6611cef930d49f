"""Wall-normal Shen transforms (oracle, test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; it
shares no code with the CUDA library.

Plain definitions of what Algorithms fst and ifst compute with fast cosine
transforms (Sec. 2, Eqs. ifft, sst1, sst2, fstB), for one wall-normal column per
Fourier mode:

    points     GC:  x_i = cos((2i+1) pi / (2N)),        sigma_i = pi / N
               GL:  x_i = cos(i pi / (N-1)),            sigma_i = pi / (c_i (N-1)),
                    c_0 = c_{N-1} = 2, c_i = 1 otherwise            (i = 0..N-1)
    inverse    u(x_i) = sum_l uhat_l phi_l(x_i)                   (Eq. ifft, S^{-1})
    scalar     S_l = (u, phi_l)_sigma = sum_i u(x_i) phi_l(x_i) sigma_i   (Eq. sst1)
    forward    uhat = B^{-1} S,  B_lq = (phi_q, phi_l)_sigma      (Eqs. sst2, fstB)

with N the number of points and Chebyshev modes and three spaces:
    'chebyshev'   T_k, k = 0..N-1           (B diagonal: pi c_k / 2, c_0 = 2,
                                             c_{N-1} = 2 for GL, else 1)
    'dirichlet'   phi_k = T_k - T_{k+2}, k = 0..N-3            (Eq. phiD)
    'biharmonic'  psi_k = T_k - 2(k+2)/(k+3) T_{k+2} + (k+1)/(k+3) T_{k+4},
                  k = 0..N-5                                   (Eq. phiN)
The Dirichlet and biharmonic mass matrices are the exactly assembled ones of
``matrices`` (Table tab:matrices); the point sums here are evaluated directly, so
the tests can pin one against the other.

Reading: Algorithm fst's scalar product for the Chebyshev space already divides by
pi c_k / 2 and its transform then applies B^{-1} once more; taken here as a slip of
the listing: the scalar product is (u, T_k)_sigma and the transform divides once.

Fields are complex (n_modes, N) arrays, mode-major; coefficient entries beyond a
space's dimension are ignored on input and zero on output.
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev as cb
from . import matrices as mat

SPACES = ("chebyshev", "dirichlet", "biharmonic")


def dim(space, N):
    """Number of basis functions of a space with N Chebyshev modes."""
    return {"chebyshev": N, "dirichlet": N - 2, "biharmonic": N - 4}[space]


def points(N, gl=False, dtype=float):
    """Quadrature points x_i, i = 0..N-1 (Sec. 2)."""
    i = np.arange(N)
    if gl:
        return np.cos(np.asarray(i, dtype=dtype) * np.asarray(np.pi, dtype=dtype) / (N - 1))
    return np.cos(np.asarray(2 * i + 1, dtype=dtype) * np.asarray(np.pi, dtype=dtype) / (2 * N))


def weights(N, gl=False):
    """Quadrature weights sigma_i (Sec. 2)."""
    if gl:
        w = np.full(N, np.pi / (N - 1))
        w[0] /= 2
        w[-1] /= 2
        return w
    return np.full(N, np.pi / N)


def cheb_at_points(N, gl=False, dtype=float):
    """T_k(x_i) as an (N points, N modes) matrix, T_k(cos t) = cos(k t).

    The angle k t is reduced exactly in integers before the cosine: GC t_i =
    (2i+1) pi / (2N), so k t_i = pi ((k (2i+1)) mod 4N) / (2N); GL t_i = i pi / (N-1),
    so k t_i = pi ((k i) mod 2(N-1)) / (N-1)."""
    i = np.arange(N)[:, None]
    k = np.arange(N)[None, :]
    pi = np.asarray(np.pi, dtype=dtype) if dtype is float else mat.PI_LD
    if gl:
        m = (k * i) % (2 * (N - 1))
        return np.cos(m.astype(dtype) * pi / (N - 1))
    m = (k * (2 * i + 1)) % (4 * N)
    return np.cos(m.astype(dtype) * pi / (2 * N))


def combination(space, N, dtype=float):
    """(N, dim) matrix P of Chebyshev coefficients of the basis: phi_l = sum_k P_kl T_k."""
    n = dim(space, N)
    P = np.zeros((N, n), dtype=dtype)
    for l in range(n):
        if space == "chebyshev":
            P[l, l] = 1
        elif space == "dirichlet":
            for k, c in enumerate(cb.dirichlet_int(l, N)):
                if c:
                    P[k, l] = c
        else:
            s = cb.biharmonic_scale(l)
            for k, c in enumerate(cb.biharmonic_int(l, N)):
                if c:
                    P[k, l] = np.asarray(c, dtype=dtype) / np.asarray(s, dtype=dtype)
    return P


def basis_at_points(space, N, gl=False, dtype=float):
    """phi_l(x_i) as an (N, dim) matrix, from the T_k(x_i) columns by Eqs. phiD / phiN."""
    T = cheb_at_points(N, gl, dtype)
    n = dim(space, N)
    if space == "chebyshev":
        return T
    if space == "dirichlet":
        return T[:, :n] - T[:, 2: n + 2]
    l = np.arange(n).astype(dtype)
    return T[:, :n] - (2 * (l + 2) / (l + 3)) * T[:, 2: n + 2] + ((l + 1) / (l + 3)) * T[:, 4: n + 4]


def mass(space, N, gl=False):
    """B_lq = (phi_q, phi_l)_sigma (float64): diagonal for 'chebyshev', Table tab:matrices otherwise."""
    if space == "chebyshev":
        c = np.ones(N)
        c[0] = 2
        if gl:
            c[-1] = 2
        return np.diag(np.pi * c / 2)
    return mat.mass_dirichlet(N, gl) if space == "dirichlet" else mat.mass_biharmonic(N, gl)


def _weights_ld(N, gl=False):
    if gl:
        w = np.full(N, mat.PI_LD / (N - 1), dtype=np.longdouble)
        w[0] /= 2
        w[-1] /= 2
        return w
    return np.full(N, mat.PI_LD / N, dtype=np.longdouble)


def _mass_ld(space, N, gl=False):
    if space == "chebyshev":
        c = np.ones(N, dtype=np.longdouble)
        c[0] = 2
        if gl:
            c[-1] = 2
        return np.diag(mat.PI_LD * c / 2)
    ex = mat.mass_dirichlet_exact(N, gl) if space == "dirichlet" else mat.mass_biharmonic_exact(N, gl)
    return mat._to_ld(*ex)


def _pad(Y, N):
    out = np.zeros(Y.shape[:-1] + (N,), dtype=complex)
    out[..., : Y.shape[-1]] = Y
    return out


def inverse(space, C, gl=False):
    """Physical values u(x_i) from coefficients (Eq. ifft in x: S^{-1}); C (..., N) complex."""
    C = np.asarray(C)
    N = C.shape[-1]
    n = dim(space, N)
    return C[..., :n] @ basis_at_points(space, N, gl).T


def scalar(space, U, gl=False):
    """Scalar products S_l = (u, phi_l)_sigma of physical values U (..., N) (Eq. sst1)."""
    U = np.asarray(U)
    N = U.shape[-1]
    V = basis_at_points(space, N, gl) * weights(N, gl)[:, None]
    return _pad(U @ V, N)


def forward(space, U, gl=False):
    """Coefficients uhat = B^{-1} (u, phi)_sigma (Eq. fstB), dense float64 solve."""
    U = np.asarray(U)
    N = U.shape[-1]
    n = dim(space, N)
    S = scalar(space, U, gl)[..., :n]
    X = sla.solve(mass(space, N, gl), S.reshape(-1, n).T).T.reshape(S.shape)
    return _pad(X, N)


def forward_ref(space, U, gl=False, steps=3):
    """``forward`` computed with the scalar product and the residuals in numpy longdouble
    and float64 corrections (iterative refinement): removes the float64 rounding that
    the mass matrices' conditioning amplifies in the plain solve at large N."""
    U = np.atleast_2d(np.asarray(U))
    N = U.shape[-1]
    n = dim(space, N)
    Vw = basis_at_points(space, N, gl, dtype=np.longdouble) * _weights_ld(N, gl)[:, None]
    Bl = _mass_ld(space, N, gl)
    lu = sla.lu_factor(mass(space, N, gl))
    out = np.zeros(U.shape, dtype=complex)
    for part, unit in (("real", 1.0), ("imag", 1j)):
        u = getattr(U, part).astype(np.longdouble)
        S = u @ Vw                                            # (modes, n) longdouble
        x = sla.lu_solve(lu, np.asarray(S, dtype=float).T).T.astype(np.longdouble)
        for _ in range(steps):
            r = S - x @ Bl.T
            x = x + sla.lu_solve(lu, np.asarray(r, dtype=float).T).T.astype(np.longdouble)
        out[:, :n] += unit * np.asarray(x, dtype=float)
    return out


def scalar_ref(space, U, gl=False):
    """``scalar`` evaluated in numpy longdouble."""
    U = np.atleast_2d(np.asarray(U))
    N = U.shape[-1]
    Vw = basis_at_points(space, N, gl, dtype=np.longdouble) * _weights_ld(N, gl)[:, None]
    out = np.zeros(U.shape, dtype=complex)
    for part, unit in (("real", 1.0), ("imag", 1j)):
        out[:, : Vw.shape[1]] += unit * np.asarray(getattr(U, part).astype(np.longdouble) @ Vw, dtype=float)
    return out


def inverse_ref(space, C, gl=False):
    """``inverse`` evaluated in numpy longdouble."""
    C = np.atleast_2d(np.asarray(C))
    N = C.shape[-1]
    n = dim(space, N)
    V = basis_at_points(space, N, gl, dtype=np.longdouble)
    out = np.zeros(C.shape, dtype=complex)
    for part, unit in (("real", 1.0), ("imag", 1j)):
        out += unit * np.asarray(getattr(C[:, :n], part).astype(np.longdouble) @ V.T, dtype=float)
    return out
