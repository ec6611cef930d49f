"""The forward transforms' least-squares form, checked on the CPU against the oracle.

The GPU forward transforms in phi and psi do not run a banded solve of B uhat = S
(Eqs. sst2, fstB).  They use two facts, checked here on the oracle's own matrices and
references so that a slip in either would show before any GPU run:

1. B = P^T diag(w) P with P = oracle.transforms.combination (phi_l = sum_k P_kl T_k) and
   w_k = (T_k, T_k)_sigma = pi c_k / 2 (the mass matrix, Table tab:matrices, from the
   discrete orthogonality of the T_k), so that uhat is the w-weighted least-squares fit
   of the Chebyshev coefficients.
2. Per parity, the basis combination factors as (I - Shift) for phi and
   (I - Shift)(I - b Shift), b_i = (K_i - 1) / (K_i + 1), for psi (Eq. phiN), so the fit
   reduces to a correction along the null space of P^T (constants; for psi also K^2)
   followed by prefix sums.

The float64 restatement below follows those steps; it must reproduce the oracle's
refined forward transform (tr.forward_ref, longdouble) to float64 rounding.
"""
import numpy as np
import pytest

from oracle import transforms as tr


def _ls_forward(space, chat, gl):
    N = chat.size
    n = tr.dim(space, N)
    out = np.zeros(N, dtype=complex)
    for h in (0, 1):
        K = np.arange(h, N, 2)
        om = np.ones(K.size)
        om[K == 0] = 0.5
        if gl:
            om[K == N - 1] = 0.5
        c = chat[K]
        r = om * c.sum() / om.sum()
        if space == "biharmonic":
            q = K ** 2.0 - (om * K ** 2.0).sum() / om.sum()
            r = r + om * q * (q * c).sum() / (om * q * q).sum()
        keep = K < n
        v = np.cumsum((c - r)[keep])
        if space == "biharmonic":
            Ku = K[keep] + 1.0
            v = np.cumsum(Ku * v) / Ku
        out[K[keep]] = v
    return out


def _cases():
    out = []
    for N in (8, 9, 16, 24, 33, 64, 96, 128):
        for gl in (False, True):
            L = N - 1 if gl else N
            if L & (L - 1) and not (L % 3 == 0 and (L // 3) & (L // 3 - 1) == 0):
                continue
            for space in ("dirichlet", "biharmonic"):
                out.append((N, gl, space))
    return out


@pytest.mark.parametrize("N,gl,space", _cases())
def test_mass_is_weighted_gram_of_the_combination(N, gl, space):
    P = tr.combination(space, N)
    w = np.pi / 2 * np.ones(N)
    w[0] = np.pi
    if gl:
        w[-1] = np.pi
    B = tr.mass(space, N, gl)
    assert np.allclose(P.T @ (w[:, None] * P), B, rtol=0, atol=1e-13 * np.abs(B).max())


@pytest.mark.parametrize("N,gl,space", _cases())
def test_least_squares_form_matches_refined_forward(N, gl, space):
    rng = np.random.default_rng(N + 17 * gl)
    X = rng.uniform(-1, 1, (3, N)) + 1j * rng.uniform(-1, 1, (3, N))
    ref = tr.forward_ref(space, X, gl=gl)
    chat = tr.forward_ref("chebyshev", X, gl=gl)
    got = np.array([_ls_forward(space, chat[m], gl) for m in range(X.shape[0])])
    assert np.abs(got - ref).max() <= 64 * 2.0 ** -53 * N * np.abs(ref).max()


def test_psi_factorisation():
    """Row K of the psi combination's transpose, K = 2 i + h: uhat_i - 2K/(K+1) uhat_{i-1}
    + (K-3)/(K-1) uhat_{i-2}; (I - S)(I - b S) with b_i = (K-1)/(K+1) has the same rows."""
    N = 40
    P = tr.combination("biharmonic", N)
    for h in (0, 1):
        K = np.arange(h, N, 2)
        R = (N - 4 - h + 1) // 2
        Lt = P[np.ix_(K, np.arange(h, N - 4, 2))]         # E_h x R_h block of parity h
        b = (K - 1.0) / (K + 1.0)
        E = K.size
        S = np.eye(E, k=-1)
        F = (np.eye(E) - S) @ (np.eye(E) - b[:, None] * S)
        assert np.allclose(F[:, :R], Lt, rtol=0, atol=1e-14)
