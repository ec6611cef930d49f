"""Pins of the transforms oracle (oracle/transforms.py) against facts fixed by the
paper and by mathematics, independent of the oracle's own formulas:

- closed forms: 1 - x^2 = (1/2) phi_0 (Eq. phiD), (1 - x^2)^2 = (3/8) psi_0 (Eq. phiN),
  T_k at the points has Chebyshev coefficients e_k;
- Algorithms fst / ifst as printed, with SciPy's discrete cosine transforms as the
  library routine (types 2 / 3 for GC points, type 1 for GL);
- numpy's Chebyshev evaluation (chebval) for the inverse transform;
- the point-sum mass matrices equal the exactly assembled ones of Table tab:matrices;
- the forward transform is the sigma-orthogonal projection (Galerkin: the residual
  u - S^{-1}(T(u)) has zero scalar product with every basis function), and it inverts
  the inverse transform on the space.
"""
import numpy as np
import pytest
import scipy.fft as sf

from oracle import transforms as tr


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


# ---------------------------------------------------------------------------
# Algorithms fst and ifst as printed (N points; "N" in the listing is the last index)
# ---------------------------------------------------------------------------

def _dct(x, type_):
    return sf.dct(x.real, type=type_, axis=-1) + 1j * sf.dct(x.imag, type=type_, axis=-1)


def _fst_scalar(space, U, gl):
    N = U.shape[-1]
    w = _dct(U, 1) * np.pi / (2 * (N - 1)) if gl else _dct(U, 2) * np.pi / (2 * N)
    y = np.zeros_like(w)
    if space == "dirichlet":
        y[..., : N - 2] = w[..., : N - 2] - w[..., 2:]
    elif space == "biharmonic":
        k = np.arange(N - 4)
        y[..., : N - 4] = w[..., : N - 4] - 2 * (k + 2) / (k + 3) * w[..., 2: N - 2] + (k + 1) / (k + 3) * w[..., 4:]
    else:
        y = w
    return y


def _ifst(space, C, gl):
    N = C.shape[-1]
    z = np.zeros_like(C)
    if space == "dirichlet":
        z[..., : N - 2] = C[..., : N - 2]
        z[..., 2:] -= C[..., : N - 2]
    elif space == "biharmonic":
        k = np.arange(N - 4)
        z[..., : N - 4] = C[..., : N - 4]
        z[..., 2: N - 2] -= 2 * (k + 2) / (k + 3) * C[..., : N - 4]
        z[..., 4:] += (k + 1) / (k + 3) * C[..., : N - 4]
    else:
        z = C.copy()
    if gl:
        y = _dct(z, 1) / 2 + z[..., :1] / 2
        y = y + ((-1.0) ** np.arange(N)) / 2 * z[..., -1:]
    else:
        y = _dct(z, 3) / 2 + z[..., :1] / 2
    return y


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
@pytest.mark.parametrize("N", [8, 33, 64])
def test_scalar_matches_fast_algorithm(space, gl, N):
    U = _rand((5, N), 10 + N)
    ref = _fst_scalar(space, U, gl)
    got = tr.scalar(space, U, gl)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
@pytest.mark.parametrize("N", [8, 33, 64])
def test_inverse_matches_fast_algorithm(space, gl, N):
    C = _rand((5, N), 20 + N)
    C[:, tr.dim(space, N):] = 0
    ref = _ifst(space, C, gl)
    got = tr.inverse(space, C, gl)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
def test_inverse_matches_chebval(space, gl):
    N = 40
    C = _rand((3, N), 3)
    C[:, tr.dim(space, N):] = 0
    x = tr.points(N, gl)
    z = C[:, : tr.dim(space, N)] @ tr.combination(space, N).T          # Chebyshev coefficients
    ref = np.array([np.polynomial.chebyshev.chebval(x, zz) for zz in z])
    assert np.abs(tr.inverse(space, C, gl) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("gl", [False, True])
def test_closed_forms(gl):
    N = 24
    x = tr.points(N, gl)
    e0 = np.zeros(N)
    e0[0] = 1
    # 1 - x^2 = (T_0 - T_2) / 2 = phi_0 / 2
    np.testing.assert_allclose(tr.forward("dirichlet", 1 - x ** 2, gl), 0.5 * e0, atol=1e-14)
    np.testing.assert_allclose(tr.inverse("dirichlet", 0.5 * e0, gl), 1 - x ** 2, atol=1e-14)
    # (1 - x^2)^2 = 3/8 T_0 - 1/2 T_2 + 1/8 T_4 = 3/8 psi_0
    np.testing.assert_allclose(tr.forward("biharmonic", (1 - x ** 2) ** 2, gl), 0.375 * e0, atol=1e-14)
    np.testing.assert_allclose(tr.inverse("biharmonic", 0.375 * e0, gl), (1 - x ** 2) ** 2, atol=1e-14)
    # T_5 (x) = 16 x^5 - 20 x^3 + 5 x
    e5 = np.zeros(N)
    e5[5] = 1
    np.testing.assert_allclose(tr.forward("chebyshev", 16 * x ** 5 - 20 * x ** 3 + 5 * x, gl), e5, atol=1e-14)
    # the last mode too (GL: c_{N-1} = 2 in the Chebyshev mass matrix)
    eN = np.zeros(N)
    eN[-1] = 1
    np.testing.assert_allclose(tr.forward("chebyshev", tr.inverse("chebyshev", eN, gl), gl), eN, atol=1e-13)


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
def test_point_sum_mass_equals_table(space, gl):
    N = 30
    V = tr.basis_at_points(space, N, gl)
    B = V.T @ (V * tr.weights(N, gl)[:, None])
    np.testing.assert_allclose(B, tr.mass(space, N, gl), atol=1e-13)


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
def test_forward_is_galerkin_projection(space, gl):
    N = 48
    U = _rand((4, N), 7)                                      # not in the space (boundary values)
    r = U - tr.inverse(space, tr.forward(space, U, gl), gl)
    S = tr.scalar(space, r, gl)
    assert np.abs(S).max() <= 1e-13 * np.abs(tr.scalar(space, U, gl)).max()
    if space != "chebyshev":
        assert np.abs(r).max() > 1e-3                       # the projection does change u


@pytest.mark.parametrize("gl", [False, True])
@pytest.mark.parametrize("space", tr.SPACES)
@pytest.mark.parametrize("N", [16, 64])
def test_roundtrip(space, gl, N):
    C = _rand((4, N), 5)
    C[:, tr.dim(space, N):] = 0
    U = tr.inverse(space, C, gl)
    # the plain float64 solve carries cond(B) * eps (biharmonic B: 2e4 at N = 64)
    assert np.abs(tr.forward(space, U, gl) - C).max() <= (1e-11 if space == "biharmonic" else 1e-13)
    assert np.abs(tr.forward_ref(space, U, gl) - C).max() <= 1e-13
    assert np.abs(tr.inverse_ref(space, C, gl) - U).max() <= 1e-13 * np.abs(U).max()
    assert np.abs(tr.scalar_ref(space, U, gl) - tr.scalar(space, U, gl)).max() <= 1e-13 * np.abs(U).max()
