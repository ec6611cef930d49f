"""The paper's O(N) algorithms (oracle/shen_on.c) against the dense definition (CPU only)."""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so


def _rhs(rng, n_modes, N):
    j = np.arange(N)
    return (rng.standard_normal((n_modes, N)) + 1j * rng.standard_normal((n_modes, N))) / (1 + j) ** 2


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("N", [8, 9, 12, 13, 64, 129])
def test_on_matches_dense(problem, N):
    rng = np.random.default_rng(N)
    z2 = np.array([0.0, 4.0, 37.0 ** 2, 143.0 ** 2])
    c = so.c_of(1 / 180, 5e-4)
    F = _rhs(rng, z2.size, N)
    U = on.solve_modes(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    for m in range(z2.size):
        ref = so.solve_mode(problem, N, z2[m], c, F[m])
        assert so.rel_l2(U[m, :n], ref) <= 1e-12
        assert np.all(U[m, n:] == 0)


@pytest.mark.parametrize("N", [10, 17, 40])
def test_compact_factorisation_equals_printed_dense_algorithm(N):
    """Algorithm LUbiharmonic with dense U (as printed) and the compact 7N-storage form agree."""
    rng = np.random.default_rng(0)
    c = 1e4
    for z2 in (0.0, 100.0, 1e4):
        f = _rhs(rng, 1, N)[0]
        u_dense = on.biharmonic_dense_lu(N, z2, c, f)
        u_comp = on.solve_modes("biharmonic", N, np.array([z2]), c, f[None, :])[0]
        assert np.max(np.abs(u_dense - u_comp)) <= 1e-13 * np.max(np.abs(u_dense))


def test_on_roundoff_relative_to_pivoted_lu():
    """Sec. 5 roundoff procedure (u ~ U(0,1), f = H u, nu = 1/5200, dt = 1e-5) used as a relative
    test: the O(N) solve stays within 10x of dense pivoted LU (plus an absolute floor)."""
    nu, dt = 1 / 5200, 1e-5
    c = so.c_of(nu, dt)
    rng = np.random.default_rng(11)
    for N in (64, 128):
        for zl in (0.0, 200.0, 1800.0):
            z2 = zl * zl
            for problem in ("helmholtz", "biharmonic"):
                n = so.n_unknowns(problem, N)
                H = so.system_matrix(problem, N, z2, c)
                u = rng.uniform(0, 1, n)
                f = np.zeros(N, complex)
                f[:n] = H @ u
                v_on = on.solve_modes(problem, N, np.array([z2]), c, f[None, :])[0, :n].real
                v_lu = so.solve_dense(H, f[:n]).real
                e_on = np.max(np.abs(u - v_on)) / np.max(np.abs(u))
                e_lu = np.max(np.abs(u - v_lu)) / np.max(np.abs(u))
                assert e_on <= 10 * e_lu + 1e-13, (problem, N, zl, e_on, e_lu)


def test_on_rejects_too_small():
    with pytest.raises(ValueError):
        on.solve_modes("biharmonic", 7, np.array([0.0]), 1.0, np.zeros((1, 7), complex))
