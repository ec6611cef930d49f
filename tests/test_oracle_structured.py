"""Pins of the oracle's O(N) extended-precision operators and refined reference
(``oracle.structured``), on the CPU.

- every closed-form row entry against the exact rational inner products of ``matrices``
  (Table tab:matrices, Eqs. N_Q, pk, rk), Gauss and Gauss-Lobatto;
- the structured products H x against the exactly assembled dense matrices in longdouble;
- the refined reference against the dense refined reference (``solve.solve_mode_ref``)
  and against the 50-digit brute force.
"""
import numpy as np
import pytest

from oracle import matrices as mat
from oracle import solve as so
from oracle import structured as st
from paper_1701_03787_gb300 import inputs

LD = np.longdouble


def _exact_ld(num_den):
    num, den = num_den
    out = np.empty(num.shape, dtype=LD)
    for idx in np.ndindex(num.shape):
        out[idx] = LD(int(num[idx])) / LD(int(den[idx])) * mat.PI_LD if num[idx] else 0
    return out


@pytest.mark.parametrize("N", [12, 40])
@pytest.mark.parametrize("gl", [False, True])
def test_closed_form_entries_match_exact_inner_products(N, gl):
    B = _exact_ld(mat.mass_dirichlet_exact(N, gl))
    A = _exact_ld(mat.stiff_dirichlet_exact(N))
    T = st.tables("helmholtz", N, gl)
    n = N - 2
    for k in range(n):
        assert abs(B[k, k] - T["b0"][k]) <= 1e-18 * abs(B[k, k])
        if k + 2 < n:
            assert B[k, k + 2] == B[k + 2, k]
            assert abs(B[k, k + 2] - T["boff"][k]) <= 1e-18
        assert abs(A[k, k] - T["a0"][k]) <= 1e-18 * abs(A[k, k])
        for j in range(k + 2, n, 2):
            assert abs(A[k, j] - T["at"][k]) <= 1e-18 * abs(A[k, j])
        for j in list(range(0, k)) + list(range(k + 1, n, 2)):
            assert A[k, j] == 0
    B = _exact_ld(mat.mass_biharmonic_exact(N, gl))
    A = _exact_ld(mat.stiff_biharmonic_exact(N))
    Q = _exact_ld(mat.bilaplace_biharmonic_exact(N))
    T = st.tables("biharmonic", N, gl)
    n = N - 4
    close = lambda x, y: abs(x - y) <= 1e-18 * max(abs(x), abs(y), 1)
    for k in range(n):
        assert close(B[k, k], T["b0"][k])
        if k + 2 < n:
            assert close(B[k, k + 2], T["b2"][k]) and close(B[k + 2, k], T["b2"][k])
            assert close(A[k, k + 2], T["ap"][k]) and close(A[k + 2, k], T["am"][k + 2])
        if k + 4 < n:
            assert close(B[k, k + 4], T["b4"][k]) and close(B[k + 4, k], T["b4"][k])
        assert close(A[k, k], T["a0"][k])
        assert close(Q[k, k], T["q0"][k])
        for j in range(k + 2, n, 2):
            assert close(Q[k, j], T["p"][k] * T["q"][j] + T["r"][k] * T["s"][j])
        for j in range(0, k):
            assert Q[k, j] == 0
        for j in range(n):
            if abs(j - k) > 4 or (j - k) % 2:
                assert B[k, j] == 0
            if abs(j - k) > 2 or (j - k) % 2:
                assert A[k, j] == 0


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("N", [12, 64, 129])
@pytest.mark.parametrize("gl", [False, True])
def test_structured_product_matches_dense(problem, N, gl):
    n = so.n_unknowns(problem, N)
    X = np.random.default_rng(N).standard_normal((3, n))
    z2 = np.array([0.0, 37.0 ** 2, 143.0 ** 2])
    c = so.c_of(1 / 2000, 1e-4)
    Y = st.system_matvec(problem, N, z2, c, X, gl)
    for i in range(3):
        ref = so._system_ld(problem, N, z2[i], c, gl) @ X[i].astype(LD)
        assert float(np.max(np.abs(Y[i] - ref)) / np.max(np.abs(ref))) <= 1e-17


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("N", [256, 1024])
def test_refined_reference_matches_dense_refined(problem, N):
    c = so.c_of(1 / 2000, 1e-4)
    z2 = np.array([0.0, 400.0 ** 2, 1145.0 ** 2])
    F = inputs.rhs_numpy(3, N, seed=N + 7)
    R = st.solve_ref(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    assert np.all(R[:, n:] == 0)
    for i in range(3):
        ref = so.solve_mode_ref(problem, N, z2[i], c, F[i])
        assert so.rel_l2(R[i, :n], ref) <= 1e-14, (i, so.rel_l2(R[i, :n], ref))


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_refined_reference_matches_brute_force(problem):
    N, c = 24, so.c_of(1 / 180, 1e-3)
    z2 = np.array([0.0, 35.0 ** 2])
    F = inputs.rhs_numpy(2, N, seed=3)
    R = st.solve_ref(problem, N, z2, c, F)
    n = so.n_unknowns(problem, N)
    for i in range(2):
        assert so.rel_l2(R[i, :n], so.solve_mp(problem, N, z2[i], c, F[i])) <= 1e-15
