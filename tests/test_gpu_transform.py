"""GPU parity of the wall-normal transforms (shen_transform) against the transforms
oracle (oracle/transforms.py, longdouble references): inverse transform (Eq. ifft),
scalar products (Eq. sst1) and forward transform (Eqs. sst2, fstB) for the Chebyshev,
Dirichlet and biharmonic spaces (Eqs. Tk, phiD, phiN).

Tolerances follow from the arithmetic: the kernels run in float-float (unit roundoff
u = 2^-47 taken conservatively), each output of the inverse transform and of the scalar
product is a sum over the column with coefficients of modulus at most 1 (cosines) or 4
(the psi combination), evaluated through lg = log2 N radix passes, so its absolute error
is below C (lg + 2) u sum_j |in_j| (times pi / N for the scalar products).  The forward
transform's mass solve multiplies that by the conditioning of B: it is checked through
its defining property (B uhat reproduces the scalar products to the same bound, scaled
by ||B||), and against the refined projection within 64 (= 2^-47 / 2^-53) times the error
of the plain float64 dense solve of the same system.

Sizes: N a power of two, and N = 3 2^p (24, 96, 1536: the FFT adds one radix-3 pass), on
Gauss points; on Gauss-Lobatto points N - 1 of either form.
"""
import numpy as np
import pytest

from oracle import transforms as tr
from paper_1701_03787_gb300 import Plan, ShenError, inputs

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -47
C_BOUND = 16


def _bound(N, in_row, scale=1.0, weight=1.0):
    lg = int(np.ceil(np.log2(N)))              # passes of the FFT (one radix-3 pass counts as one)
    return C_BOUND * (lg + 2) * U_DF * weight * scale * np.abs(in_row).sum()


def _values(n_modes, N, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (n_modes, N)) + 1j * rng.uniform(-1, 1, (n_modes, N))


def _run(plan, kind, space, X):
    import torch
    x = torch.as_tensor(np.ascontiguousarray(X), device="cuda")
    out = plan.transform(kind, space, x)
    torch.cuda.synchronize()
    return out.cpu().numpy()


WEIGHT = {"chebyshev": 1.0, "dirichlet": 2.0, "biharmonic": 4.0}


@pytest.mark.parametrize("N", [8, 16, 24, 32, 96, 128, 1024, 1536])
@pytest.mark.parametrize("space", tr.SPACES)
def test_inverse_matches_oracle(N, space):
    with Plan(N, 4, 4, 1 / 180, 1e-3) as plan:
        C = inputs.rhs_numpy(plan.n_modes, N, seed=N + 3)      # trailing entries nonzero: ignored
        U = _run(plan, "inverse", space, C)
    Cs = C.copy()
    Cs[:, tr.dim(space, N):] = 0
    ref = tr.inverse_ref(space, Cs)
    for m in range(C.shape[0]):
        err = np.abs(U[m] - ref[m]).max()
        assert err <= _bound(N, Cs[m], weight=WEIGHT[space]), (m, err)


@pytest.mark.parametrize("N", [8, 16, 24, 32, 96, 128, 1024, 1536])
@pytest.mark.parametrize("space", tr.SPACES)
def test_scalar_matches_oracle(N, space):
    with Plan(N, 4, 4, 1 / 180, 1e-3) as plan:
        X = _values(plan.n_modes, N, seed=N + 5)
        S = _run(plan, "scalar", space, X)
    ref = tr.scalar_ref(space, X)
    n = tr.dim(space, N)
    for m in range(X.shape[0]):
        err = np.abs(S[m] - ref[m]).max()
        assert err <= _bound(N, X[m], scale=np.pi / N, weight=WEIGHT[space]), (m, err)
        assert np.all(S[m, n:] == 0)


def _forward_cases():
    return [(N, s) for N in (8, 16, 24, 64, 96, 128, 1024) for s in tr.SPACES]


@pytest.mark.parametrize("N,space", _forward_cases())
def test_forward_is_projection(N, space):
    """B uhat = (u, phi)_sigma: the defining equation of the forward transform (Eq. fstB)."""
    with Plan(N, 4, 4, 1 / 180, 1e-3) as plan:
        X = _values(plan.n_modes, N, seed=N + 7)
        Uh = _run(plan, "forward", space, X)
    n = tr.dim(space, N)
    B = tr.mass(space, N)
    S_ref = tr.scalar_ref(space, X)[:, :n]
    normB = np.abs(B).sum(axis=1).max()
    for m in range(X.shape[0]):
        assert np.all(Uh[m, n:] == 0)
        r = B @ Uh[m, :n] - S_ref[m]
        tol = _bound(N, X[m], scale=np.pi / N, weight=WEIGHT[space]) + 8 * (int(np.log2(N)) + 2) * U_DF * normB * np.abs(
            Uh[m, :n]).max()
        assert np.abs(r).max() <= tol, (m, np.abs(r).max(), tol)


def _f64_factor_bound(N, got, ref, f64):
    """The float-float path may err by the ratio of unit roundoffs (2^-47 / 2^-53 = 64)
    times the plain float64 dense solve's error on the same inputs, plus the scalar
    products' own rounding."""
    e_got = np.abs(got - ref).max(axis=1)
    e_64 = np.abs(f64 - ref).max(axis=1)
    floor = 8 * (int(np.log2(N)) + 2) * U_DF * np.abs(ref).max(axis=1)
    return e_got, 64 * e_64.max() + floor


@pytest.mark.parametrize("N", [8, 64, 96, 192, 256, 512, 768, 1024])
@pytest.mark.parametrize("space", tr.SPACES)
def test_forward_matches_refined_projection(N, space):
    """Random values (not in the space) against the refined projection: the conditioning
    of B (biharmonic: ~1e9 at N = 1024) shows in every float64 or float-float solve."""
    with Plan(N, 4, 4, 1 / 180, 1e-3) as plan:
        X = _values(plan.n_modes, N, seed=N + 9)
        Uh = _run(plan, "forward", space, X)
    e, tol = _f64_factor_bound(N, Uh, tr.forward_ref(space, X), tr.forward(space, X))
    assert np.all(e <= tol), (e.max(), tol.min())


@pytest.mark.parametrize("N", [8, 64, 96, 1024, 1536])
@pytest.mark.parametrize("space", tr.SPACES)
def test_forward_inverts_inverse(N, space):
    """Coefficients of the workload's spectrum -> values (longdouble oracle, rounded to
    float64) -> GPU forward: back to the coefficients."""
    with Plan(N, 4, 4, 1 / 180, 1e-3) as plan:
        C = inputs.rhs_numpy(plan.n_modes, N, seed=N + 11)
        C[:, tr.dim(space, N):] = 0
        U = tr.inverse_ref(space, C)
        Ch = _run(plan, "forward", space, U)
    e, tol = _f64_factor_bound(N, Ch, C, tr.forward(space, U))
    assert np.all(e <= tol), (e.max(), tol.min())
    if space != "biharmonic" or N <= 64:
        assert np.all(e <= 1e-12 * np.abs(C).max(axis=1))


@pytest.mark.parametrize("kind", ["inverse", "scalar", "forward"])
def test_in_place_equals_out_of_place(kind):
    import torch
    N = 64
    with Plan(N, 6, 4, 1 / 180, 1e-3) as plan:
        x = torch.as_tensor(_values(plan.n_modes, N, seed=3), device="cuda")
        y = plan.transform(kind, "dirichlet", x)
        x2 = x.clone()
        plan.transform(kind, "dirichlet", x2, out=x2)
        torch.cuda.synchronize()
        assert torch.equal(y, x2)


def test_largest_N():
    N = 4096
    with Plan(N, 2, 2, 1 / 180, 1e-3) as plan:
        C = inputs.rhs_numpy(plan.n_modes, N, seed=41)
        U = _run(plan, "inverse", "dirichlet", C)
        S = _run(plan, "scalar", "dirichlet", U)
    Cs = C.copy()
    Cs[:, N - 2:] = 0
    ref = tr.inverse_ref("dirichlet", Cs[:1])[0]
    assert np.abs(U[0] - ref).max() <= _bound(N, Cs[0], weight=2.0)
    sref = tr.scalar_ref("dirichlet", U[:1])[0]
    assert np.abs(S[0] - sref).max() <= _bound(N, U[0], scale=np.pi / N, weight=2.0)


@pytest.mark.parametrize("space", tr.SPACES)
def test_largest_N_forward(space):
    """N = 4096, where each thread of the least-squares mass solve owns a run of 32
    frequencies: coefficients of the workload's spectrum -> values (longdouble oracle,
    rounded to float64) -> GPU forward, back to the coefficients."""
    N = 4096
    with Plan(N, 2, 2, 1 / 180, 1e-3) as plan:
        C = inputs.rhs_numpy(plan.n_modes, N, seed=43)
        C[:, tr.dim(space, N):] = 0
        U = np.repeat(tr.inverse_ref(space, C[:1]), plan.n_modes, axis=0)
        Ch = _run(plan, "forward", space, U)
    assert np.all(Ch[1:] == Ch[0])                      # identical columns, identical results
    e, tol = _f64_factor_bound(N, Ch[:1], C[:1], tr.forward(space, U[:1]))
    assert np.all(e <= tol), (e.max(), tol.min())
    if space != "biharmonic":
        assert np.all(e <= 1e-12 * np.abs(C[:1]).max(axis=1))


def test_full_size_sampled():
    """The benchmark's workload (N = 1024, 1024 x 1024 grid, one launch per transform),
    checked on sampled modes."""
    import torch
    N, Nx, Nz = 1024, 1024, 1024
    with Plan(N, Nx, Nz, 1 / 2000, 1e-4, df_only=True) as plan:
        c = inputs.rhs_torch(plan.n_modes, N, seed=5)
        u = plan.transform("inverse", "dirichlet", c)
        s = plan.transform("scalar", "biharmonic", u)
        modes = inputs.sample_modes(plan.n_modes, 2e-5, seed=5, must_include=(0, plan.n_modes - 1))
        C, U, S = c[modes].cpu().numpy(), u[modes].cpu().numpy(), s[modes].cpu().numpy()
        del c, u, s
        torch.cuda.empty_cache()
    Cs = C.copy()
    Cs[:, N - 2:] = 0
    Uref = tr.inverse_ref("dirichlet", Cs)
    Sref = tr.scalar_ref("biharmonic", U)
    for i in range(len(modes)):
        assert np.abs(U[i] - Uref[i]).max() <= _bound(N, Cs[i], weight=2.0), modes[i]
        assert np.abs(S[i] - Sref[i]).max() <= _bound(N, U[i], scale=np.pi / N, weight=4.0), modes[i]


def test_unsupported_plans():
    import torch
    with Plan(80, 4, 4, 1 / 180, 1e-3) as plan:             # N neither 2^p nor 3 2^p
        x = torch.zeros((plan.n_modes, 80), dtype=torch.complex128, device="cuda")
        with pytest.raises(ShenError) as e:
            plan.transform("inverse", "dirichlet", x)
        assert e.value.status == 5
    with Plan(64, 4, 4, 1 / 180, 1e-3, gl=True) as plan:    # Gauss-Lobatto points, N - 1 = 63
        x = torch.zeros((plan.n_modes, 64), dtype=torch.complex128, device="cuda")
        with pytest.raises(ShenError) as e:
            plan.transform("scalar", "chebyshev", x)
        assert e.value.status == 5


# ---------------------------------------------------------------------------
# Gauss-Lobatto points (N - 1 a power of two): DCT-I through the even extension
# ---------------------------------------------------------------------------

GL_N = [9, 17, 25, 65, 97, 129, 1025]


@pytest.mark.parametrize("N", GL_N)
@pytest.mark.parametrize("space", tr.SPACES)
def test_gl_inverse_and_scalar_match_oracle(N, space):
    with Plan(N, 4, 4, 1 / 180, 1e-3, gl=True) as plan:
        C = inputs.rhs_numpy(plan.n_modes, N, seed=N + 13)
        X = _values(plan.n_modes, N, seed=N + 14)
        U = _run(plan, "inverse", space, C)
        S = _run(plan, "scalar", space, X)
    Cs = C.copy()
    Cs[:, tr.dim(space, N):] = 0
    Uref = tr.inverse_ref(space, Cs, gl=True)
    Sref = tr.scalar_ref(space, X, gl=True)
    for m in range(C.shape[0]):
        assert np.abs(U[m] - Uref[m]).max() <= _bound(N - 1, Cs[m], weight=WEIGHT[space]), m
        # GL weights pi / (N - 1), half at the ends
        assert np.abs(S[m] - Sref[m]).max() <= _bound(N - 1, X[m], scale=np.pi / (N - 1), weight=WEIGHT[space]), m
        assert np.all(S[m, tr.dim(space, N):] == 0)


@pytest.mark.parametrize("N", [9, 25, 65, 97, 257, 513, 769, 1025])
@pytest.mark.parametrize("space", tr.SPACES)
def test_gl_forward_matches_refined_projection(N, space):
    with Plan(N, 4, 4, 1 / 180, 1e-3, gl=True) as plan:
        X = _values(plan.n_modes, N, seed=N + 15)
        Uh = _run(plan, "forward", space, X)
        C = inputs.rhs_numpy(plan.n_modes, N, seed=N + 16)
        C[:, tr.dim(space, N):] = 0
        V = tr.inverse_ref(space, C, gl=True)
        Ch = _run(plan, "forward", space, V)
    e, tol = _f64_factor_bound(N - 1, Uh, tr.forward_ref(space, X, gl=True), tr.forward(space, X, gl=True))
    assert np.all(e <= tol), (e.max(), tol.min())
    e, tol = _f64_factor_bound(N - 1, Ch, C, tr.forward(space, V, gl=True))
    assert np.all(e <= tol), (e.max(), tol.min())


@pytest.mark.parametrize("gl", [False, True])
def test_transform_shards_equal_full(gl):
    """shen_transform_modes on mode ranges (shards) gives the full transform's columns."""
    import torch
    N = 65 if gl else 64
    with Plan(N, 12, 10, 1 / 180, 1e-3, gl=gl) as plan:
        x = torch.as_tensor(_values(plan.n_modes, N, seed=77), device="cuda")
        for kind in ("inverse", "scalar", "forward"):
            full = plan.transform(kind, "biharmonic", x)
            parts = [plan.transform_modes(kind, "biharmonic", a, x[a:b].contiguous())
                     for a, b in ((0, 7), (7, 30), (30, plan.n_modes))]
            torch.cuda.synchronize()
            assert torch.equal(torch.cat(parts), full), kind
        with pytest.raises(ShenError):
            plan.transform_modes("inverse", "dirichlet", plan.n_modes - 2, x[:5].contiguous())
