"""GPU parity of the on-chip float-float sweeps (shapes 2 and 3 of the float-float solves:
one lane per real chain, the forward result kept in Tensor Memory and shared memory, the
rest spilled to global memory).

- every mode against the refined reference (``oracle.structured.solve_ref``) at the
  reduced-precision bar, 1e-10 per mode, and against the paper's O(N) algorithm in
  float64 (``shen_on.c``) at the same bar;
- shape 2 (Tensor Memory + shared + global) equals shape 3 (shared + global) bit for bit:
  the arithmetic is the same, only where y is kept differs;
- in place (u == f) and mode ranges (shen_solve_modes, the mode order instead of the
  class order) give the same bits as the whole-plan call.
Sizes cover every split of y: N = 8 and 64 (all on chip), 129 (odd N: the parity chains
differ in length), 1024 (all three tiers), 4096 and 8192 (mostly spilled)."""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from oracle import structured as st
from paper_1701_03787_gb300 import Plan, ShenError, inputs

pytestmark = pytest.mark.gpu

CASES = [(8, 4, 6, 1e-2, 1e-2), (64, 32, 32, 1 / 180, 1e-3), (129, 8, 6, 1e-3, 5e-4),
         (1024, 64, 64, 1 / 2000, 1e-4), (4096, 6, 8, 1 / 2000, 1e-4), (8192, 4, 4, 1 / 2000, 1e-4)]


@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
@pytest.mark.parametrize("N,Nx,Nz,nu,dt", CASES)
def test_onchip_shapes(problem, N, Nx, Nz, nu, dt):
    import torch
    c = so.c_of(nu, dt)
    z2 = so.mode_z2(Nx, Nz)
    with Plan(N, Nx, Nz, nu, dt) as plan:
        f = inputs.rhs_torch(plan.n_modes, N, seed=N + 5)
        F = f.cpu().numpy()
        out = {}
        for shape in (3, 2):
            plan.set_shape(problem, shape)
            out[shape] = plan.solve(problem, f, precision="df").cpu().numpy()
        g = f.clone()
        plan.solve(problem, g, u=g, precision="df")                       # in place, shape 2
        inplace = g.cpu().numpy()
        half = plan.n_modes // 2
        parts = [plan.solve_modes(problem, 0, f[:half].contiguous(), precision="df"),
                 plan.solve_modes(problem, half, f[half:].contiguous(), precision="df")]
        ranged = torch.cat(parts).cpu().numpy()
        plan.set_shape(problem, 0)
    assert np.array_equal(out[2], out[3])
    assert np.array_equal(inplace, out[2])
    assert np.array_equal(ranged, out[2])
    n = so.n_unknowns(problem, N)
    R = st.solve_ref(problem, N, z2, c, F)
    C = on.solve_modes(problem, N, z2, c, F)
    U = out[2]
    assert np.all(U[:, n:] == 0)
    for m in range(plan.n_modes):
        assert so.rel_l2(U[m, :n], R[m, :n]) <= 1e-10, m
        assert so.rel_l2(U[m, :n], C[m, :n]) <= 1e-10, m


def test_onchip_shapes_refuse_wall_first():
    with Plan(64, 8, 8, 1 / 180, 1e-3, wall_first=True) as plan:
        for shape in (2, 3):
            with pytest.raises(ShenError) as e:
                plan.set_shape("biharmonic", shape)
            assert e.value.status == 5
