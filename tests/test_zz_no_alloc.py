"""The no-allocation batched solve, called through the C ABI (collected last).

shen_batch_solve_noalloc serves callers that cannot allocate device memory at solve
time, for example an application whose device memory is divided up in advance by its
own pool allocator.  It must give the same result as shen_batch_solve, bit for bit (same
arithmetic; only where the forward sweep's intermediate is kept differs), and that result
must meet the oracle's bars.  Two calls in a row check that the fixed scratch shared
between calls (its work-queue counter) is reset by every call, and an in-place call
(u == f) checks the path where the float-float sweep keeps its intermediate in the output
column, over the input rows.
"""
import ctypes

import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import BatchPlan, binding, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df": 1e-10}
INSTS = [dict(N=64, Nx=8, Nz=8, nu=1 / 180, dt=1e-3), dict(N=129, Nx=4, Nz=6, nu=1e-3, dt=5e-4),
         dict(N=9, Nx=2, Nz=4, nu=1e-2, dt=1e-2), dict(N=256, Nx=16, Nz=8, nu=1 / 2000, dt=1e-4)]


def _noalloc(bp, problem, precision, f, u):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = binding.lib().shen_batch_solve_noalloc(bp._h, binding.PROBLEMS[problem], ctypes.c_void_p(f.data_ptr()),
                                                ctypes.c_void_p(u.data_ptr()), binding.PRECISIONS[precision],
                                                stream)
    assert st == 0, binding.status_string(st)
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_noalloc_matches_batch_solve_twice(problem, precision):
    import torch
    with BatchPlan(INSTS) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, INSTS, seed=11)
        F = f.cpu().numpy()
        R = bp.solve(problem, f, precision=precision).cpu().numpy()
        outs = []
        for _ in range(2):
            u = torch.full_like(f, complex(np.nan, np.nan))
            _noalloc(bp, problem, precision, f, u)
            outs.append(u.cpu().numpy())
        g = f.clone()                                            # in place: u == f
        _noalloc(bp, problem, precision, g, g)
        outs.append(g.cpu().numpy())
        offsets = list(bp.offsets)
    for U in outs:
        assert np.array_equal(U, R)
    # the oracle's O(N) solves of every instance (the paper's algorithm in float64)
    for i, inst in enumerate(INSTS):
        N = inst["N"]
        n = so.n_unknowns(problem, N)
        z2 = so.mode_z2(inst["Nx"], inst["Nz"])
        Fi = F[offsets[i]:offsets[i + 1]].reshape(-1, N)
        Ui = outs[-1][offsets[i]:offsets[i + 1]].reshape(-1, N)
        Ri = on.solve_modes(problem, N, z2, so.c_of(inst["nu"], inst["dt"]), Fi)
        for m in range(Ri.shape[0]):
            assert so.rel_l2(Ui[m, :n], Ri[m, :n]) <= TOL[precision], (i, m)
            assert np.all(Ui[m, n:] == 0)
