"""The no-allocation batched solve, called through the C ABI (collected last).

shen_batch_solve_noalloc serves callers that cannot allocate device memory at solve
time (for example while a stream is captured into a CUDA graph, or under a pool
allocator that owns all device memory).  It must give the same result as
shen_batch_solve; two calls in a row check that the fixed scratch it shares between
calls (its work-queue counter) is reset by every call.
"""
import ctypes

import numpy as np
import pytest

from oracle import solve as so
from paper_1701_03787_gb300 import BatchPlan, binding, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df": 1e-10}


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem", ["helmholtz", "biharmonic"])
def test_noalloc_matches_batch_solve_twice(problem, precision):
    import torch
    insts = [dict(N=64, Nx=8, Nz=8, nu=1 / 180, dt=1e-3), dict(N=129, Nx=4, Nz=6, nu=1e-3, dt=5e-4),
             dict(N=9, Nx=2, Nz=4, nu=1e-2, dt=1e-2), dict(N=256, Nx=16, Nz=8, nu=1 / 2000, dt=1e-4)]
    L = binding.lib()
    prob = binding.PROBLEMS[problem]
    prec = binding.PRECISIONS[precision]
    with BatchPlan(insts) as bp:
        f = inputs.batch_rhs_torch(bp.offsets, insts, seed=11)
        ref = bp.solve(problem, f, precision=precision)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        outs = []
        for _ in range(2):
            u = torch.full_like(f, complex(np.nan, np.nan))
            st = L.shen_batch_solve_noalloc(bp._h, prob,
                                            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                            prec, stream)
            assert st == 0, binding.status_string(st)
            torch.cuda.synchronize()
            outs.append(u.cpu().numpy())
        R = ref.cpu().numpy()
    for U in outs:
        for i, inst in enumerate(insts):
            N = inst["N"]
            n = so.n_unknowns(problem, N)
            Ui = U[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N)
            Ri = R[bp.offsets[i]:bp.offsets[i + 1]].reshape(-1, N)
            for m in range(Ri.shape[0]):
                assert so.rel_l2(Ui[m, :n], Ri[m, :n]) <= TOL[precision], (i, m)
                assert np.all(Ui[m, n:] == 0)
