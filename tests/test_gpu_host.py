"""GPU tests of solves on host fields (chunked copy-in / solve / copy-out pipeline).

The pipeline runs the same kernels on the same modes as the device-resident solve, so
its result must equal that solve bit for bit, whether the field fits one staging slot
or spans several (slots reused within a call and across calls), in place or not, from
pinned or pageable host memory.  A few modes are also checked against the O(N) oracle.
"""
import numpy as np
import pytest

from oracle import on
from oracle import solve as so
from paper_1701_03787_gb300 import Plan, ShenError, inputs

pytestmark = pytest.mark.gpu

PRECISIONS = {"helmholtz": ["fp64", "df_r1", "df"], "biharmonic": ["fp64", "df"]}
CASES = [(p, q) for p in PRECISIONS for q in PRECISIONS[p]]


def _device_solve(plan, problem, f_host, precision):
    import torch
    f = f_host.to("cuda")
    u = plan.solve(problem, f, precision=precision)
    torch.cuda.synchronize()
    return u.cpu()


@pytest.mark.parametrize("problem,precision", CASES)
def test_host_solve_equals_device_solve_small(problem, precision):
    import torch
    with Plan(130, 12, 10, 1 / 180, 1e-3) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=31, device="cpu").pin_memory()
        u = plan.solve_host(problem, f, precision=precision)
        torch.cuda.synchronize()
        ref = _device_solve(plan, problem, f, precision)
        assert torch.equal(u, ref)
        # a few columns against the paper's O(N) algorithm (float64 oracle)
        z2 = so.mode_z2(12, 10)
        c = so.c_of(1 / 180, 1e-3)
        modes = [0, 7, plan.n_modes - 1]
        F = f.numpy()[modes]
        U = on.solve_modes(problem, 130, z2[modes], c, F)
        err = np.abs(u.numpy()[modes] - U).max() / np.abs(U).max()
        assert err < (1e-12 if precision == "fp64" else 1e-10)


@pytest.mark.parametrize("problem,precision", [("helmholtz", "df_r1"), ("biharmonic", "df"),
                                               ("biharmonic", "fp64")])
def test_host_solve_multi_chunk_in_place_and_repeated(problem, precision):
    import torch
    # N = 1024 on a 256 x 256 grid: 33,024 modes, 541 MB per field, three staging chunks
    with Plan(1024, 256, 256, 1 / 2000, 1e-4) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=32, device="cpu").pin_memory()
        ref = _device_solve(plan, problem, f, precision)
        u1 = plan.solve_host(problem, f, precision=precision)
        u2 = plan.solve_host(problem, f, precision=precision)     # slots reused across calls
        g = f.clone().pin_memory()
        plan.solve_host(problem, g, g, precision=precision)        # in place
        torch.cuda.synchronize()
        assert torch.equal(u1, ref)
        assert torch.equal(u2, ref)
        assert torch.equal(g, ref)
        _, _, _, dev_bytes = plan.info()
        assert dev_bytes > 3 * (256 << 20) - 1


def test_host_solve_pageable_memory_and_two_streams():
    import torch
    with Plan(257, 64, 48, 1 / 2000, 1e-4) as plan:
        fh = inputs.rhs_torch(plan.n_modes, plan.N, seed=33, device="cpu")            # pageable
        fb = inputs.rhs_torch(plan.n_modes, plan.N, seed=34, device="cpu").pin_memory()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        uh = plan.solve_host("helmholtz", fh, precision="df", stream=s1)
        ub = plan.solve_host("biharmonic", fb, precision="df", stream=s2)
        s1.synchronize()
        s2.synchronize()
        assert torch.equal(uh, _device_solve(plan, "helmholtz", fh, "df"))
        assert torch.equal(ub, _device_solve(plan, "biharmonic", fb, "df"))


def test_host_solve_rejections():
    import torch
    with Plan(64, 8, 8, 1 / 180, 1e-3) as plan:
        f = inputs.rhs_torch(plan.n_modes, plan.N, seed=35, device="cpu")
        with pytest.raises(ValueError):
            plan.solve_host("helmholtz", f.to("cuda"))
        with pytest.raises(ValueError):
            plan.solve_host("helmholtz", f[:-1])
        with pytest.raises(ShenError):
            plan.solve_host("biharmonic", f, precision="df_r1")        # no mixed biharmonic path
