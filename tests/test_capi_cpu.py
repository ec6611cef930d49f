"""The C ABI library builds, loads and exports what include/shensolve.h declares (CPU only).

No call here reaches the GPU: only argument validation paths that return before
any CUDA call, and the static helpers.
"""
import ctypes
import shutil

import pytest

nvcc_missing = shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def L():
    if nvcc_missing:
        pytest.skip("no CUDA toolkit")
    from paper_1701_03787_gb300 import build
    build.build()
    from paper_1701_03787_gb300 import binding
    return binding.lib()


def test_exports_every_declared_symbol(L):
    from paper_1701_03787_gb300 import binding
    declared = binding.declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(L, name), name


def test_status_strings_and_version(L):
    from paper_1701_03787_gb300 import binding
    assert L.shen_version() >= 100
    assert binding.status_string(0) == "ok"
    for s in range(1, 6):
        assert binding.status_string(s) != "unknown status"
    assert binding.status_string(99) == "unknown status"


@pytest.mark.parametrize("args", [
    (7, 32, 32, 1e-3, 1e-3),        # N below 8
    (8193, 32, 32, 1e-3, 1e-3),     # N above 8192
    (64, 31, 32, 1e-3, 1e-3),       # odd Nx
    (64, 32, 0, 1e-3, 1e-3),        # Nz < 2
    (64, 32, 32, 0.0, 1e-3),        # nu = 0
    (64, 32, 32, 1e-3, -1.0),       # dt < 0
    (64, 32, 32, float("nan"), 1e-3),
])
def test_plan_create_rejects_bad_arguments(L, args):
    h = ctypes.c_void_p()
    N, Nx, Nz, nu, dt = args
    st = L.shen_plan_create(ctypes.byref(h), N, Nx, Nz, nu, dt, 6.283185307179586, 3.141592653589793, 0, None)
    assert st == 1
    assert not h.value


def test_null_plan_and_pointers_rejected(L):
    assert L.shen_helmholtz_solve(None, None, None, 0, None) == 1
    assert L.shen_biharmonic_solve(None, None, None, 0, None) == 1
    assert L.shen_rhs_matvec(None, 0, None, None, 0.0, None, None) == 1
    assert L.shen_rhs_matvec_ex(None, 0, None, None, 0.0, None, 5, None) == 1
    assert L.shen_residual(None, 0, None, None, None, None) == 1
    assert L.shen_velocity(None, None, None, None, None, None, 5, None) == 1
    assert L.shen_mass_matvec(None, 0, None, None, 0.0, None, None) == 1
    assert L.shen_linear_step(None, None, None, None, None, None, None, None, None, 5, None) == 1
    assert L.shen_last_error_detail(None, None, None) == 1
    assert L.shen_rhs_matvec_ex(None, 0, None, None, 0.0, None, 3, None) == 5     # no such path
    assert L.shen_rhs_matvec_ex(None, 0, None, None, 0.0, None, 99, None) == 1
    assert L.shen_solve_host(None, 0, None, None, 0, None) == 1
    assert L.shen_plan_autotune(None, 0, None, None, None, None, None) == 1
    assert L.shen_batch_autotune(None, 0, None, None, None, None, None) == 1
    assert L.shen_plan_info(None, None, None, None, None) == 1
    L.shen_plan_destroy(None)
    z = (ctypes.c_double * 2)(0.0, -1.0)
    h = ctypes.c_void_p()
    assert L.shen_plan_create_z2(ctypes.byref(h), 64, 2, ctypes.cast(z, ctypes.c_void_p), 1e-3, 1e-3, 0, None) == 1
    for bad_flags in (8, 9, 0x80000000):                                                  # unknown flags
        assert L.shen_plan_create(ctypes.byref(h), 64, 32, 32, 1e-3, 1e-3, 6.28, 3.14, bad_flags, None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1701_03787_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        binding.lib()
