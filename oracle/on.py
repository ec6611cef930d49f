"""Loader for ``shen_on.c``, the paper's O(N) algorithms in plain C (oracle, test infrastructure).

``build()`` compiles the C file with gcc into ``oracle/_build/`` (git-ignored);
the loader builds on first use when the library is missing.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "shen_on.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libshen_on.so")

_lib = None


def build(force=False):
    """Compile shen_on.c (gcc, OpenMP) into oracle/_build/libshen_on.so."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        P = ctypes.c_void_p
        _lib.on_helmholtz_solve.argtypes = [i, d, P, P, P]
        _lib.on_biharmonic_solve.argtypes = [i, d, d, P, P, P]
        _lib.on_biharmonic_solve_dense_lu.argtypes = [i, d, d, P, P, P]
        _lib.on_helmholtz_solve_modes.argtypes = [i, l, P, P, P]
        _lib.on_biharmonic_solve_modes.argtypes = [i, l, P, P, P, P]
        _lib.on_set_threads.argtypes = [i]
        _lib.on_set_threads.restype = None
        for f in ("on_helmholtz_solve", "on_biharmonic_solve", "on_biharmonic_solve_dense_lu",
                  "on_helmholtz_solve_modes", "on_biharmonic_solve_modes", "on_max_threads"):
            getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def max_threads():
    return int(lib().on_max_threads())


def set_threads(n):
    """Threads of the mode batches (OpenMP); returns the previous count."""
    prev = max_threads()
    lib().on_set_threads(int(n))
    return prev


def solve_modes(problem, N, z2, c, F):
    """O(N) solves of every mode: F complex128 (n_modes, N) -> U complex128 (n_modes, N)."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    n_modes = F.shape[0]
    assert F.shape[1] == N
    U = np.zeros_like(F)
    z2 = np.ascontiguousarray(z2, dtype=np.float64)
    if problem == "helmholtz":
        alpha = np.ascontiguousarray(z2 + c)
        rc = lib().on_helmholtz_solve_modes(N, n_modes, _ptr(alpha), _ptr(F), _ptr(U))
    else:
        a = np.ascontiguousarray(-(2.0 * z2 + c))
        b = np.ascontiguousarray(z2 * (z2 + c))
        rc = lib().on_biharmonic_solve_modes(N, n_modes, _ptr(a), _ptr(b), _ptr(F), _ptr(U))
    if rc != 0:
        raise ValueError(f"O(N) oracle rejected N={N}")
    return U


def biharmonic_dense_lu(N, z2, c, f):
    """One mode by Algorithm LUbiharmonic with the dense U of the printed algorithm."""
    f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128)[:N])
    f = np.concatenate([f, np.zeros(N - f.size, complex)]) if f.size < N else f
    u = np.zeros(N, np.complex128)
    n = N - 4
    work = np.zeros(n * n + 9 * n)
    rc = lib().on_biharmonic_solve_dense_lu(N, -(2.0 * z2 + c), z2 * (z2 + c), _ptr(f), _ptr(u), _ptr(work))
    if rc != 0:
        raise ValueError(f"N={N} too small")
    return u
