"""Thin Python binding of libshensolve (ctypes; argument marshalling only).

Every operation runs in the library's CUDA kernels; this module only converts
arguments (tensor data pointers, stream handles, enums) and raises on a non-OK
status.  It never computes anything itself and has no fallback: if the library
is missing, importing it raises.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libshensolve.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "shensolve.h")

SHEN_OK, SHEN_ERR_ARG, SHEN_ERR_ALLOC, SHEN_ERR_CUDA, SHEN_ERR_SINGULAR, SHEN_ERR_UNSUPPORTED = range(6)
SHEN_HELMHOLTZ, SHEN_BIHARMONIC = 0, 1
SHEN_PLAN_DF_ONLY, SHEN_PLAN_GL, SHEN_PLAN_WALL_FIRST = 1, 2, 4
PRECISIONS = {"fp64": 0, "fp32_r1": 1, "fp32_r2": 2, "df_r1": 3, "df_r2": 4, "df": 5, "auto": 6, "fp64_r1": 7}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}
PROBLEMS = {"helmholtz": SHEN_HELMHOLTZ, "biharmonic": SHEN_BIHARMONIC}
SPACES = {"chebyshev": 0, "dirichlet": 1, "biharmonic": 2}
TRANSFORMS = {"inverse": 0, "scalar": 1, "forward": 2}

_lib = None


class ShenError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


def lib():
    """Load libshensolve.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libshensolve.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, Lg = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    sig = {
        "shen_plan_create": ([P, I, I, I, D, D, D, D, ctypes.c_uint, P], I),
        "shen_plan_create_z2": ([P, I, Lg, P, D, D, ctypes.c_uint, P], I),
        "shen_helmholtz_solve": ([P, P, P, I, P], I),
        "shen_biharmonic_solve": ([P, P, P, I, P], I),
        "shen_solve_modes": ([P, I, Lg, Lg, P, P, I, P], I),
        "shen_rhs_matvec": ([P, I, P, P, D, P, P], I),
        "shen_rhs_matvec_ex": ([P, I, P, P, D, P, I, P], I),
        "shen_residual": ([P, I, P, P, P, P], I),
        "shen_transform": ([P, I, I, P, P, P], I),
        "shen_transform_modes": ([P, I, I, Lg, Lg, P, P, P], I),
        "shen_solve_refine": ([P, I, P, P, P, I, I, P], I),
        "shen_plan_set_shape": ([P, I, I], I),
        "shen_plan_get_shape": ([P, I, P], I),
        "shen_velocity": ([P, P, P, P, P, P, I, P], I),
        "shen_mass_matvec": ([P, I, P, P, D, P, P], I),
        "shen_linear_step": ([P, P, P, P, P, P, P, P, P, I, P], I),
        "shen_last_error_detail": ([P, P, P], I),
        "shen_solve_host": ([P, I, P, P, I, P], I),
        "shen_plan_info": ([P, P, P, P, P], I),
        "shen_plan_check": ([P, P], I),
        "shen_plan_destroy": ([P], None),
        "shen_batch_plan_create": ([P, I, P, ctypes.c_uint, P], I),
        "shen_batch_info": ([P, P, P, P, P], I),
        "shen_batch_offsets": ([P, P], I),
        "shen_batch_solve": ([P, I, P, P, I, P], I),
        "shen_batch_check": ([P], I),
        "shen_batch_solve_noalloc": ([P, I, P, P, I, P], I),
        "shen_batch_solve_host": ([P, I, P, P, I, P], I),
        "shen_batch_autotune": ([P, I, P, P, P, P, P], I),
        "shen_plan_autotune": ([P, I, P, P, P, P, P], I),
        "shen_batch_destroy": ([P], None),
        "shen_status_string": ([I], ctypes.c_char_p),
        "shen_version": ([], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def declared_symbols():
    """Names of the functions declared in include/shensolve.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(shen_[a-z0-9_]+)\s*\(", text)))


def status_string(status):
    return lib().shen_status_string(int(status)).decode()


def check(status, what):
    if status != SHEN_OK:
        raise ShenError(status, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _prec(precision):
    if isinstance(precision, str):
        return PRECISIONS[precision]
    return int(precision)


def _problem(problem):
    if isinstance(problem, str):
        return PROBLEMS[problem]
    return int(problem)


def _field_ok(t, n_modes, N, name):
    import torch
    if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
    if t.numel() != n_modes * N:
        raise ValueError(f"{name} has {t.numel()} entries, expected n_modes*N = {n_modes * N}")


class Plan:
    """One channel's plan (C type shen_plan_t).  Fields are complex128 CUDA tensors of
    shape (n_modes, N) in mode-major order."""

    def __init__(self, N, Nx=None, Nz=None, nu=None, dt=None, Lx=None, Lz=None, z2=None, stream=None,
                 df_only=False, gl=False, wall_first=False):
        import math
        self._h = ctypes.c_void_p()
        if z2 is not None:
            import numpy as np
            z = np.ascontiguousarray(np.asarray(z2, dtype=np.float64))
            st = lib().shen_plan_create_z2(ctypes.byref(self._h), int(N), int(z.size),
                                           z.ctypes.data_as(ctypes.c_void_p), float(nu), float(dt),
                                           (SHEN_PLAN_DF_ONLY if df_only else 0) | (SHEN_PLAN_GL if gl else 0)
                                           | (SHEN_PLAN_WALL_FIRST if wall_first else 0),
                                           _stream(stream))
        else:
            Lx = 2 * math.pi if Lx is None else Lx
            Lz = math.pi if Lz is None else Lz
            st = lib().shen_plan_create(ctypes.byref(self._h), int(N), int(Nx), int(Nz), float(nu), float(dt),
                                        float(Lx), float(Lz),
                                        (SHEN_PLAN_DF_ONLY if df_only else 0) | (SHEN_PLAN_GL if gl else 0)
                                           | (SHEN_PLAN_WALL_FIRST if wall_first else 0),
                                        _stream(stream))
        check(st, "shen_plan_create")
        n_modes, n_classes, n = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        nbytes = ctypes.c_longlong()
        check(lib().shen_plan_info(self._h, ctypes.byref(n_modes), ctypes.byref(n_classes), ctypes.byref(n),
                                   ctypes.byref(nbytes)), "shen_plan_info")
        self.N, self.n_modes, self.n_classes, self.device_bytes = n.value, n_modes.value, n_classes.value, nbytes.value

    @property
    def handle(self):
        return self._h

    def info(self):
        """(n_modes, n_classes, N, device_bytes); device_bytes includes host-solve staging."""
        n_modes, n_classes, n = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        nbytes = ctypes.c_longlong()
        check(lib().shen_plan_info(self._h, ctypes.byref(n_modes), ctypes.byref(n_classes), ctypes.byref(n),
                                   ctypes.byref(nbytes)), "shen_plan_info")
        return n_modes.value, n_classes.value, n.value, nbytes.value

    def close(self):
        if self._h:
            lib().shen_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _solve(self, fn, name, f, u, precision, stream):
        import torch
        _field_ok(f, self.n_modes, self.N, "f")
        if u is None:
            u = torch.empty_like(f)
        _field_ok(u, self.n_modes, self.N, "u")
        check(fn(self._h, _ptr(f), _ptr(u), _prec(precision), _stream(stream)), name)
        return u

    def helmholtz_solve(self, f, u=None, precision="fp64", stream=None):
        return self._solve(lib().shen_helmholtz_solve, "shen_helmholtz_solve", f, u, precision, stream)

    def biharmonic_solve(self, f, u=None, precision="fp64", stream=None):
        return self._solve(lib().shen_biharmonic_solve, "shen_biharmonic_solve", f, u, precision, stream)

    def solve(self, problem, f, u=None, precision="fp64", stream=None):
        if _problem(problem) == SHEN_HELMHOLTZ:
            return self.helmholtz_solve(f, u, precision, stream)
        return self.biharmonic_solve(f, u, precision, stream)

    def solve_modes(self, problem, mode_begin, f, u=None, precision="fp64", stream=None):
        """Solve the modes [mode_begin, mode_begin + f.shape[0]) (a shard)."""
        import torch
        count = f.numel() // self.N
        _field_ok(f, count, self.N, "f")
        if u is None:
            u = torch.empty_like(f)
        _field_ok(u, count, self.N, "u")
        check(lib().shen_solve_modes(self._h, _problem(problem), int(mode_begin), int(count), _ptr(f), _ptr(u),
                                     _prec(precision), _stream(stream)), "shen_solve_modes")
        return u

    def solve_host(self, problem, f, u=None, precision="fp64", stream=None):
        """Solve a field held in (preferably pinned) host memory; returns u (host).  The
        call is asynchronous on `stream` (default: the current stream); synchronise the
        stream before reading u."""
        import torch
        if f.dtype != torch.complex128 or f.is_cuda or not f.is_contiguous() or f.numel() != self.n_modes * self.N:
            raise ValueError("f must be a contiguous complex128 host tensor of n_modes*N entries")
        if u is None:
            u = torch.empty_like(f, pin_memory=f.is_pinned())
        if u.dtype != torch.complex128 or u.is_cuda or not u.is_contiguous() or u.numel() != f.numel():
            raise ValueError("u must be a contiguous complex128 host tensor shaped like f")
        check(lib().shen_solve_host(self._h, _problem(problem), _ptr(f), _ptr(u), _prec(precision),
                                    _stream(stream)), "shen_solve_host")
        return u

    def rhs_matvec(self, problem, x, y=None, beta=0.0, out=None, stream=None, precision="fp64"):
        import torch
        _field_ok(x, self.n_modes, self.N, "x")
        if y is not None:
            _field_ok(y, self.n_modes, self.N, "y")
        if out is None:
            out = torch.empty_like(x)
        _field_ok(out, self.n_modes, self.N, "out")
        check(lib().shen_rhs_matvec_ex(self._h, _problem(problem), _ptr(x), _ptr(y), float(beta), _ptr(out),
                                       _prec(precision), _stream(stream)), "shen_rhs_matvec_ex")
        return out

    def autotune(self, problem, f, u=None, stream=None):
        """Time the candidate paths of `problem` on the fields f (read) and u (overwritten)
        and record the fastest for precision "auto".  Returns (precision name, ms)."""
        import torch
        _field_ok(f, self.n_modes, self.N, "f")
        if u is None:
            u = torch.empty_like(f)
        _field_ok(u, self.n_modes, self.N, "u")
        chosen, ms = ctypes.c_int(), ctypes.c_float()
        check(lib().shen_plan_autotune(self._h, _problem(problem), _ptr(f), _ptr(u), ctypes.byref(chosen),
                                       ctypes.byref(ms), _stream(stream)), "shen_plan_autotune")
        return PRECISION_NAMES[chosen.value], ms.value

    def linear_step(self, u_old, g_old, load_u=None, load_g=None, out=None, precision="auto", stream=None):
        """One linear step: returns (u_new, g_new, v, w) (see shen_linear_step)."""
        import torch
        for t, nm in ((u_old, "u_old"), (g_old, "g_old")):
            _field_ok(t, self.n_modes, self.N, nm)
        for t, nm in ((load_u, "load_u"), (load_g, "load_g")):
            if t is not None:
                _field_ok(t, self.n_modes, self.N, nm)
        if out is None:
            out = tuple(torch.zeros_like(u_old) for _ in range(4))
        for t in out:
            _field_ok(t, self.n_modes, self.N, "out")
        u_new, g_new, v, w = out
        check(lib().shen_linear_step(self._h, _ptr(u_old), _ptr(g_old), _ptr(load_u), _ptr(load_g), _ptr(u_new),
                                     _ptr(g_new), _ptr(v), _ptr(w), _prec(precision), _stream(stream)),
              "shen_linear_step")
        return u_new, g_new, v, w

    def mass_matvec(self, problem, x, y=None, beta=0.0, out=None, stream=None):
        """out = B x + beta y with the problem space's mass matrix (float-float)."""
        import torch
        _field_ok(x, self.n_modes, self.N, "x")
        if y is not None:
            _field_ok(y, self.n_modes, self.N, "y")
        if out is None:
            out = torch.empty_like(x)
        _field_ok(out, self.n_modes, self.N, "out")
        check(lib().shen_mass_matvec(self._h, _problem(problem), _ptr(x), _ptr(y), float(beta), _ptr(out),
                                     _stream(stream)), "shen_mass_matvec")
        return out

    def velocity(self, u, g, v=None, w=None, f=None, precision="df", stream=None):
        """(v, w) from the wall-normal velocity u and g (Sec. 3, Eqs. ffin, f3, g3); f is
        written too when given.  Mode (0, 0) of v and w is left as passed in."""
        import torch
        _field_ok(u, self.n_modes, self.N, "u")
        _field_ok(g, self.n_modes, self.N, "g")
        if v is None:
            v = torch.zeros_like(u)
        if w is None:
            w = torch.zeros_like(u)
        _field_ok(v, self.n_modes, self.N, "v")
        _field_ok(w, self.n_modes, self.N, "w")
        if f is not None:
            _field_ok(f, self.n_modes, self.N, "f")
        check(lib().shen_velocity(self._h, _ptr(u), _ptr(g), _ptr(v), _ptr(w), _ptr(f), _prec(precision),
                                  _stream(stream)), "shen_velocity")
        return v, w

    def solve_refine(self, problem, f, u=None, work=None, steps=1, residual="fp64", stream=None):
        """Float32 sweeps plus `steps` refinement steps with a float64 ("fp64") or float-float
        ("df") residual (shen_solve_refine); returns u."""
        import torch
        _field_ok(f, self.n_modes, self.N, "f")
        u = torch.empty_like(f) if u is None else u
        work = torch.empty_like(f) if work is None else work
        _field_ok(u, self.n_modes, self.N, "u")
        _field_ok(work, self.n_modes, self.N, "work")
        check(lib().shen_solve_refine(self._h, _problem(problem), _ptr(f), _ptr(u), _ptr(work), int(steps),
                                      _prec(residual), _stream(stream)), "shen_solve_refine")
        return u

    def set_shape(self, problem, shape):
        """Shape (0..3) of the float-float sweeps of `problem` (see shen_plan_set_shape)."""
        check(lib().shen_plan_set_shape(self._h, _problem(problem), int(shape)), "shen_plan_set_shape")

    def shape(self, problem):
        v = ctypes.c_int()
        check(lib().shen_plan_get_shape(self._h, _problem(problem), ctypes.byref(v)), "shen_plan_get_shape")
        return v.value

    def transform(self, kind, space, x, out=None, stream=None):
        """Wall-normal transform of every mode column (see shen_transform): kind "inverse"
        (coefficients -> values at the Gauss points), "scalar" (values -> scalar products
        with the basis) or "forward" (values -> coefficients); space "chebyshev",
        "dirichlet" or "biharmonic".  out may be x (in place)."""
        import torch
        _field_ok(x, self.n_modes, self.N, "x")
        if out is None:
            out = torch.empty_like(x)
        _field_ok(out, self.n_modes, self.N, "out")
        k = TRANSFORMS[kind] if isinstance(kind, str) else int(kind)
        sp = SPACES[space] if isinstance(space, str) else int(space)
        check(lib().shen_transform(self._h, k, sp, _ptr(x), _ptr(out), _stream(stream)), "shen_transform")
        return out

    def transform_modes(self, kind, space, mode_begin, x, out=None, stream=None):
        """shen_transform on the modes [mode_begin, mode_begin + x.shape[0]) (a shard)."""
        import torch
        count = x.numel() // self.N
        _field_ok(x, count, self.N, "x")
        if out is None:
            out = torch.empty_like(x)
        _field_ok(out, count, self.N, "out")
        k = TRANSFORMS[kind] if isinstance(kind, str) else int(kind)
        sp = SPACES[space] if isinstance(space, str) else int(space)
        check(lib().shen_transform_modes(self._h, k, sp, int(mode_begin), int(count), _ptr(x), _ptr(out),
                                         _stream(stream)), "shen_transform_modes")
        return out

    def residual(self, problem, f, u, rel=None, stream=None):
        """Per-mode relative residual ||f - H u|| / ||f|| (float64 CUDA tensor of n_modes)."""
        import torch
        _field_ok(f, self.n_modes, self.N, "f")
        _field_ok(u, self.n_modes, self.N, "u")
        if rel is None:
            rel = torch.empty(self.n_modes, dtype=torch.float64, device=f.device)
        if rel.dtype != torch.float64 or not rel.is_cuda or not rel.is_contiguous() or rel.numel() != self.n_modes:
            raise ValueError("rel must be a contiguous float64 CUDA tensor of n_modes entries")
        check(lib().shen_residual(self._h, _problem(problem), _ptr(f), _ptr(u), _ptr(rel), _stream(stream)),
              "shen_residual")
        return rel

    def error_detail(self):
        """(largest relative residual of the last residual(), factorisations with a bad pivot)."""
        mx, ns = ctypes.c_double(), ctypes.c_long()
        check(lib().shen_last_error_detail(self._h, ctypes.byref(mx), ctypes.byref(ns)), "shen_last_error_detail")
        return mx.value, ns.value

    def check_device(self):
        where = ctypes.c_long()
        check(lib().shen_plan_check(self._h, ctypes.byref(where)), "shen_plan_check")


class InstanceDesc(ctypes.Structure):
    """C struct shen_instance_desc."""
    _fields_ = [("N", ctypes.c_int), ("Nx", ctypes.c_int), ("Nz", ctypes.c_int),
                ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("Lx", ctypes.c_double), ("Lz", ctypes.c_double)]


class BatchPlan:
    """Batched plan (C type shen_batch_t): many channels with uneven N in one launch.

    instances: sequence of dicts with keys N, Nx, Nz, nu, dt and optional Lx, Lz.
    The batched field is a flat complex128 CUDA tensor of ``field_elems`` entries;
    ``offsets[i]`` is where instance i's (n_modes_i, N_i) block starts."""

    def __init__(self, instances, stream=None, gl=False):
        import math
        descs = (InstanceDesc * len(instances))()
        for d, inst in zip(descs, instances):
            d.N, d.Nx, d.Nz = int(inst["N"]), int(inst["Nx"]), int(inst["Nz"])
            d.nu, d.dt = float(inst["nu"]), float(inst["dt"])
            d.Lx = float(inst.get("Lx", 2 * math.pi))
            d.Lz = float(inst.get("Lz", math.pi))
        self._h = ctypes.c_void_p()
        check(lib().shen_batch_plan_create(ctypes.byref(self._h), len(instances), ctypes.cast(descs, ctypes.c_void_p),
                                           SHEN_PLAN_GL if gl else 0, _stream(stream)), "shen_batch_plan_create")
        self.n_instances = len(instances)
        i = self.info()
        self.n_modes, self.field_elems, self.n_classes, self.device_bytes = (
            i["n_modes"], i["field_elems"], i["n_classes"], i["device_bytes"])
        offs = (ctypes.c_long * (len(instances) + 1))()
        check(lib().shen_batch_offsets(self._h, ctypes.cast(offs, ctypes.c_void_p)), "shen_batch_offsets")
        self.offsets = list(offs)

    def info(self):
        """dict of n_modes, field_elems, n_classes and device_bytes (the latter includes the
        host-solve staging once solve_host has run)."""
        n_modes, elems, ncls = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        nbytes = ctypes.c_longlong()
        check(lib().shen_batch_info(self._h, ctypes.byref(n_modes), ctypes.byref(elems), ctypes.byref(ncls),
                                    ctypes.byref(nbytes)), "shen_batch_info")
        return {"n_modes": n_modes.value, "field_elems": elems.value, "n_classes": ncls.value,
                "device_bytes": nbytes.value}

    def close(self):
        if self._h:
            lib().shen_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, problem, f, u=None, precision="fp64", stream=None):
        import torch
        if f.dtype != torch.complex128 or not f.is_cuda or not f.is_contiguous() or f.numel() != self.field_elems:
            raise ValueError(f"f must be a contiguous complex128 CUDA tensor of {self.field_elems} entries")
        if u is None:
            u = torch.empty_like(f)
        check(lib().shen_batch_solve(self._h, _problem(problem), _ptr(f), _ptr(u), _prec(precision),
                                     _stream(stream)), "shen_batch_solve")
        return u

    def solve_host(self, problem, f, u=None, precision="fp64", stream=None):
        """Solve a batched field held in (preferably pinned) host memory; returns u (host).
        Asynchronous on `stream` (default: the current stream); synchronise the stream
        before reading u."""
        import torch
        if f.dtype != torch.complex128 or f.is_cuda or not f.is_contiguous() or f.numel() != self.field_elems:
            raise ValueError(f"f must be a contiguous complex128 host tensor of {self.field_elems} entries")
        if u is None:
            u = torch.empty_like(f, pin_memory=f.is_pinned())
        if u.dtype != torch.complex128 or u.is_cuda or not u.is_contiguous() or u.numel() != f.numel():
            raise ValueError("u must be a contiguous complex128 host tensor shaped like f")
        check(lib().shen_batch_solve_host(self._h, _problem(problem), _ptr(f), _ptr(u), _prec(precision),
                                          _stream(stream)), "shen_batch_solve_host")
        return u

    def autotune(self, problem, f, u=None, stream=None):
        """As Plan.autotune, for the batched field."""
        import torch
        if f.dtype != torch.complex128 or not f.is_cuda or not f.is_contiguous() or f.numel() != self.field_elems:
            raise ValueError(f"f must be a contiguous complex128 CUDA tensor of {self.field_elems} entries")
        if u is None:
            u = torch.empty_like(f)
        chosen, ms = ctypes.c_int(), ctypes.c_float()
        check(lib().shen_batch_autotune(self._h, _problem(problem), _ptr(f), _ptr(u), ctypes.byref(chosen),
                                        ctypes.byref(ms), _stream(stream)), "shen_batch_autotune")
        return PRECISION_NAMES[chosen.value], ms.value

    def check_device(self):
        check(lib().shen_batch_check(self._h), "shen_batch_check")
