"""Thin ctypes binding of the C ABI in ``include/cbs.h`` (argument marshalling
only: every step of the solve runs in the CUDA library).

Device buffers are torch CUDA tensors: media float64 of shape (n[D-1], ..., n[0]),
fields/sources complex128 of shape (D+1, n[D-1], ..., n[0]).  The library must
have been built (``__graft_entry__.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build_lib

CBS_OK, CBS_EINVAL, CBS_ENOMEM, CBS_ECUDA, CBS_ENOCONV, CBS_EDIVERGED, CBS_ETIMEOUT = range(7)
CBS_FP64, CBS_FP32_REFINE, CBS_FP32 = 0, 1, 2
CBS_SHIFT_MIDRANGE, CBS_SHIFT_MEDIAN, CBS_SHIFT_MEC = 0, 1, 2
CBS_GRID_STAGGERED, CBS_GRID_COLLOCATED = 0, 1
PRECISIONS = {"fp64": CBS_FP64, "fp32_refine": CBS_FP32_REFINE, "fp32": CBS_FP32}
STATUS_NAMES = {0: "CBS_OK", 1: "CBS_EINVAL", 2: "CBS_ENOMEM", 3: "CBS_ECUDA", 4: "CBS_ENOCONV",
                5: "CBS_EDIVERGED", 6: "CBS_ETIMEOUT"}
SUPPORTED_SIZES = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024, 2048)


class cbs_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3)]


class cbs_boundary(ctypes.Structure):
    _fields_ = [("n_abs", (ctypes.c_int * 2) * 3), ("gamma_max", ctypes.c_double), ("power", ctypes.c_double)]


DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class cbs_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nu", ctypes.c_double), ("beta", ctypes.c_double),
                ("shift_rule", ctypes.c_int), ("tol", ctypes.c_double), ("tol_inner", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("grid_kind", ctypes.c_int), ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class cbs_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("residual_checks", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("rel_increment", ctypes.c_double),
                ("a1", ctypes.c_double * 2), ("a2", ctypes.c_double * 2), ("lambda1", ctypes.c_double),
                ("lambda2", ctypes.c_double), ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {"iters": self.iters, "outer_iters": self.outer_iters, "residual_checks": self.residual_checks,
                "rel_residual": self.rel_residual, "rel_increment": self.rel_increment,
                "a1": complex(self.a1[0], self.a1[1]), "a2": complex(self.a2[0], self.a2[1]),
                "lambda1": self.lambda1, "lambda2": self.lambda2, "t_setup_ms": self.t_setup_ms,
                "t_solve_ms": self.t_solve_ms, "kernel_launches": self.kernel_launches}


EXPORTS = ("solver_create", "solve_forward", "solve_adjoint", "residual_norm", "born_iterate", "green_apply",
           "operator_apply", "scale_source", "unscale_field", "solver_scalars", "solver_time_kernels",
           "solver_destroy", "cbs_last_error", "green_apply_noalloc", "medium_gradient", "cbs_selftest",
           "cufft_baseline_iterate", "cbs_fp64_rate")

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return build_lib.LIB


def load(path: str | None = None):
    """Load the CUDA library (no compute).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        V, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        S = ctypes.c_int
        lib.solver_create.restype = S
        lib.solver_create.argtypes = [ctypes.POINTER(cbs_grid), D, D, V, V, V, ctypes.POINTER(cbs_boundary),
                                      ctypes.POINTER(cbs_options), ctypes.POINTER(V)]
        for name in ("solve_forward", "solve_adjoint"):
            f = getattr(lib, name)
            f.restype = S
            f.argtypes = [V, V, V, V, ctypes.POINTER(cbs_info)]
        lib.residual_norm.restype = S
        lib.residual_norm.argtypes = [V, V, V, I, ctypes.POINTER(D)]
        lib.born_iterate.restype = S
        lib.born_iterate.argtypes = [V, V, V, I, I, ctypes.POINTER(D)]
        lib.green_apply.restype = S
        lib.green_apply.argtypes = [V, V, V, I]
        lib.operator_apply.restype = S
        lib.operator_apply.argtypes = [V, V, V, I]
        lib.scale_source.restype = S
        lib.scale_source.argtypes = [V, V, V, I]
        lib.unscale_field.restype = S
        lib.unscale_field.argtypes = [V, V, V]
        lib.solver_scalars.restype = S
        lib.solver_scalars.argtypes = [V, ctypes.POINTER(D)]
        lib.solver_time_kernels.restype = S
        lib.solver_time_kernels.argtypes = [V, V, V, I, ctypes.c_char_p, I, ctypes.POINTER(D), I,
                                            ctypes.POINTER(I)]
        lib.solver_destroy.restype = None
        lib.solver_destroy.argtypes = [V]
        lib.cbs_last_error.restype = ctypes.c_char_p
        lib.cbs_last_error.argtypes = [V]
        lib.medium_gradient.restype = S
        lib.medium_gradient.argtypes = [V, V, V, V, V, V, V, V, V, I]
        lib.green_apply_noalloc.restype = S
        lib.green_apply_noalloc.argtypes = [ctypes.POINTER(cbs_grid), D, ctypes.POINTER(D), V, V, I, V]
        lib.cbs_selftest.restype = S
        lib.cbs_selftest.argtypes = [I, ctypes.POINTER(I)]
        lib.cbs_fp64_rate.restype = S
        lib.cbs_fp64_rate.argtypes = [ctypes.POINTER(D)]
        lib.cufft_baseline_iterate.restype = S
        lib.cufft_baseline_iterate.argtypes = [V, V, V, I, I, ctypes.POINTER(D)]
        if path is None:
            _lib = lib
        return lib


CBS_SELFTEST_BULK_TIMEOUT = 1


def fp64_rate() -> float:
    """Measured float64 FMA rate of the current device in TFLOP/s (cbs_fp64_rate)."""
    lib = load()
    out = ctypes.c_double(0.0)
    st = lib.cbs_fp64_rate(ctypes.byref(out))
    if st != CBS_OK:
        raise CBSError(st, "cbs_fp64_rate failed")
    return float(out.value)


def selftest_bulk_timeout() -> int:
    """Run the bulk-copy timeout self-test on the current device: a barrier that never completes makes the
    kernel's bounded wait expire.  Returns CBS_ETIMEOUT when the kernel noticed and reported it."""
    lib = load()
    out = ctypes.c_int(-1)
    st = lib.cbs_selftest(CBS_SELFTEST_BULK_TIMEOUT, ctypes.byref(out))
    if st != CBS_OK:
        raise CBSError(st, "self-test launch failed")
    return out.value


class CBSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _check_field(t, shape):
    import torch
    if t.device.type != "cuda" or t.dtype != torch.complex128 or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected a contiguous cuda complex128 tensor of shape {tuple(shape)}")


def solver_create(c0, rho, alpha, dx: float, omega: float, nabs, gamma_max: float, power: float = 2.0,
                  precision="fp64", nu: float = 0.8, beta: float = 0.95, shift_rule: int = CBS_SHIFT_MIDRANGE,
                  tol: float = 1e-6, tol_inner: float = 1e-4, max_iter: int = 100000, check_every: int = 50,
                  stream=None, collocated: bool = False, allocator=None):
    """c0, rho, alpha: cuda float64 tensors of the grid shape (n[D-1], ..., n[0]).  allocator="torch" serves
    the solver's device arrays from torch's caching allocator (on `stream`) instead of cudaMalloc."""
    import torch
    lib = load()
    for t in (c0, rho, alpha):
        if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous() or t.shape != c0.shape:
            raise ValueError("medium arrays must be contiguous cuda float64 tensors of one shape")
    g = cbs_grid()
    g.ndim = c0.dim()
    for a in range(g.ndim):
        g.n[a] = int(c0.shape[g.ndim - 1 - a])
    b = cbs_boundary()
    for a in range(g.ndim):
        b.n_abs[a][0], b.n_abs[a][1] = int(nabs[a][0]), int(nabs[a][1])
    b.gamma_max = float(gamma_max)
    b.power = float(power)
    o = cbs_options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.nu, o.beta, o.shift_rule = float(nu), float(beta), int(shift_rule)
    o.tol, o.tol_inner, o.max_iter, o.check_every = float(tol), float(tol_inner), int(max_iter), int(check_every)
    o.grid_kind = CBS_GRID_COLLOCATED if collocated else CBS_GRID_STAGGERED
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(int(stream.cuda_stream))
    callbacks = None
    if allocator == "torch":
        callbacks = _torch_allocator(stream)
        o.dev_alloc, o.dev_free = callbacks
    elif allocator is not None:
        raise ValueError("allocator must be None or 'torch'")
    h = ctypes.c_void_p()
    st = lib.solver_create(ctypes.byref(g), float(dx), float(omega), _ptr(c0), _ptr(rho), _ptr(alpha),
                           ctypes.byref(b), ctypes.byref(o), ctypes.byref(h))
    if st != CBS_OK:
        raise CBSError(st, lib.cbs_last_error(None).decode())
    sv = Solver(h, tuple(c0.shape), o)
    sv._callbacks = callbacks  # the C side calls them until solver_destroy
    return sv


def _torch_allocator(stream):
    """dev_alloc / dev_free callbacks over torch's caching allocator, blocks associated with `stream`."""
    import torch

    dev = stream.device

    def alloc(nbytes, _stream, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
        except RuntimeError:  # out of memory: the solver reports CBS_ENOMEM
            return None

    def free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return DEV_ALLOC_FN(alloc), DEV_FREE_FN(free)


class Solver:
    """Owner of one ``cbs_solver*``; methods mirror the C entry points."""

    def __init__(self, handle, shape, options):
        self._h = handle
        self.shape = shape
        self.ndim = len(shape)
        self.ncomp = self.ndim + 1
        self.options = options
        self._callbacks = None
        self._lib = load()

    @property
    def field_shape(self):
        return (self.ncomp,) + tuple(self.shape)

    def _raise(self, st):
        raise CBSError(st, self._lib.cbs_last_error(self._h).decode())

    def destroy(self):
        if self._h:
            self._lib.solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def _solve(self, fn, src, field, x0, allow=(CBS_OK,)):
        _check_field(src, self.field_shape)
        _check_field(field, self.field_shape)
        if x0 is not None:
            _check_field(x0, self.field_shape)
        info = cbs_info()
        st = fn(self._h, _ptr(src), _ptr(field), _ptr(x0), ctypes.byref(info))
        if st not in allow:
            self._raise(st)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[st]
        return d

    def solve_forward(self, src, field, x0=None, allow_noconv=False):
        return self._solve(self._lib.solve_forward, src, field, x0,
                           (CBS_OK, CBS_ENOCONV) if allow_noconv else (CBS_OK,))

    def solve_adjoint(self, src, field, x0=None, allow_noconv=False):
        return self._solve(self._lib.solve_adjoint, src, field, x0,
                           (CBS_OK, CBS_ENOCONV) if allow_noconv else (CBS_OK,))

    def residual_norm(self, field, src, adjoint=False) -> float:
        _check_field(field, self.field_shape)
        _check_field(src, self.field_shape)
        r = ctypes.c_double()
        st = self._lib.residual_norm(self._h, _ptr(field), _ptr(src), int(adjoint), ctypes.byref(r))
        if st != CBS_OK:
            self._raise(st)
        return r.value

    def born_iterate(self, y, x, n_iter: int, adjoint=False):
        import numpy as np
        _check_field(y, self.field_shape)
        _check_field(x, self.field_shape)
        inc = np.zeros(max(int(n_iter), 1))
        st = self._lib.born_iterate(self._h, _ptr(y), _ptr(x), int(n_iter), int(adjoint),
                                    inc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st != CBS_OK:
            self._raise(st)
        return inc[: int(n_iter)]

    def green_apply(self, v, out, adjoint=False):
        _check_field(v, self.field_shape)
        _check_field(out, self.field_shape)
        st = self._lib.green_apply(self._h, _ptr(v), _ptr(out), int(adjoint))
        if st != CBS_OK:
            self._raise(st)

    def operator_apply(self, x, out, adjoint=False):
        _check_field(x, self.field_shape)
        _check_field(out, self.field_shape)
        st = self._lib.operator_apply(self._h, _ptr(x), _ptr(out), int(adjoint))
        if st != CBS_OK:
            self._raise(st)

    def scale_source(self, src, y, adjoint=False):
        _check_field(src, self.field_shape)
        _check_field(y, self.field_shape)
        st = self._lib.scale_source(self._h, _ptr(src), _ptr(y), int(adjoint))
        if st != CBS_OK:
            self._raise(st)

    def unscale_field(self, x, field):
        _check_field(x, self.field_shape)
        _check_field(field, self.field_shape)
        st = self._lib.unscale_field(self._h, _ptr(x), _ptr(field))
        if st != CBS_OK:
            self._raise(st)

    def medium_gradient(self, c0, rho, alpha, src, field, adj_field, grad_c0, grad_rho, accumulate=False):
        """Adjoint-state gradient contribution of one source (see include/cbs.h)."""
        for t in (src, field, adj_field):
            _check_field(t, self.field_shape)
        st = self._lib.medium_gradient(self._h, _ptr(c0), _ptr(rho), _ptr(alpha), _ptr(src), _ptr(field),
                                       _ptr(adj_field), _ptr(grad_c0), _ptr(grad_rho), int(accumulate))
        if st != CBS_OK:
            self._raise(st)

    def scalars(self) -> dict:
        out = (ctypes.c_double * 6)()
        st = self._lib.solver_scalars(self._h, out)
        if st != CBS_OK:
            self._raise(st)
        return {"a1": complex(out[0], out[1]), "a2": complex(out[2], out[3]), "lambda1": out[4],
                "lambda2": out[5]}

    def cufft_iterate(self, y, x, n_iter: int, adjoint=False) -> float:
        """The cuFFT comparison build of n_iter float32 iterations (x updated in place); ms per iteration."""
        _check_field(y, self.field_shape)
        _check_field(x, self.field_shape)
        ms = ctypes.c_double()
        st = self._lib.cufft_baseline_iterate(self._h, _ptr(y), _ptr(x), int(n_iter), int(adjoint), ctypes.byref(ms))
        if st != CBS_OK:
            self._raise(st)
        return ms.value

    def time_kernels(self, y, x, n_iter: int):
        _check_field(y, self.field_shape)
        _check_field(x, self.field_shape)
        names = ctypes.create_string_buffer(256)
        ms = (ctypes.c_double * 8)()
        nk = ctypes.c_int()
        st = self._lib.solver_time_kernels(self._h, _ptr(y), _ptr(x), int(n_iter), names, 256, ms, 8,
                                           ctypes.byref(nk))
        if st != CBS_OK:
            self._raise(st)
        labels = names.raw.split(b"\0")[: nk.value]
        return {lab.decode(): ms[i] for i, lab in enumerate(labels)}
