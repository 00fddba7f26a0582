"""Python handle on the FP64 CPU oracle (``cbs_oracle.c``).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.  It shares nothing with the CUDA library and never
loads it.  Arrays are numpy complex128 of shape ``(C, n[D-1], ..., n[0])`` with
components ``(u_x, u_y, [u_z], p)`` (velocity at staggered points, App. B.1 of
Stanziola et al., arXiv 2507.16087).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CBS_ORACLE_SRC / CBS_ORACLE_LIB: only the planted-mistake test sets them, in child processes, to run the pins
# against a copy of this source with one deliberate slip (tests/test_oracle_mutants.py)
_SRC = os.environ.get("CBS_ORACLE_SRC") or os.path.join(_HERE, "cbs_oracle.c")
_LIB_PATH = os.environ.get("CBS_ORACLE_LIB") or os.path.join(_HERE, "_build", "libcbs_oracle.so")
_lock = threading.Lock()
_lib = None

SHIFT_MIDRANGE = 0
SHIFT_MEDIAN = 1
SHIFT_MEC = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, OpenMP over independent lines)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double, ctypes.c_double,
                                   D, D, D, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.orc_destroy.argtypes = [P]
        lib.orc_scalars.argtypes = [P, D]
        lib.orc_get_v.argtypes = [P, P]
        lib.orc_scale_source.argtypes = [P, P, P, ctypes.c_int]
        lib.orc_unscale.argtypes = [P, P, P]
        lib.orc_green.argtypes = [P, P, P, ctypes.c_int]
        lib.orc_apply.argtypes = [P, P, P, ctypes.c_int]
        lib.orc_residual.argtypes = [P, P, P, ctypes.c_int]
        lib.orc_residual.restype = ctypes.c_double
        lib.orc_iterate.argtypes = [P, P, P, ctypes.c_long, ctypes.c_double, ctypes.c_int, D]
        lib.orc_solve.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_long, ctypes.c_long,
                                  ctypes.c_int, D]
        lib.orc_solve.restype = ctypes.c_long
        lib.orc_fft1d.argtypes = [P, ctypes.c_long, ctypes.c_long, ctypes.c_int]
        lib.orc_fftn.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fft1d(x, sign: int = -1) -> np.ndarray:
    """Own 1-D DFT (sign -1 forward, +1 inverse without 1/n)."""
    a = _c128(x).copy()
    _load().orc_fft1d(_ptr(a), a.size, 1, sign)
    return a


def fftn(x, sign: int = -1) -> np.ndarray:
    """Own D-dim DFT over all axes of ``x`` (sign +1 includes 1/N)."""
    a = _c128(x).copy()
    n = np.array(a.shape[::-1], dtype=np.int64)
    _load().orc_fftn(_ptr(a), a.ndim, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), sign)
    return a


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


class Problem:
    """Set-up (Sec. 2.3.1 / Algorithm 1 preprocessing) plus the operators.

    ``shape`` is the numpy shape of one component, i.e. ``(n[D-1], ..., n[0])``;
    ``c0``, ``rho``, ``alpha`` (Np/m) have that shape.  ``nabs`` is
    ``[[lo, hi]] * D`` in axis order x, y, z.
    """

    def __init__(self, c0, rho, alpha, dx: float, omega: float, nabs, gamma_max: float,
                 power: float = 2.0, beta: float = 0.95, shift_rule: int = SHIFT_MIDRANGE,
                 collocated: bool = False):
        lib = _load()
        c0 = np.ascontiguousarray(c0, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        alpha = np.ascontiguousarray(alpha, dtype=np.float64)
        self.shape = c0.shape
        self.ndim = c0.ndim
        self.ncomp = self.ndim + 1
        n = np.array(self.shape[::-1], dtype=np.int64)
        nab = np.zeros((3, 2), dtype=np.int32)
        nab[: self.ndim] = np.asarray(nabs, dtype=np.int32).reshape(self.ndim, 2)
        dp = ctypes.POINTER(ctypes.c_double)
        self._h = lib.orc_create(self.ndim, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(dx), float(omega),
                                 c0.ctypes.data_as(dp), rho.ctypes.data_as(dp), alpha.ctypes.data_as(dp),
                                 nab.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(gamma_max), float(power),
                                 float(beta), int(shift_rule), int(bool(collocated)))
        if not self._h:
            raise ValueError("oracle set-up rejected the inputs")
        self._lib = lib
        self.dx = dx
        self.omega = omega

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def field_shape(self):
        return (self.ncomp,) + tuple(self.shape)

    def _empty(self):
        return np.zeros(self.field_shape, dtype=np.complex128)

    def scalars(self) -> dict:
        out = np.zeros(6)
        self._lib.orc_scalars(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return {"a1": complex(out[0], out[1]), "a2": complex(out[2], out[3]), "lambda1": out[4], "lambda2": out[5]}

    def v(self) -> np.ndarray:
        o = self._empty()
        self._lib.orc_get_v(self._h, _ptr(o))
        return o

    def scale_source(self, s, adjoint: bool = False) -> np.ndarray:
        s = _c128(s)
        o = self._empty()
        self._lib.orc_scale_source(self._h, _ptr(s), _ptr(o), int(adjoint))
        return o

    def unscale(self, x) -> np.ndarray:
        x = _c128(x)
        o = self._empty()
        self._lib.orc_unscale(self._h, _ptr(x), _ptr(o))
        return o

    def green(self, v, adjoint: bool = False) -> np.ndarray:
        v = _c128(v)
        o = self._empty()
        self._lib.orc_green(self._h, _ptr(v), _ptr(o), int(adjoint))
        return o

    def apply(self, x, adjoint: bool = False) -> np.ndarray:
        x = _c128(x)
        o = self._empty()
        self._lib.orc_apply(self._h, _ptr(x), _ptr(o), int(adjoint))
        return o

    def residual(self, x, y, adjoint: bool = False) -> float:
        x = _c128(x)
        y = _c128(y)
        return float(self._lib.orc_residual(self._h, _ptr(x), _ptr(y), int(adjoint)))

    def iterate(self, y, x0=None, n_iter: int = 1, nu: float = 0.5, adjoint: bool = False):
        """Run ``n_iter`` Born iterations (eq. BornAlt); returns (x, increments)."""
        y = _c128(y)
        x = self._empty() if x0 is None else _c128(x0).copy()
        inc = np.zeros(max(int(n_iter), 1))
        self._lib.orc_iterate(self._h, _ptr(y), _ptr(x), int(n_iter), float(nu), int(adjoint),
                              inc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return x, inc[: int(n_iter)]

    def solve(self, y, tol: float, max_iter: int = 100000, check_every: int = 10, nu: float = 0.5,
              x0=None, adjoint: bool = False):
        """Iterate until ||y - A_s x|| / ||y|| <= tol; returns (x, iterations, residual)."""
        y = _c128(y)
        x = self._empty() if x0 is None else _c128(x0).copy()
        res = ctypes.c_double(0.0)
        it = self._lib.orc_solve(self._h, _ptr(y), _ptr(x), float(nu), float(tol), int(max_iter), int(check_every),
                                 int(adjoint), ctypes.byref(res))
        return x, int(it), float(res.value)

    def solve_field(self, s, tol: float, **kw):
        """Physical source (s_u, s_p) -> physical field (u, p) (Algorithm 1 end to end)."""
        y = self.scale_source(s)
        x, it, res = self.solve(y, tol, **kw)
        return self.unscale(x), it, res
