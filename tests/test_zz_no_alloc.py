"""The allocation-free (L+I)^-1 apply (green_apply_noalloc), for callers that
cannot call cudaMalloc, against the solver's green_apply on the same input.

It runs last (file name) so that a run stopping at the first failure has run
every other test before it; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2507_16087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grid(cbs, shape):
    g = cbs.cbs_grid()
    g.ndim = len(shape)
    for a in range(g.ndim):
        g.n[a] = int(shape[g.ndim - 1 - a])
    return g


def _noalloc(cbs, shape, dx, scalars, v, out, adjoint):
    L = cbs.load()
    g = _grid(cbs, shape)
    sc = (ctypes.c_double * 6)(*scalars)
    return L.green_apply_noalloc(ctypes.byref(g), float(dx), sc, v.data_ptr(), out.data_ptr(), int(adjoint),
                                 ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream)))


@pytest.mark.parametrize("shape", [(96, 64), (16, 24, 12), (128, 128, 128)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_noalloc_green_matches_green_apply_twice(shape, adjoint):
    from paper_2507_16087_gb300 import cbs

    dev = "cuda:0"
    p = W.smooth_random_medium(shape, seed=31, n_abs=4)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)  # noqa: E731
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max, precision="fp64")
    sc = s.scalars()
    scalars = [sc["a1"].real, sc["a1"].imag, sc["a2"].real, sc["a2"].imag, sc["lambda1"], sc["lambda2"]]
    for call in range(2):  # two calls in a row share the static scratch
        v = T(W.random_source(shape, 40 + call))
        ref = torch.zeros_like(v)
        s.green_apply(v, ref, adjoint)
        out = torch.full_like(v, complex(np.nan, np.nan))
        st = _noalloc(cbs, shape, p.dx, scalars, v, out, adjoint)
        assert st == cbs.CBS_OK, cbs.load().cbs_last_error(None)
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= 1e-12, (call, err)
    s.destroy()


def test_noalloc_rejects_grids_beyond_its_maximum():
    from paper_2507_16087_gb300 import cbs

    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    out = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    st = _noalloc(cbs, (256, 128, 128), 1e-3, [0, 1e9, 1e-3, 1e-3, 1e9, 1e-3], dummy, out, False)
    assert st == cbs.CBS_EINVAL
    assert b"exceeds the allocation-free maximum" in cbs.load().cbs_last_error(None)
