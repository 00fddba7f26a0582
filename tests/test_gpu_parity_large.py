"""GPU parity at the axis extents the larger workloads run, and full-size checks.

The serving grids (64^3 .. 192^3, 512^2 .. 2048^2) and the 512^3 shell run the
512-, 1024- and 2048-point instances of the row, strided-axis and last-axis
kernels (and the 96- and 192-point 3 * 2^k instances).  Each instance is
compared with the float64 oracle here on grids that are long along one axis
and short along the others, so the oracle finishes in seconds:

  * one (L+I)^-1 apply (App. B.1 symbol, forward and adjoint): float64 1e-12,
    float32 2e-6 (rounding ~ eps log N);
  * 20 Born iterations (eq. BornAlt, Algorithm 1, forward and adjoint):
    float64 1e-11, float32 1e-5.

At 512^3, where the oracle cannot iterate in seconds, the checks are
  * 20 float32 iterations of the shell workload against 20 float64
    iterations of the GPU path (1e-5); the uniform-medium closed form at
    sampled voxels (constant coefficients are diagonal under the DFT); the
    reciprocity of the pressure-pressure block (two solves).
The comparisons with converged oracle solves at full size are in
test_gpu_zy_full_size.py.
"""

import numpy as np
import pytest

from oracle import dense
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _cbs():
    from paper_2507_16087_gb300 import cbs
    return cbs


def T(a, dt=None):
    a = np.ascontiguousarray(a)
    if dt is None:
        dt = torch.complex128 if np.iscomplexobj(a) else torch.float64
    return torch.tensor(a, dtype=dt, device=DEV).contiguous()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def trel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def make(shape, seed, precision, n_abs=3, **kw):
    p = W.smooth_random_medium(shape, seed=seed, n_abs=n_abs)
    p.gamma_max = 0.5 * p.omega
    kw.setdefault("nu", 0.5)
    s = _cbs().solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max,
                             precision=precision, **kw)
    return p, s


# numpy shapes (n[D-1], ..., n[0]): each long extent once along x (row kernels), y (strided-axis kernel, 3D)
# and the last axis (all-components pencil kernel)
LARGE = [
    (64, 2048), (2048, 64), (1024, 1024), (512, 512), (48, 1024), (1024, 24),
    (16, 16, 512), (16, 512, 16), (512, 16, 16),
    (8, 8, 1024), (8, 1024, 8), (1024, 8, 8),
    (8, 8, 2048), (8, 2048, 8), (2048, 8, 8),
    (8, 16, 192), (8, 192, 16), (192, 8, 16), (96, 12, 8),
]


@pytest.mark.parametrize("shape", LARGE)
@pytest.mark.parametrize("adjoint", [False, True])
def test_large_extent_green_and_iterations_match_oracle(shape, adjoint):
    seed = 100 + sum(shape)
    p, s64 = make(shape, seed, "fp64")
    _, s32 = make(shape, seed, "fp32")
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    # one (L+I)^-1 apply
    v = W.random_source(shape, seed + 1)
    ref = P.green(v, adjoint)
    for s, tol in ((s64, 1e-12), (s32, 2e-6)):
        out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        s.green_apply(T(v), out, adjoint)
        assert rel(out.cpu().numpy(), ref) <= tol, (tol, shape)
    # 20 Born iterations
    y = P.scale_source(W.random_source(shape, seed + 2), adjoint)
    xr, incr = P.iterate(y, n_iter=20, nu=0.5, adjoint=adjoint)
    for s, tol in ((s64, 1e-11), (s32, 1e-5)):
        x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        inc = s.born_iterate(T(y), x, 20, adjoint)
        assert rel(x.cpu().numpy(), xr) <= tol, (tol, shape)
        assert np.allclose(inc, incr, rtol=1e-9 if s is s64 else 1e-4, atol=0)


@pytest.mark.parametrize("shape", [(64, 2048), (2048, 64), (16, 16, 512), (512, 16, 16)])
def test_large_extent_operator_apply_matches_oracle(shape):
    """A_s x (the float64 residual's operator, SYM_L symbol) at the long extents."""
    seed = 200 + sum(shape)
    p, s = make(shape, seed, "fp64")
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    x = W.random_source(shape, seed + 1)
    for adjoint in (False, True):
        out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        s.operator_apply(T(x), out, adjoint)
        assert rel(out.cpu().numpy(), P.apply(x, adjoint)) <= 1e-12


# ------------------------------------------------------------------- 512^3
def test_skull_512_fp32_iterations_match_fp64():
    """512^3 skull-like shell with a bowl source: 20 float32 Born iterations against 20 float64
    iterations of the GPU path on the same scaled source (the oracle cannot iterate at this size in
    seconds; both GPU paths are checked against it at the 512-point extents above)."""
    cbs = _cbs()
    p = W.skull_shell(512)
    args = (T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max)
    src = T(p.source)
    del p
    s64 = cbs.solver_create(*args, precision="fp64")
    y = torch.zeros(s64.field_shape, dtype=torch.complex128, device=DEV)
    s64.scale_source(src, y)
    del src
    x64 = torch.zeros_like(y)
    inc64 = s64.born_iterate(y, x64, 20)
    s64.destroy()
    s32 = cbs.solver_create(*args, precision="fp32")
    x32 = torch.zeros_like(y)
    inc32 = s32.born_iterate(y, x32, 20)
    s32.destroy()
    assert trel(x32, x64) <= 1e-5
    assert np.allclose(inc32, inc64, rtol=1e-4, atol=0)


def test_uniform_medium_closed_form_512():
    """P6 at 512^3: uniform absorbing medium, no layer, single-voxel pressure source.  The discrete solution
    is, per DFT wavenumber, p^ = (s / (rho c^2)) / (q + |k|^2 / d) with d = i omega rho, q = i omega /
    (rho c^2) (the Schur complement of App. B.1's per-wavenumber block, since (i k_eta e^{-i k dx/2})
    (i k_eta e^{i k dx/2}) = -k_eta^2); its inverse DFT is summed at sampled voxels one wavenumber slab
    at a time.  The GPU solve (FP32 + refinement to 1e-9) must match at every sample."""
    cbs = _cbs()
    n = 512
    shape = (n, n, n)
    dx = W.grid_step(6.0)
    om = 2 * np.pi * W.F0
    c0v, rhov, alv = 1500.0, 1000.0, 60.0
    src_pos = (200, 260, 250)   # (x, y, z)
    s = cbs.solver_create(T(np.full(shape, c0v)), T(np.full(shape, rhov)), T(np.full(shape, alv)), dx, om,
                          [[0, 0]] * 3, 0.0, precision="fp32_refine", tol=1e-9, check_every=50)
    src = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    src[(3,) + tuple(src_pos[::-1])] = 1.0
    field = torch.zeros_like(src)
    info = s.solve_forward(src, field)
    assert info["rel_residual"] <= 1e-9
    rng = np.random.default_rng(512)
    offs = [(0, 0, 0), (1, 0, 0), (0, -1, 0), (0, 0, 3), (7, -5, 2), (20, 0, 0), (-33, 12, 5)]
    offs += [tuple(int(v) for v in rng.integers(-60, 61, 3)) for _ in range(9)]
    pts = [tuple(src_pos[a] + o[a] for a in range(3)) for o in offs]
    got = np.array([complex(field[(3,) + (z, y, x)].item()) for (x, y, z) in pts])
    c2 = c0v ** 2 / (1 - 2j * alv * c0v / om)
    d = 1j * om * rhov
    q = 1j * om / (rhov * c2)
    k = dense.wavenumbers(n, dx)
    j = np.arange(n)
    # phases e^{2 pi i j (r - r_s) / n} per axis and sample: (n, n_samples)
    E = [np.exp(2j * np.pi * np.outer(j, [pt[a] - src_pos[a] for pt in pts]) / n) for a in range(3)]
    k2xy = k[None, :] ** 2 + k[:, None] ** 2           # (y, x)
    acc = np.zeros(len(pts), dtype=np.complex128)
    for jz in range(n):
        ph = 1.0 / (rhov * c2) / (q + (k2xy + k[jz] ** 2) / d)   # p^ of a unit source at the origin, (y, x)
        t = ph @ E[0]                                             # sum over x -> (y, samples)
        acc += E[2][jz] * np.einsum("ys,ys->s", E[1], t)
    ref = acc / n ** 3
    err = np.abs(got - ref)
    assert np.max(err) <= 1e-6 * np.max(np.abs(ref)), (np.max(err), np.max(np.abs(ref)))
    assert np.all(err <= 1e-5 * np.abs(ref) + 1e-7 * np.max(np.abs(ref)))


def test_reciprocity_512():
    """P9 at 512^3 (sphere inclusion with absorption, 24-cell layer): the pressure at b from a pressure source
    at a equals the pressure at a from the same source at b, both points in the water background (the
    row-scaled pressure block is symmetric: the staggered derivative pair satisfies E = -D^T).  A third
    point shows the check can fail."""
    cbs = _cbs()
    p = W.inclusion_medium((512, 512, 512), 120, 1800.0, 1300.0, 1.0, ppw=6.0, n_abs=24)
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max,
                          precision="fp32_refine", tol=1e-8, check_every=50)
    a, b, c = (100, 256, 256), (140, 300, 230), (150, 200, 300)   # (x, y, z), outside the sphere and layer
    fields = {}
    for name, pt in (("a", a), ("b", b)):
        src = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        src[(3,) + pt[::-1]] = 1.0
        f = torch.zeros_like(src)
        info = s.solve_forward(src, f)
        assert info["rel_residual"] <= 1e-8
        fields[name] = f
        del src
    pab = complex(fields["a"][(3,) + b[::-1]].item())
    pba = complex(fields["b"][(3,) + a[::-1]].item())
    assert abs(pab - pba) <= 1e-5 * abs(pab), (pab, pba)
    pac = complex(fields["a"][(3,) + c[::-1]].item())
    assert abs(pac - pba) > 1e-3 * abs(pba)
