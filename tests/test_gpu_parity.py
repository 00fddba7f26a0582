"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (relative L2 unless stated):
  FP64 path: set-up scalars 1e-13; source scaling 1e-14; one (L+I)^-1 or A_s
  apply 1e-12 (FFT rounding ~ eps log N); 20-50 Born iterations 1e-11; converged
  solves run to residual 1e-12 on both sides 1e-10.
  FP32 path: one apply 2e-6 (float32 eps * log N * a few); FP32 + FP64
  refinement converged to residual <= 1e-8: 1e-5 against the oracle.
Sizes span several FFT tiles and ragged edges: extents 8..192 with factors 2
and 3, grids whose x extent is smaller than a block's column tile, and 2D/3D.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cbs():
    from paper_2507_16087_gb300 import cbs
    return cbs


DEV = "cuda:0"


def T(a, dt=None):
    a = np.ascontiguousarray(a)
    if dt is None:
        dt = torch.complex128 if np.iscomplexobj(a) else torch.float64
    return torch.tensor(a, dtype=dt, device=DEV).contiguous()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(shape, seed=1, n_abs=3, gamma_scale=0.5, precision="fp64", **kw):
    p = W.smooth_random_medium(shape, seed=seed, n_abs=n_abs)
    p.gamma_max = gamma_scale * p.omega
    cbs = _cbs()
    kw.setdefault("nu", 0.5)
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max, precision=precision, **kw)
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    return p, s, P


SHAPES = [(16, 16), (24, 32), (96, 64), (12, 48), (8, 8, 8), (16, 24, 12), (12, 16, 32), (24, 8, 96)]


@pytest.mark.parametrize("shape", SHAPES)
def test_setup_scalars_match(shape):
    _, s, P = make(shape, seed=3)
    g, o = s.scalars(), P.scalars()
    for k in ("a1", "a2", "lambda1", "lambda2"):
        assert abs(g[k] - o[k]) <= 1e-13 * abs(o[k]), (k, g[k], o[k])


@pytest.mark.parametrize("shape", [(24, 32), (16, 24, 12)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_scale_source_matches(shape, adjoint):
    _, s, P = make(shape, seed=4)
    src = W.random_source(shape, 5)
    y = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.scale_source(T(src), y, adjoint)
    assert rel(y.cpu().numpy(), P.scale_source(src, adjoint)) <= 1e-14


@pytest.mark.parametrize("shape", SHAPES + [(128, 128), (64, 64, 64)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_green_apply_fp64(shape, adjoint):
    _, s, P = make(shape, seed=6)
    v = W.random_source(shape, 7)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.green_apply(T(v), out, adjoint)
    ref = P.green(v, adjoint)
    assert rel(out.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("shape", [(24, 32), (96, 64), (16, 24, 12), (64, 64, 64), (128, 256), (24, 128, 128),
                                   (16, 256, 128)])
def test_green_apply_fp32(shape):
    _, s, P = make(shape, seed=8, precision="fp32")
    v = W.random_source(shape, 9)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.green_apply(T(v), out)
    assert rel(out.cpu().numpy(), P.green(v)) <= 2e-6


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_operator_apply_fp64(shape, adjoint):
    _, s, P = make(shape, seed=10)
    x = W.random_source(shape, 11)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.operator_apply(T(x), out, adjoint)
    assert rel(out.cpu().numpy(), P.apply(x, adjoint)) <= 1e-12


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_born_iterations_fp64(shape, adjoint):
    _, s, P = make(shape, seed=12)
    y = P.scale_source(W.random_source(shape, 13), adjoint)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    inc = s.born_iterate(T(y), x, 40, adjoint)
    xr, incr = P.iterate(y, n_iter=40, nu=0.5, adjoint=adjoint)
    assert rel(x.cpu().numpy(), xr) <= 1e-11
    assert np.allclose(inc, incr, rtol=1e-9, atol=0)


@pytest.mark.parametrize("shape", [(16, 24, 32), (24, 128, 128), (256, 128)])
def test_born_iterations_fp32(shape):
    _, s, P = make(shape, seed=14, precision="fp32")
    y = P.scale_source(W.random_source(shape, 15))
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.born_iterate(T(y), x, 30)
    xr, _ = P.iterate(y, n_iter=30, nu=0.5)
    assert rel(x.cpu().numpy(), xr) <= 1e-5


@pytest.mark.parametrize("shape", [(24, 32), (16, 12, 8)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_converged_solve_fp64_matches_oracle_and_dense(shape, adjoint):
    p, s, P = make(shape, seed=16, tol=1e-12, check_every=20)
    src = W.random_source(shape, 17)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = (s.solve_adjoint if adjoint else s.solve_forward)(T(src), field)
    assert info["rel_residual"] <= 1e-12
    y = P.scale_source(src, adjoint)
    x, _, res = P.solve(y, 1e-12, check_every=20, adjoint=adjoint)
    got = field.cpu().numpy()
    assert rel(got, P.unscale(x)) <= 1e-10
    if adjoint:
        ref = dense.solve_adjoint(src, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    else:
        ref = dense.solve(src, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    assert rel(got, ref) <= 1e-10
    # the residual entry point agrees with the solver's own report
    r = s.residual_norm(field, T(src), adjoint)
    assert r <= 1.5e-12


@pytest.mark.parametrize("shape", [(96, 64), (16, 24, 32)])
def test_fp32_refine_matches_oracle(shape):
    p, s, P = make(shape, seed=18, precision="fp32_refine", tol=1e-8, check_every=20)
    src = W.random_source(shape, 19)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(T(src), field)
    assert info["rel_residual"] <= 1e-8 and info["outer_iters"] >= 1
    ref, _, _ = P.solve_field(src, 1e-12, check_every=25)
    assert rel(field.cpu().numpy(), ref) <= 1e-5
    assert s.residual_norm(field, T(src)) <= 1.01e-8


def test_fp32_refine_residual_1e6_error_stated():
    """North-star pairing: mixed path run to residual 1e-6 -> error vs the FP64 oracle <= 1e-5."""
    shape = (64, 64)
    p, s, P = make(shape, seed=20, precision="fp32_refine", tol=1e-6, check_every=20, n_abs=8)
    src = W.random_source(shape, 21)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(T(src), field)
    assert info["rel_residual"] <= 1e-6
    ref, _, _ = P.solve_field(src, 1e-12, check_every=25)
    assert rel(field.cpu().numpy(), ref) <= 1e-5


# ------------------------------------------------------------------- edge cases
def test_zero_source_gives_zero_field():
    shape = (16, 16)
    _, s, _ = make(shape, tol=1e-8)
    field = torch.ones(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(torch.zeros_like(field), field)
    assert torch.count_nonzero(field).item() == 0 and info["rel_residual"] == 0


def test_warm_start_and_noconv():
    shape = (24, 32)
    cbs = _cbs()
    p, s, P = make(shape, seed=22, tol=1e-10, max_iter=40, check_every=20)
    src = T(W.random_source(shape, 23))
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(src, field, allow_noconv=True)
    assert info["status"] == "CBS_ENOCONV" and info["iters"] == 40
    with pytest.raises(cbs.CBSError):
        s.solve_forward(src, field)
    # resuming from the returned field continues the same iteration
    f2 = torch.zeros_like(field)
    s.solve_forward(src, f2, x0=field.clone(), allow_noconv=True)
    y = P.scale_source(src.cpu().numpy())
    x, _ = P.iterate(y, n_iter=80, nu=0.5)
    assert rel(f2.cpu().numpy(), P.unscale(x)) <= 1e-11


def test_rejects_invalid_media_and_sizes():
    cbs = _cbs()
    shape = (16, 16)
    c0 = np.full(shape, 1500.0)
    rho = np.full(shape, 1000.0)
    al = np.zeros(shape)
    for bad in ("c", "rho", "alpha", "nan"):
        c, r, a = c0.copy(), rho.copy(), al.copy()
        if bad == "c":
            c[3, 3] = -1
        elif bad == "rho":
            r[0, 0] = 0
        elif bad == "alpha":
            a[5, 5] = -0.1
        else:
            c[2, 7] = np.nan
        with pytest.raises(cbs.CBSError) as e:
            cbs.solver_create(T(c), T(r), T(a), 1e-3, 3e6, [[2, 2], [2, 2]], 1e6)
        assert e.value.status == cbs.CBS_EINVAL
    with pytest.raises(cbs.CBSError):
        cbs.solver_create(T(np.full((10, 16), 1500.0)), T(np.full((10, 16), 1e3)), T(np.zeros((10, 16))), 1e-3, 3e6,
                          [[1, 1], [1, 1]], 1e6)
    with pytest.raises(cbs.CBSError):
        cbs.solver_create(T(c0), T(rho), T(al), 1e-3, 3e6, [[1, 1], [1, 1]], 1e6, nu=1.5)


def test_deterministic_reruns():
    shape = (12, 16, 32)
    _, s, P = make(shape, seed=24, precision="fp32_refine", tol=1e-7, check_every=10)
    src = T(W.random_source(shape, 25))
    f1 = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    f2 = torch.zeros_like(f1)
    i1 = s.solve_forward(src, f1)
    i2 = s.solve_forward(src, f2)
    assert torch.equal(f1, f2) and i1["iters"] == i2["iters"]


# -------------------------------------------------- full-size properties (128^3)
def test_uniform_medium_closed_form_full_size():
    """Uniform absorbing medium without a layer: exact per-wavenumber solution at 128^3."""
    cbs = _cbs()
    shape = (128, 128, 128)
    dx = W.grid_step(6.0)
    om = 2 * np.pi * W.F0
    al = 60.0
    c0, rho, alpha = np.full(shape, 1500.0), np.full(shape, 1000.0), np.full(shape, al)
    src = np.zeros((4,) + shape, dtype=np.complex128)
    src[3, 64, 64, 30] = 1.0
    src[0, 40, 70, 64] = 0.5j
    ref = dense.uniform_solve(src, 1500.0, 1000.0, al, dx, om)
    for prec, tol, bound in (("fp64", 1e-11, 1e-9), ("fp32_refine", 1e-9, 1e-7)):
        s = cbs.solver_create(T(c0), T(rho), T(alpha), dx, om, [[0, 0]] * 3, 0.0, precision=prec, tol=tol,
                              check_every=50)
        field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        s.solve_forward(T(src), field)
        assert rel(field.cpu().numpy(), ref) <= bound, prec
        s.destroy()


def test_sphere_128_first_iterations_and_precisions():
    """Full-size sphere workload (128^3, 20-cell layer, point source): the first iterations match the
    oracle; FP32+refinement and FP64 solves to 1e-6 agree; the true residual is recomputed."""
    cbs = _cbs()
    p = W.sphere_128()
    src = p.source
    s64 = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max, precision="fp64",
                            tol=1e-6, check_every=50, nu=0.5)
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    y = P.scale_source(src)
    x = torch.zeros(s64.field_shape, dtype=torch.complex128, device=DEV)
    s64.born_iterate(T(y), x, 3)
    xr, _ = P.iterate(y, n_iter=3, nu=0.5)
    assert rel(x.cpu().numpy(), xr) <= 1e-12
    f64 = torch.zeros(s64.field_shape, dtype=torch.complex128, device=DEV)
    i64 = s64.solve_forward(T(src), f64)
    s32 = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max,
                            precision="fp32_refine", tol=1e-6, check_every=50)
    f32 = torch.zeros_like(f64)
    i32 = s32.solve_forward(T(src), f32)
    assert i64["rel_residual"] <= 1e-6 and i32["rel_residual"] <= 1e-6
    assert s64.residual_norm(f32, T(src)) <= 1.01e-6
    assert s64.residual_norm(f64, T(src)) <= 1.01e-6
    # both are within the stopping tolerance of the same solution
    assert rel(f32.cpu().numpy(), f64.cpu().numpy()) <= 1e-4


@pytest.mark.parametrize("rule", ["median", "mec"])
def test_shift_rules_match_oracle_and_solution(rule):
    cbs = _cbs()
    shape = (24, 32)
    code = {"median": cbs.CBS_SHIFT_MEDIAN, "mec": cbs.CBS_SHIFT_MEC}[rule]
    orc = {"median": O.SHIFT_MEDIAN, "mec": O.SHIFT_MEC}[rule]
    p, s, _ = make(shape, seed=34, shift_rule=code, tol=1e-12, check_every=20)
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, shift_rule=orc)
    g, o = s.scalars(), P.scalars()
    if rule == "median":
        for k in ("a1", "a2", "lambda1", "lambda2"):
            assert abs(g[k] - o[k]) <= 1e-13 * abs(o[k])
    else:
        # support-point circle (64 directions) vs the exact circle: same centre to within the polygon's sag
        for k, lam in (("a1", "lambda1"), ("a2", "lambda2")):
            assert abs(g[k] - o[k]) <= 2e-3 * o[lam]
            assert g[lam] >= o[lam] * (1 - 1e-12)          # exact circle is the smallest
            assert g[lam] <= o[lam] * (1 + 5e-3)
    src = W.random_source(shape, 35)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.solve_forward(T(src), field)
    ref = dense.solve(src, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    assert rel(field.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("shape", [(24, 32), (12, 8, 24)])
def test_collocated_grid_matches_oracle(shape):
    """App. B's collocated variant: symbol, iterations and converged field against the oracle / dense system."""
    p, s, _ = make(shape, seed=36, collocated=True, tol=1e-12, check_every=20)
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, collocated=True)
    g, o = s.scalars(), P.scalars()
    for k in ("a1", "a2", "lambda1", "lambda2"):
        assert abs(g[k] - o[k]) <= 1e-13 * abs(o[k])
    v = W.random_source(shape, 37)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.green_apply(T(v), out)
    assert rel(out.cpu().numpy(), P.green(v)) <= 1e-12
    y = P.scale_source(v)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.born_iterate(T(y), x, 30)
    xr, _ = P.iterate(y, n_iter=30, nu=0.5)
    assert rel(x.cpu().numpy(), xr) <= 1e-11
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.solve_forward(T(v), field)
    ref = dense.solve(v, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power, collocated=True)
    assert rel(field.cpu().numpy(), ref) <= 1e-10


def test_bulk_copy_wait_expires_and_reports():
    """Failure detection without a fault: a bulk copy that delivers half the bytes its barrier expects never
    completes the phase; the bounded wait gives up, the kernel reports CBS_ETIMEOUT and returns, and the
    context still computes correctly afterwards."""
    cbs = _cbs()
    assert cbs.selftest_bulk_timeout() == cbs.CBS_ETIMEOUT
    _, s, P = make((16, 16), seed=2)
    v = W.random_source((16, 16), 3)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.green_apply(T(v), out)
    assert rel(out.cpu().numpy(), P.green(v)) <= 1e-12


@pytest.mark.parametrize("shape", [(64, 64, 64), (128, 32, 48), (96, 24, 32), (192, 8, 16), (256, 16, 16),
                                   (16, 24, 32)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_last_axis_tile_kernel_matches_register_kernel_and_oracle(shape, adjoint, monkeypatch):
    """The tile-staged last-axis kernel (tensor copies into shared memory, one component transformed at a
    time) does the same arithmetic in the same order as the all-in-registers kernel: float32 Born
    iterations agree to float32 rounding (contraction into FMAs may differ), and both match the float64
    oracle."""
    monkeypatch.setenv("CBS_TILE_LAST", "1")
    _, s, P = make(shape, seed=40, precision="fp32")
    monkeypatch.delenv("CBS_TILE_LAST")
    _, s_reg, _ = make(shape, seed=40, precision="fp32")
    y = P.scale_source(W.random_source(shape, 41), adjoint)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    x_reg = torch.zeros_like(x)
    s.born_iterate(T(y), x, 12, adjoint)
    s_reg.born_iterate(T(y), x_reg, 12, adjoint)
    assert rel(x.cpu().numpy(), x_reg.cpu().numpy()) <= 1e-6
    xr, _ = P.iterate(y, n_iter=12, nu=0.5, adjoint=adjoint)
    assert rel(x.cpu().numpy(), xr) <= 1e-5


@pytest.mark.parametrize("shape", [(16, 32, 32), (12, 32, 64), (24, 64, 32), (8, 128, 64), (16, 128, 128),
                                   (48, 64, 128), (16, 128, 32), (24, 32, 128)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_plane_kernels_match_row_axis_kernels_and_oracle(shape, adjoint, monkeypatch):
    """The x-y plane kernels (a CTA pair per (component, z) plane, both transforms on chip) against the
    row + strided-axis kernels and the float64 oracle, float32 Born iterations."""
    monkeypatch.setenv("CBS_PLANE", "1")
    _, s, P = make(shape, seed=42, precision="fp32")
    monkeypatch.delenv("CBS_PLANE")
    monkeypatch.setenv("CBS_NO_PLANE", "1")
    _, s_ref, _ = make(shape, seed=42, precision="fp32")
    monkeypatch.delenv("CBS_NO_PLANE")
    y = P.scale_source(W.random_source(shape, 43), adjoint)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    x_ref = torch.zeros_like(x)
    inc = s.born_iterate(T(y), x, 12, adjoint)
    inc_ref = s_ref.born_iterate(T(y), x_ref, 12, adjoint)
    assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 2e-6
    xr, incr = P.iterate(y, n_iter=12, nu=0.5, adjoint=adjoint)
    assert rel(x.cpu().numpy(), xr) <= 1e-5
    assert np.allclose(inc, incr, rtol=1e-4, atol=0)


def test_plane_kernels_solve_sphere_128(monkeypatch):
    """The 128^3 sphere workload solved to 1e-6 with the plane kernels: the float64 residual of the
    result is recomputed and the field agrees with the row + axis kernel solve within the tolerance."""
    cbs = _cbs()
    p = W.sphere_128()
    args = (T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max)
    monkeypatch.setenv("CBS_PLANE", "1")
    s = cbs.solver_create(*args, precision="fp32_refine", tol=1e-6, check_every=50)
    monkeypatch.delenv("CBS_PLANE")
    monkeypatch.setenv("CBS_NO_PLANE", "1")
    s_ref = cbs.solver_create(*args, precision="fp32_refine", tol=1e-6, check_every=50)
    monkeypatch.delenv("CBS_NO_PLANE")
    s64 = cbs.solver_create(*args, precision="fp64", tol=1e-6)
    f = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    f_ref = torch.zeros_like(f)
    info = s.solve_forward(T(p.source), f)
    info_ref = s_ref.solve_forward(T(p.source), f_ref)
    assert info["rel_residual"] <= 1e-6
    assert s64.residual_norm(f, T(p.source)) <= 1.01e-6
    assert abs(info["iters"] - info_ref["iters"]) <= 100
    assert rel(f.cpu().numpy(), f_ref.cpu().numpy()) <= 1e-4


def test_torch_caching_allocator_serves_solver_memory():
    """allocator='torch': the solver's arrays come from torch's caching allocator (counted by
    torch.cuda.memory_allocated while the solver lives, returned on destroy) and the solve is bitwise the
    same as with cudaMalloc."""
    cbs = _cbs()
    shape = (16, 24, 32)
    p = W.smooth_random_medium(shape, seed=50, n_abs=3)
    args = (T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max)
    src = T(W.random_source(shape, 51))
    f_t = torch.zeros((4,) + shape, dtype=torch.complex128, device=DEV)
    f_c = torch.zeros_like(f_t)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    s_t = cbs.solver_create(*args, precision="fp32_refine", tol=1e-8, allocator="torch")
    held = torch.cuda.memory_allocated() - base
    n = 4 * int(np.prod(shape))
    assert held >= n * (3 * 16 + 3 * 8)  # x, y, w in float64 and float32 at least
    s_c = cbs.solver_create(*args, precision="fp32_refine", tol=1e-8)
    assert torch.cuda.memory_allocated() - base == held  # cudaMalloc memory is not torch's
    i_t = s_t.solve_forward(src, f_t)
    i_c = s_c.solve_forward(src, f_c)
    assert i_t["iters"] == i_c["iters"] and i_t["rel_residual"] <= 1e-8
    assert torch.equal(f_t, f_c)
    s_t.destroy()
    s_c.destroy()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("shape", [(16, 24, 32), (64, 64, 64), (96, 128)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_cufft_baseline_matches_fused_kernels_and_oracle(shape, adjoint):
    """The cuFFT comparison build runs the same float32 iteration: it matches the fused kernels to float32
    rounding and the float64 oracle to the float32 tolerance."""
    _, s, P = make(shape, seed=44, precision="fp32")
    y = P.scale_source(W.random_source(shape, 45), adjoint)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    x_ref = torch.zeros_like(x)
    ms = s.cufft_iterate(T(y), x, 10, adjoint)
    assert ms > 0
    s.born_iterate(T(y), x_ref, 10, adjoint)
    assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 2e-6
    xr, _ = P.iterate(y, n_iter=10, nu=0.5, adjoint=adjoint)
    assert rel(x.cpu().numpy(), xr) <= 1e-5


@pytest.mark.parametrize("shape", [(16, 128, 64), (12, 256, 32), (24, 64, 64), (16, 96, 48), (8, 192, 32)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_pipelined_axis_kernel_matches_plain_axis_kernel_and_oracle(shape, adjoint, monkeypatch):
    """The persistent strided-axis kernel (tiles staged by tensor copies, two stages) computes the same
    transform as the one-tile-per-block kernel: float32 Born iterations agree to rounding and match the
    float64 oracle."""
    monkeypatch.setenv("CBS_AXIS_PIPE", "1")
    _, s, P = make(shape, seed=46, precision="fp32")
    monkeypatch.delenv("CBS_AXIS_PIPE")
    _, s_ref, _ = make(shape, seed=46, precision="fp32")
    y = P.scale_source(W.random_source(shape, 47), adjoint)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    x_ref = torch.zeros_like(x)
    s.born_iterate(T(y), x, 12, adjoint)
    s_ref.born_iterate(T(y), x_ref, 12, adjoint)
    assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-6
    xr, _ = P.iterate(y, n_iter=12, nu=0.5, adjoint=adjoint)
    assert rel(x.cpu().numpy(), xr) <= 1e-5


@pytest.mark.parametrize("shape", [(24, 32), (16, 12, 24)])
def test_collocated_grid_adjoint_matches_oracle(shape):
    """App. B's collocated variant, adjoint: the conjugate-transposed symbol and the adjoint Born iterations
    against the oracle."""
    p, s, _ = make(shape, seed=36, collocated=True)
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, collocated=True)
    v = W.random_source(shape, 38)
    out = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.green_apply(T(v), out, adjoint=True)
    assert rel(out.cpu().numpy(), P.green(v, adjoint=True)) <= 1e-12
    y = P.scale_source(v, True)
    x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    s.born_iterate(T(y), x, 30, adjoint=True)
    xr, _ = P.iterate(y, n_iter=30, nu=0.5, adjoint=True)
    assert rel(x.cpu().numpy(), xr) <= 1e-11


_FUSED_VARIANTS = [(v, sh) for v in ("0", "1", "2", "3", "6") for sh in ((16, 24, 128), (8, 16, 512), (24, 256))]
# the other float32 row lengths (192, 1024, 2048 points): three field
# buffers against the default, y staged in the transform's buffer
_FUSED_VARIANTS += [("0", sh) for sh in ((8, 12, 192), (8, 1024), (8, 2048))]


@pytest.mark.parametrize("var,shape", _FUSED_VARIANTS)
def test_fused_row_kernel_variants_match_default_and_oracle(var, shape, monkeypatch):
    """The fused update + next forward row kernel's variants (three field buffers, twiddles from the table, y
    staged in the transform's buffer, the last two together) give the default kernel's float32 Born iterations
    to rounding and match the oracle."""
    monkeypatch.setenv("CBS_FUSED_VAR", var)
    _, s, P = make(shape, seed=48, precision="fp32")
    monkeypatch.delenv("CBS_FUSED_VAR")
    _, s_ref, _ = make(shape, seed=48, precision="fp32")
    for adjoint in (False, True):
        y = P.scale_source(W.random_source(shape, 49), adjoint)
        x = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
        x_ref = torch.zeros_like(x)
        inc = s.born_iterate(T(y), x, 12, adjoint)
        inc_ref = s_ref.born_iterate(T(y), x_ref, 12, adjoint)
        assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-6
        assert np.allclose(inc, inc_ref, rtol=1e-5, atol=0)
        xr, _ = P.iterate(y, n_iter=12, nu=0.5, adjoint=adjoint)
        assert rel(x.cpu().numpy(), xr) <= 1e-5
