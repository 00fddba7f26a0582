"""Pins for the oracle's set-up and iteration.

* P2: the Born fixed point equals a dense LAPACK solve of the plain system, and
  does not depend on the shift rule, beta or nu (which only precondition).
* P3: the iteration matrix has spectral radius < 1 and the observed
  contraction of the increments approaches it.
* P4/P5: at exit the true residual is below the tolerance; the increment
  vanishes at the fixed point.
* P6: uniform medium -> exact per-wavenumber solution at any size.
* P9: reciprocity of the pressure-pressure block.
* P11: constant density -> the second-order Helmholtz equation of App. A.
* P12: adjoint solve against the dense A^H solve and the dot-product identity.
* Set-up invariants: Re a_j >= 0, Re diag >= 0, max|v_j| = beta, input checks.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W


def _problem(shape, seed, n_abs=2, gamma_scale=0.5, **kw):
    p = W.smooth_random_medium(shape, seed=seed, n_abs=n_abs, **kw)
    p.gamma_max = gamma_scale * p.omega
    return p


def _oracle(p, **kw):
    return O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power, **kw)


def _dense(p, src):
    return dense.solve(src, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape,seed", [((16, 16), 1), ((12, 10), 2), ((8, 8, 8), 3)])
def test_born_fixed_point_equals_dense_solve(shape, seed):
    p = _problem(shape, seed)
    src = W.random_source(shape, seed + 100)
    P = _oracle(p)
    field, it, res = P.solve_field(src, 1e-12, check_every=25)
    assert res <= 1e-12
    assert _rel(field, _dense(p, src)) <= 1e-10


@pytest.mark.parametrize("kw", [dict(shift_rule=O.SHIFT_MEDIAN), dict(beta=0.7), dict(beta=0.99)])
def test_solution_independent_of_preconditioner_choices(kw):
    shape = (12, 12)
    p = _problem(shape, 5)
    src = W.random_source(shape, 6)
    ref = _dense(p, src)
    f, _, _ = _oracle(p, **kw).solve_field(src, 1e-12, check_every=25)
    assert _rel(f, ref) <= 1e-10
    f, _, _ = _oracle(p).solve_field(src, 1e-12, check_every=25, nu=0.9)
    assert _rel(f, ref) <= 1e-10


def test_iteration_matrix_spectral_radius_below_one():
    shape = (10, 8)
    p = _problem(shape, 7)
    P = _oracle(p)
    C = P.ncomp
    n = C * int(np.prod(shape))
    v = P.v().ravel()
    B = 1 - v
    # dense (L+I) from the operator applied to unit vectors, then the iteration matrix
    # M = I - nu B + nu B (L+I)^-1 B  of x <- x + nu B [(L+I)^-1 (B x + y) - x]
    Lp = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        Lp[:, j] = P.apply(e.reshape(P.field_shape)).ravel() - v * e + e
    nu = 0.5
    G = np.linalg.inv(Lp)
    M = np.eye(n) - nu * np.diag(B) + nu * (B[:, None] * G * B[None, :])
    rho_M = np.max(np.abs(np.linalg.eigvals(M)))
    assert rho_M < 1.0
    # the increments of a long run contract at the spectral radius
    src = W.random_source(shape, 8)
    y = P.scale_source(src)
    _, inc = P.iterate(y, n_iter=200, nu=nu)
    # ||x_{k+1}-x_k|| / ||x_{k+1}|| over iterations 100..200 (||x|| has settled by then)
    ratio = (inc[199] / inc[99]) ** (1 / 100)
    assert ratio <= rho_M + 1e-3 and ratio >= rho_M - 1.5e-2


def test_residual_at_exit_and_vanishing_increment():
    shape = (16, 12)
    p = _problem(shape, 9)
    P = _oracle(p)
    y = P.scale_source(W.random_source(shape, 10))
    x, it, res = P.solve(y, 1e-9, check_every=7)
    assert res <= 1e-9 and it % 7 == 0
    # recomputed independently with the dense plain definition (scaled variables)
    sc = P.scalars()
    A = dense.assemble(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    D, N = len(shape), int(np.prod(shape))
    cinv = np.concatenate([np.full(D * N, sc["lambda1"] ** -0.5), np.full(N, sc["lambda2"] ** -0.5)])
    r = y.ravel() - cinv * (A @ (cinv * x.ravel()))
    assert np.linalg.norm(r) / np.linalg.norm(y) <= 1e-9 * (1 + 1e-6)
    x2, inc = P.iterate(y, x0=x, n_iter=1)
    assert inc[0] <= 1e-8


def test_increment_is_relative_and_scale_free():
    """Algorithm 1 stops on the relative increment ||x_{k+1} - x_k|| / ||x_{k+1}||: from a zero start x_1 - x_0 is
    x_1 itself, so the first increment is exactly 1; and the iteration is linear in y, so a source scaled by s
    scales every iterate by s and leaves every increment unchanged."""
    shape = (12, 10)
    p = _problem(shape, 21)
    P = _oracle(p)
    y = P.scale_source(W.random_source(shape, 22))
    x, inc = P.iterate(y, n_iter=8)
    assert abs(inc[0] - 1.0) <= 1e-14
    assert np.all(inc[1:] > 0) and np.all(inc[1:] < 1)
    s = 1e3 * (0.6 - 0.8j)
    xs, incs = P.iterate(s * y, n_iter=8)
    assert _rel(xs, s * x) <= 1e-12
    assert np.allclose(incs, inc, rtol=1e-10, atol=0)


@pytest.mark.parametrize("shape", [(32, 24), (12, 10, 8)])
def test_uniform_medium_closed_form(shape):
    dx = W.grid_step(6.0)
    om = 2 * np.pi * W.F0
    al = 20.0
    c0 = np.full(shape, 1500.0)
    rho = np.full(shape, 1000.0)
    alpha = np.full(shape, al)
    src = W.random_source(shape, 12)
    P = O.Problem(c0, rho, alpha, dx, om, [[0, 0]] * len(shape), 0.0)
    f, _, res = P.solve_field(src, 1e-12, check_every=50, max_iter=200000)
    ref = dense.uniform_solve(src, 1500.0, 1000.0, al, dx, om)
    assert _rel(f, ref) <= 1e-9


def test_reciprocity_pressure_block():
    shape = (16, 16)
    p = _problem(shape, 13)
    P = _oracle(p)
    a, b = (3, 4), (11, 9)
    ya = np.zeros(P.field_shape, dtype=np.complex128)
    yb = np.zeros(P.field_shape, dtype=np.complex128)
    ya[(2,) + a] = 1.0
    yb[(2,) + b] = 1.0
    xa, _, _ = P.solve(ya, 1e-12, check_every=25)
    xb, _, _ = P.solve(yb, 1e-12, check_every=25)
    assert abs(xa[(2,) + b] - xb[(2,) + a]) <= 1e-10 * abs(xa[(2,) + b])
    # velocity responses are not reciprocal in the same way (sanity: the test can fail)
    assert abs(xa[(0,) + b] - xb[(0,) + a]) > 1e-6 * abs(xa[(0,) + b])


@pytest.mark.parametrize("shape", [(16, 14), (8, 6, 6)])
def test_constant_density_reduces_to_second_order(shape):
    rng = np.random.default_rng(3)
    dx = W.grid_step(6.0)
    om = 2 * np.pi * W.F0
    c0 = 1500.0 + 600.0 * rng.random(shape)
    alpha = 10.0 + 10.0 * rng.random(shape)
    rho = np.full(shape, 1200.0)
    s_p = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    src = np.zeros((len(shape) + 1,) + shape, dtype=np.complex128)
    src[-1] = s_p
    p2 = dense.second_order_pressure(s_p, c0, alpha, dx, om)
    f1 = dense.solve(src, c0, rho, alpha, dx, om, [[0, 0]] * len(shape), 0.0)
    assert _rel(f1[-1], p2) <= 1e-11
    P = O.Problem(c0, rho, alpha, dx, om, [[0, 0]] * len(shape), 0.0)
    f, _, _ = P.solve_field(src, 1e-12, check_every=50, max_iter=400000)
    assert _rel(f[-1], p2) <= 1e-9


@pytest.mark.parametrize("shape", [(12, 12), (6, 6, 6)])
def test_adjoint_solve_matches_dense_and_dot_identity(shape):
    p = _problem(shape, 17)
    P = _oracle(p)
    g = W.random_source(shape, 18)
    yg = P.scale_source(g, adjoint=True)
    x, _, res = P.solve(yg, 1e-12, check_every=25, adjoint=True)
    lam = P.unscale(x)
    ref = dense.solve_adjoint(g, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    assert _rel(lam, ref) <= 1e-10
    # <A^-1 y1, y2> = <y1, A^-H y2> on the scaled system
    y1 = P.scale_source(W.random_source(shape, 19))
    y2 = P.scale_source(W.random_source(shape, 20))
    x1, _, _ = P.solve(y1, 1e-12, check_every=25)
    x2, _, _ = P.solve(y2, 1e-12, check_every=25, adjoint=True)
    lhs, rhs = np.vdot(y2, x1), np.vdot(x2, y1)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


# ------------------------------------------------------------------ set-up invariants
def test_setup_invariants():
    shape = (20, 16)
    p = _problem(shape, 23, n_abs=4, gamma_scale=1.0)
    P = _oracle(p)
    sc = P.scalars()
    v = P.v()
    beta = 0.95
    assert sc["a1"].real >= 0 and sc["a2"].real >= 0
    d = sc["a1"] + sc["lambda1"] * v[:-1]
    q = sc["a2"] + sc["lambda2"] * v[-1]
    assert d.real.min() >= -1e-9 * abs(sc["a1"]) and q.real.min() >= -1e-12 * abs(sc["a2"])
    # |v| <= beta with equality attained (eq. C)
    assert np.isclose(np.abs(v[:-1]).max(), beta, rtol=1e-14)
    assert np.isclose(np.abs(v[-1]).max(), beta, rtol=1e-14)
    # midrange: the bounding box of the diagonal values is centred on the shift
    assert np.isclose(d.real.min() + d.real.max(), 2 * sc["a1"].real, rtol=1e-12)
    assert np.isclose(d.imag.min() + d.imag.max(), 2 * sc["a1"].imag, rtol=1e-12)
    assert np.isclose(q.imag.min() + q.imag.max(), 2 * sc["a2"].imag, rtol=1e-12)
    # velocity diagonal: Im d = omega * staggered density (App. B.1)
    rs = 0.5 * (p.rho + np.roll(p.rho, -1, axis=1))
    assert np.allclose(d[0].imag, p.omega * rs, rtol=1e-12)


def test_median_shift_rule():
    shape = (9, 7)
    p = _problem(shape, 29)
    P = _oracle(p, shift_rule=O.SHIFT_MEDIAN)
    sc = P.scalars()
    dg, q, _, _ = dense.diagonals(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    dv = np.concatenate([x.ravel() for x in dg])
    assert np.isclose(sc["a1"], np.median(dv.real) + 1j * np.median(dv.imag), rtol=1e-13)
    assert np.isclose(sc["a2"], np.median(q.real) + 1j * np.median(q.imag), rtol=1e-13)


def test_uniform_no_layer_degenerate_scaling():
    shape = (8, 8)
    om = 2 * np.pi * W.F0
    P = O.Problem(np.full(shape, 1500.0), np.full(shape, 1000.0), np.zeros(shape), W.grid_step(6), om,
                  [[0, 0]] * 2, 0.0)
    sc = P.scalars()
    # max|d - a1| = 0: lambda falls back to |a|
    assert np.isclose(sc["lambda1"], abs(sc["a1"])) and np.isclose(sc["lambda2"], abs(sc["a2"]))
    assert np.allclose(P.v(), 0)


@pytest.mark.parametrize("bad", ["c_zero", "rho_neg", "alpha_neg", "nan"])
def test_invalid_inputs_rejected(bad):
    shape = (6, 6)
    c0, rho, al = np.full(shape, 1500.0), np.full(shape, 1000.0), np.zeros(shape)
    if bad == "c_zero":
        c0[2, 2] = 0
    elif bad == "rho_neg":
        rho[1, 3] = -5
    elif bad == "alpha_neg":
        al[0, 0] = -1
    else:
        c0[4, 4] = np.nan
    with pytest.raises(ValueError):
        O.Problem(c0, rho, al, 1e-3, 1e6, [[1, 1]] * 2, 1e5)


def _mec_brute(pts):
    """Smallest circle over all pair / triple circles containing every point (O(n^4), tiny n)."""
    best = (None, np.inf)
    n = len(pts)
    cands = []
    for i in range(n):
        for j in range(i + 1, n):
            cands.append(((pts[i] + pts[j]) / 2, abs(pts[i] - pts[j]) / 2))
            for k in range(j + 1, n):
                a, b, c = pts[i], pts[j], pts[k]
                d = 2 * (a.real * (b.imag - c.imag) + b.real * (c.imag - a.imag) + c.real * (a.imag - b.imag))
                if d == 0:
                    continue
                ux = (abs(a) ** 2 * (b.imag - c.imag) + abs(b) ** 2 * (c.imag - a.imag) + abs(c) ** 2 * (a.imag - b.imag)) / d
                uy = (abs(a) ** 2 * (c.real - b.real) + abs(b) ** 2 * (a.real - c.real) + abs(c) ** 2 * (b.real - a.real)) / d
                cands.append((ux + 1j * uy, abs(a - (ux + 1j * uy))))
    for c, r in cands:
        if r < best[1] and np.all(np.abs(pts - c) <= r * (1 + 1e-9)):
            best = (c, r)
    return best


def test_mec_shift_is_the_minimum_enclosing_circle():
    shape = (5, 4)
    p = _problem(shape, 31, n_abs=1, gamma_scale=0.7)
    P = _oracle(p, shift_rule=O.SHIFT_MEC)
    sc = P.scalars()
    dg, q, _, _ = dense.diagonals(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    dv = np.concatenate([x.ravel() for x in dg])
    c1, r1 = _mec_brute(dv)
    c2, r2 = _mec_brute(q.ravel())
    assert abs(sc["a1"] - c1) <= 1e-9 * r1 and abs(sc["a2"] - c2) <= 1e-9 * r2
    # with beta the largest |v| is beta, and no other centre has a smaller enclosing radius
    assert np.isclose(sc["lambda1"] * 0.95, r1, rtol=1e-9) and np.isclose(sc["lambda2"] * 0.95, r2, rtol=1e-9)
    Pm = _oracle(p)
    assert Pm.scalars()["lambda1"] >= sc["lambda1"] * (1 - 1e-12)


def test_mec_shift_same_solution():
    shape = (12, 12)
    p = _problem(shape, 32)
    src = W.random_source(shape, 33)
    f, _, _ = _oracle(p, shift_rule=O.SHIFT_MEC).solve_field(src, 1e-12, check_every=25)
    assert _rel(f, _dense(p, src)) <= 1e-10


@pytest.mark.parametrize("shape", [(12, 10), (6, 8, 6)])
def test_collocated_variant_matches_dense_and_symbol_identity(shape):
    """App. B's collocated grid: the Born fixed point equals the dense collocated system; (L+I)^-1 inverts L+I."""
    p = _problem(shape, 37)
    src = W.random_source(shape, 38)
    P = _oracle(p, collocated=True)
    f, _, _ = P.solve_field(src, 1e-12, check_every=25)
    ref = dense.solve(src, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power, collocated=True)
    assert _rel(f, ref) <= 1e-10
    # differs from the staggered solution (the variant changes the discretisation)
    assert _rel(f, _dense(p, src)) > 1e-4
    x = W.random_source(shape, 39)
    v = P.v()
    Lx = P.apply(x) - v * x
    assert np.max(np.abs(P.green(Lx + x) - x)) <= 1e-12 * np.max(np.abs(x))
