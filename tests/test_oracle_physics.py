"""Physics pins for the oracle, independent of its own formulas.

* Analytic series (App. C) self-checks: the incident series sums to the closed
  form, the interface conditions hold on both sides, zero contrast scatters
  nothing.
* P7: a point source in water with the absorbing layer matches the free-space
  Green's function (2D Hankel, 3D spherical wave) including its amplitude:
  pins the time convention, the source normalisation and the layer.
* 1-D interface: reflection coefficient (Z2 - Z1)/(Z2 + Z1), Z = rho c, for
  density-only and sound-speed-only jumps, converging under refinement: pins
  the density/sound-speed placement in the two rows.
* P8: scattering of a plane wave by a fluid disc against the Bessel series;
  the error (staircasing of a strong-contrast interface at 6 points per
  wavelength) must shrink under refinement at fixed geometry.
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W

OM = 2 * np.pi * W.F0


# --------------------------------------------------------- absorption (eq. 118)
def test_complex_sound_speed_attenuates_at_alpha():
    """alpha is an amplitude attenuation in Np/m: with the complex sound speed of eq. 118 and outgoing waves
    e^{-ikx} (e^{+i omega t}), the wavenumber k = omega / c has Im k = -alpha to first order in
    eps = alpha c0 / omega (the next term is eps^2 / 2 relative), so the wave decays as e^{-alpha x}, and
    Re k = omega / c0 to the same order.  Checked for the series' c and for the plain definition's c^2."""
    from oracle import dense

    c0 = 1500.0
    for alpha in (1.0, 10.0, 50.0):
        eps = alpha * c0 / OM
        one = np.full((2, 2), 1.0)
        _, _, _, c2 = dense.diagonals(c0 * one, 1000.0 * one, alpha * one, 1e-4, OM, ((0, 0), (0, 0)), 0.0)
        for c in (A.complex_c(c0, alpha, OM), np.sqrt(c2[0, 0])):
            k = OM / c
            assert k.imag < 0
            assert abs(-k.imag - alpha) <= eps ** 2 * alpha
            assert abs(k.real - OM / c0) <= eps ** 2 * OM / c0


# ------------------------------------------------------------ series self-checks
def test_sphere_incident_series_is_point_source():
    rng = np.random.default_rng(1)
    centre = np.zeros(3)
    src = np.array([0.05, 0.0, 0.0])
    pts = (rng.random((40, 3)) - 0.5) * 0.04
    ser = A.sphere_incident_series(pts, centre, src, OM, 1500.0, 1.0)
    k0 = OM / 1500.0
    R = np.linalg.norm(pts - src, axis=1)
    closed = np.exp(-1j * k0 * R) / (4 * np.pi * R)
    assert np.max(np.abs(ser - closed)) <= 1e-9 * np.max(np.abs(closed))


def test_sphere_no_contrast_scatters_nothing():
    Am, Bm, _, _ = A.sphere_coefficients(OM, 0.01, 1500.0, 1000.0, 1500.0, 1000.0, 0.0, 0.05, 1.0, m_max=60)
    assert np.max(np.abs(Am)) <= 1e-12 * np.max(np.abs(Bm))


@pytest.mark.parametrize("kind", ["sphere", "disc"])
def test_series_interface_conditions(kind):
    a, c1, r1, al1 = 0.008, 2200.0, 1600.0, 20.0
    eps = 1e-7
    th = np.linspace(0.1, 3.0, 6)
    if kind == "sphere":
        src = np.array([0.0, 0.0, 0.03])

        def p(r):
            pts = np.stack([r * np.sin(th), 0 * th, r * np.cos(th)], -1)
            return A.sphere_field(pts, np.zeros(3), src, OM, a, 1500.0, 1000.0, c1, r1, al1, 1.0, m_max=80)
    else:
        def p(r):
            pts = np.stack([r * np.sin(th), r * np.cos(th)], -1)
            inc, s = A.disc_fields(pts, np.zeros(2), OM, a, 1500.0, 1000.0, c1, r1, al1, m_max=80)
            return np.where(r > a, inc + s, s)
    po, pi = p(a + eps), p(a - eps)
    assert np.max(np.abs(po - pi)) <= 1e-3 * np.max(np.abs(pi))
    # (1/rho) dp/dr continuous (normal velocity)
    dpo = (p(a + 3 * eps) - po) / (2 * eps) / 1000.0
    dpi = (pi - p(a - 3 * eps)) / (2 * eps) / r1
    assert np.max(np.abs(dpo - dpi)) <= 1e-2 * np.max(np.abs(dpi))
    # and p itself is not trivially continuous in the derivative (density jump)
    assert np.max(np.abs(dpo * 1000.0 - dpi * r1)) > 1e-2 * np.max(np.abs(dpi * r1))


# --------------------------------------------------------------- point sources
def test_point_source_2d_matches_hankel():
    N, nabs = 96, 16
    p = W.inclusion_medium((N, N), 0, 1500.0, 1000.0, 0.0, ppw=6, n_abs=nabs)
    src = W.point_source((N, N), (N // 2, N // 2))
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    f, _, res = P.solve_field(src, 1e-8, check_every=50)
    yy, xx = np.mgrid[0:N, 0:N]
    R = np.hypot(xx - N // 2, yy - N // 2) * p.dx
    interior = (xx >= nabs) & (xx < N - nabs) & (yy >= nabs) & (yy < N - nabs)
    m = (R > 1500.0 / W.F0) & interior
    ref = A.point_source_2d(np.where(R > 0, R, 1.0), p.omega, 1500.0, p.dx)
    assert np.linalg.norm(f[2][m] - ref[m]) / np.linalg.norm(ref[m]) <= 2e-3
    # the time convention matters: the e^{+ikr} (incoming) wave does not fit
    wrong = np.conj(ref)
    assert np.linalg.norm(f[2][m] - wrong[m]) / np.linalg.norm(ref[m]) > 0.5


def test_point_source_3d_matches_spherical_wave():
    N, nabs = 40, 12
    p = W.inclusion_medium((N, N, N), 0, 1500.0, 1000.0, 0.0, ppw=6, n_abs=nabs)
    src = W.point_source((N, N, N), (N // 2, N // 2, N // 2))
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    f, _, _ = P.solve_field(src, 1e-7, check_every=50)
    zz, yy, xx = np.mgrid[0:N, 0:N, 0:N]
    R = np.sqrt((xx - N // 2) ** 2 + (yy - N // 2) ** 2 + (zz - N // 2) ** 2) * p.dx
    inn = lambda a: (a >= nabs) & (a < N - nabs)  # noqa: E731
    m = (R > 1500.0 / W.F0) & inn(xx) & inn(yy) & inn(zz)
    ref = A.point_source_3d(np.where(R > 0, R, 1.0), p.omega, 1500.0, p.dx)
    assert np.linalg.norm(f[3][m] - ref[m]) / np.linalg.norm(ref[m]) <= 6e-3


# ------------------------------------------------------------- 1-D interface
def _reflection(ppw, c2, r2, N=1024, nabs=128, xs=300, xi=700):
    dx = W.grid_step(ppw)
    k = OM / 1500.0
    c0, rho, al = np.full(N, 1500.0), np.full(N, 1000.0), np.zeros(N)
    gmax = W.layer_gamma_max(nabs, dx)
    src = np.zeros((2, N), complex)
    src[1, xs] = 1.0
    f0, _, _ = O.Problem(c0, rho, al, dx, OM, [[nabs, nabs]], gmax).solve_field(src, 1e-11, check_every=50)
    c1, r1 = c0.copy(), rho.copy()
    c1[xi:], r1[xi:] = c2, r2
    f1, _, _ = O.Problem(c1, r1, al, dx, OM, [[nabs, nabs]], gmax).solve_field(src, 1e-11, check_every=50)
    x = np.arange(N)
    x_int = xi - 0.5  # staggered point between the last medium-1 cell and the first medium-2 cell
    amp = f0[1][xs + 50] * np.exp(1j * k * 50 * dx)  # right-going wave amplitude at the source
    sel = (x > nabs + 10) & (x < xs - 10)
    R = (f1[1] - f0[1])[sel] * np.exp(1j * k * (2 * x_int - xs - x[sel]) * dx) / amp
    return R.mean()


@pytest.mark.parametrize("c2,r2", [(1500.0, 1100.0), (1650.0, 1000.0), (1500.0, 2000.0)])
def test_interface_reflection_coefficient(c2, r2):
    exact = (c2 * r2 - 1.5e6) / (c2 * r2 + 1.5e6)
    e6 = abs(_reflection(6, c2, r2) - exact) / abs(exact)
    e12 = abs(_reflection(12, c2, r2) - exact) / abs(exact)
    assert e12 <= 0.06
    assert e12 <= e6 / 3.0


# ------------------------------------------------------------------ disc series
def _disc_error(N, R0, nabs, ppw, cin=2500.0, rin=1800.0, a_db=1.0, tol=1e-7):
    p = W.inclusion_medium((N, N), R0, cin, rin, a_db, ppw=ppw, n_abs=nabs)
    m = p.meta
    src = A.scattered_field_source(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, m["centre"],
                                   1500.0, 1000.0)
    f, _, _ = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max).solve_field(src, tol,
                                                                                            check_every=50)
    yy, xx = np.mgrid[0:N, 0:N].astype(float)
    pts = np.stack([xx * p.dx, yy * p.dx], -1)
    inc, sc = A.disc_fields(pts, np.array(m["centre"], float) * p.dx, p.omega, R0 * p.dx, 1500.0, 1000.0,
                            cin, rin, m["alpha_in"])
    r = np.hypot(xx - m["centre"][0], yy - m["centre"][1])
    mask = (r > R0 * 1.2) & (xx >= nabs) & (xx < N - nabs) & (yy >= nabs) & (yy < N - nabs)
    return np.linalg.norm(f[2][mask] - sc[mask]) / np.linalg.norm(sc[mask])


@pytest.mark.slow
def test_disc_scattering_series_and_refinement():
    e6 = _disc_error(64, 9, 12, 6)
    e12 = _disc_error(128, 18, 24, 12)
    assert e6 <= 0.4
    assert e12 <= 0.15
    assert e12 <= e6 / 2.0
