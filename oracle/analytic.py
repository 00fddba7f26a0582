"""Analytic fields for the physics pins: free-space point sources and the fluid
disc / sphere scattering series (App. C of Stanziola et al., arXiv 2507.16087,
which follows Anderson 1950 / McNew et al. 2009).

TEST INFRASTRUCTURE.

Time convention.  The first-order system i omega u + grad p / rho + gamma u = s_u
with gamma >= 0 and alpha >= 0 gives wavenumbers with Im k <= 0, so outgoing
waves are e^{-i k r}: the e^{+i omega t} convention.  Hence spherical Hankel
h_m^(2) = j_m - i y_m and cylindrical H_m^(2) = J_m - i Y_m below, and a plane
wave travelling in +y is e^{-i k y}.

Point-source normalisation.  A single-voxel pressure source s_p = S on a grid
of step dx is, for a spectral discretisation, a band-limited spike of integral
S dx^D, so (lap + k^2) p = -i omega S dx^D / c^2 delta and
  3D: p = (i omega S dx^3 / c^2) e^{-i k R} / (4 pi R)
  2D: p = (i omega S dx^2 / c^2) (-i/4) H_0^(2)(k R)
(App. A gives the equivalent second-order source -i omega s_p / c^2).

Interface conditions (App. C): continuity of p and of the normal velocity,
which for u_r = (i / (rho c)) dp/d(kr) is continuity of (1/Z) dp/d(kr),
Z = rho c.  Inside an absorbing scatterer c is the complex sound speed of
eq. 118 (principal root), k = omega / c, Z = rho c.

App. C writes the monopole coefficient as h_m(k0 R) with R the sphere radius;
the addition theorem for a source at distance r_s from the centre gives
h_m(k0 r_s) (times -i k0 / (4 pi) for a unit e^{-ikR}/(4 pi R) source), which
is used here.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def complex_c(c0, alpha, omega):
    """Complex sound speed c = sqrt(c0^2 / (1 - 2 i alpha c0 / omega)) (eq. 118), principal root."""
    return np.sqrt(c0 ** 2 / (1 - 2j * alpha * c0 / omega))


def h2(m, z, derivative=False):
    return special.spherical_jn(m, z, derivative=derivative) - 1j * special.spherical_yn(m, z, derivative=derivative)


def H2(m, z):
    return special.hankel2(m, z)


def H2p(m, z):
    return special.h2vp(m, z)


# ---------------------------------------------------------------- point sources
def point_source_3d(R, omega, c, dx, S=1.0):
    k = omega / c
    return (1j * omega * S * dx ** 3 / c ** 2) * np.exp(-1j * k * R) / (4 * np.pi * R)


def point_source_2d(R, omega, c, dx, S=1.0):
    k = omega / c
    return (1j * omega * S * dx ** 2 / c ** 2) * (-0.25j) * H2(0, k * R)


# ------------------------------------------------------------------------ sphere
def sphere_coefficients(omega, a, c0, rho0, c1, rho1, alpha1, r_s, amp, m_max=150):
    """A_m (scattered, outside) and B_m (inside) for a monopole of complex amplitude ``amp`` (field
    amp e^{-ikR}/(4 pi R)) at distance r_s from the centre of a fluid sphere of radius a.

    Per order m the 2x2 interface system of App. C is solved directly:
      (2m+1) L_m j'_m(k0 a)/Z0 + h'_m(k0 a) A_m / Z0 = j'_m(k1 a) B_m / Z1
      (2m+1) L_m j_m(k0 a)     + h_m(k0 a) A_m       = j_m(k1 a) B_m
    with L_m = amp (-i k0 / (4 pi)) h_m(k0 r_s)."""
    k0 = omega / c0
    cc1 = complex_c(c1, alpha1, omega)
    k1 = omega / cc1
    Z0, Z1 = rho0 * c0, rho1 * cc1
    A = np.zeros(m_max + 1, dtype=np.complex128)
    B = np.zeros(m_max + 1, dtype=np.complex128)
    for m in range(m_max + 1):
        L = amp * (-1j * k0 / (4 * np.pi)) * h2(m, k0 * r_s)
        M = np.array([[h2(m, k0 * a, True) / Z0, -special.spherical_jn(m, k1 * a, derivative=True) / Z1],
                      [h2(m, k0 * a), -special.spherical_jn(m, k1 * a)]], dtype=np.complex128)
        rhs = -(2 * m + 1) * L * np.array([special.spherical_jn(m, k0 * a, derivative=True) / Z0,
                                             special.spherical_jn(m, k0 * a)])
        A[m], B[m] = np.linalg.solve(M, rhs)
    return A, B, k0, k1


def sphere_field(points, centre, src, omega, a, c0, rho0, c1, rho1, alpha1, amp, m_max=150):
    """Total pressure at ``points`` (..., 3) for the monopole at ``src``: closed-form incident field
    outside plus the scattered series; the interior series inside."""
    points = np.asarray(points, dtype=np.float64)
    centre = np.asarray(centre, dtype=np.float64)
    src = np.asarray(src, dtype=np.float64)
    axis = src - centre
    r_s = np.linalg.norm(axis)
    axis = axis / r_s
    rel = points - centre
    r = np.linalg.norm(rel, axis=-1)
    cos_t = np.where(r > 0, (rel @ axis) / np.where(r > 0, r, 1.0), 1.0)
    A, B, k0, k1 = sphere_coefficients(omega, a, c0, rho0, c1, rho1, alpha1, r_s, amp, m_max)
    out = np.zeros(r.shape, dtype=np.complex128)
    inside = r < a
    ro, co = r[~inside], cos_t[~inside]
    ri, ci = r[inside], cos_t[inside]
    so = np.zeros(ro.shape, dtype=np.complex128)
    si = np.zeros(ri.shape, dtype=np.complex128)
    for m in range(m_max + 1):
        so += A[m] * special.eval_legendre(m, co) * h2(m, k0 * ro)
        si += B[m] * special.eval_legendre(m, ci) * special.spherical_jn(m, k1 * ri)
    R = np.linalg.norm(points[~inside] - src, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):  # the source point itself is singular
        out[~inside] = amp * np.exp(-1j * k0 * R) / (4 * np.pi * R) + so
    out[inside] = si
    return out


def sphere_incident_series(points, centre, src, omega, c0, amp, m_max=150):
    """Incident monopole field as its order-by-order series (valid for r < r_s)."""
    points = np.asarray(points, dtype=np.float64)
    axis = np.asarray(src, float) - np.asarray(centre, float)
    r_s = np.linalg.norm(axis)
    axis = axis / r_s
    rel = points - np.asarray(centre, float)
    r = np.linalg.norm(rel, axis=-1)
    cos_t = (rel @ axis) / r
    k0 = omega / c0
    out = np.zeros(r.shape, dtype=np.complex128)
    for m in range(m_max + 1):
        L = amp * (-1j * k0 / (4 * np.pi)) * h2(m, k0 * r_s)
        out += (2 * m + 1) * L * special.eval_legendre(m, cos_t) * special.spherical_jn(m, k0 * r)
    return out


# -------------------------------------------------------------------------- disc
def disc_coefficients(omega, a, c0, rho0, c1, rho1, alpha1, m_max=150):
    """Plane wave e^{-i k0 (y - y_c)} (phase referenced to the disc centre) on a fluid disc of radius a: p_inc = sum eps_m (-i)^m J_m(k0 r) cos(m th),
    p_sc = sum A_m H_m^(2)(k0 r) cos(m th), p_in = sum B_m J_m(k1 r) cos(m th), th from +y.
    Interface: p and (1/Z) dp/d(kr) continuous (the 2D form of App. C)."""
    k0 = omega / c0
    cc1 = complex_c(c1, alpha1, omega)
    k1 = omega / cc1
    Z0, Z1 = rho0 * c0, rho1 * cc1
    A = np.zeros(m_max + 1, dtype=np.complex128)
    B = np.zeros(m_max + 1, dtype=np.complex128)
    for m in range(m_max + 1):
        inc = (1.0 if m == 0 else 2.0) * (-1j) ** m
        M = np.array([[H2p(m, k0 * a) / Z0, -special.jvp(m, k1 * a) / Z1],
                      [H2(m, k0 * a), -special.jv(m, k1 * a)]], dtype=np.complex128)
        rhs = -inc * np.array([special.jvp(m, k0 * a) / Z0, special.jv(m, k0 * a)])
        A[m], B[m] = np.linalg.solve(M, rhs)
    return A, B, k0, k1


def disc_fields(points, centre, omega, a, c0, rho0, c1, rho1, alpha1, m_max=150):
    """(incident, scattered-or-interior) pressure at ``points`` (..., 2) in (x, y) order.  Outside the
    disc the second array is the scattered field; inside it is the total interior field."""
    points = np.asarray(points, dtype=np.float64)
    rel = points - np.asarray(centre, float)
    r = np.hypot(rel[..., 0], rel[..., 1])
    th = np.arctan2(rel[..., 0], rel[..., 1])  # angle from +y
    A, B, k0, k1 = disc_coefficients(omega, a, c0, rho0, c1, rho1, alpha1, m_max)
    inc = np.exp(-1j * k0 * rel[..., 1])
    out = np.zeros(r.shape, dtype=np.complex128)
    inside = r < a
    for m in range(m_max + 1):
        cm = np.cos(m * th)
        out[~inside] += A[m] * H2(m, k0 * r[~inside]) * cm[~inside]
        out[inside] += B[m] * special.jv(m, k1 * r[inside]) * cm[inside]
    return inc, out


def disc_incident_series(points, centre, omega, c0, m_max=150):
    points = np.asarray(points, dtype=np.float64)
    rel = points - np.asarray(centre, float)
    r = np.hypot(rel[..., 0], rel[..., 1])
    th = np.arctan2(rel[..., 0], rel[..., 1])
    k0 = omega / c0
    out = np.zeros(r.shape, dtype=np.complex128)
    for m in range(m_max + 1):
        out += (1.0 if m == 0 else 2.0) * (-1j) ** m * special.jv(m, k0 * r) * np.cos(m * th)
    return out


def scattered_field_source(c0, rho, alpha, dx, omega, nabs, gamma_max, centre, c_bg, rho_bg, power=2.0):
    """Physical source whose solution is the field scattered by the inclusion under the plane wave
    p_inc = e^{-i k0 (y - y_c)}, u_inc = (0, p_inc / (rho_bg c_bg)): with D the diagonal block of the
    row-scaled system and D_bg the same for the background medium (same layer), the row-scaled source
    is -(D - D_bg) X_inc, nonzero only where the medium differs from the background.  Returned in
    physical form (s_u = s_hat_u / (S+ rho), s_p = s_hat_p rho c^2) for a 2D grid."""
    from . import dense

    shape = c0.shape
    assert len(shape) == 2
    k0 = omega / c_bg
    ny, nx = shape
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    yc = centre[1]
    p_c = np.exp(-1j * k0 * (yy - yc) * dx)            # p at cell centres
    p_sy = np.exp(-1j * k0 * (yy + 0.5 - yc) * dx)     # at the u_y staggered points
    u_y = p_sy / (rho_bg * c_bg)
    d, q, rho_s, c2 = dense.diagonals(c0, rho, alpha, dx, omega, nabs, gamma_max, power)
    bg = np.ones(shape)
    d0, q0, _, _ = dense.diagonals(c_bg * bg, rho_bg * bg, 0 * bg, dx, omega, nabs, gamma_max, power)
    s = np.zeros((3,) + shape, dtype=np.complex128)
    s[1] = -(d[1] - d0[1]) * u_y / rho_s[1]
    s[2] = -(q - q0) * p_c * (rho * c2)
    return s
