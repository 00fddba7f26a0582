"""Physics checks of the CUDA path at the workloads' full sizes: the 128^2 disc
(FP64 to 1e-8) against the Bessel series and against the oracle, and the
128^3 sphere (FP32 + refinement to 1e-6) against the sphere series, with the
error falling under 2x refinement at fixed geometry (the staircased sharp
interface limits the accuracy at 6 points per wavelength)."""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def _disc_case(N, R0, nabs, ppw, precision, tol):
    from paper_2507_16087_gb300 import cbs

    p = W.inclusion_medium((N, N), R0, 2500.0, 1800.0, 1.0, ppw=ppw, n_abs=nabs)
    m = p.meta
    src = A.scattered_field_source(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, m["centre"], 1500.0,
                                   1000.0)
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max, precision=precision,
                          tol=tol)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(T(src), field)
    yy, xx = np.mgrid[0:N, 0:N].astype(float)
    pts = np.stack([xx * p.dx, yy * p.dx], -1)
    inc, sc = A.disc_fields(pts, np.array(m["centre"], float) * p.dx, p.omega, R0 * p.dx, 1500.0, 1000.0, 2500.0,
                            1800.0, m["alpha_in"])
    r = np.hypot(xx - m["centre"][0], yy - m["centre"][1])
    mask = (r > R0 * 1.2) & (xx >= nabs) & (xx < N - nabs) & (yy >= nabs) & (yy < N - nabs)
    f = field.cpu().numpy()
    err = np.linalg.norm(f[2][mask] - sc[mask]) / np.linalg.norm(sc[mask])
    return err, info, f, p, src


def test_disc_128_fp64_series_and_oracle():
    err, info, f, p, src = _disc_case(128, 20, 16, 6.0, "fp64", 1e-8)
    assert info["rel_residual"] <= 1e-8
    assert err <= 0.3
    # the oracle, run to the same residual, gives the same field within cond * tol
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    ref, _, _ = P.solve_field(src, 1e-10, check_every=50, nu=0.8)
    assert np.linalg.norm(f - ref) / np.linalg.norm(ref) <= 1e-6
    # refinement at fixed geometry (radius 3.33 wavelengths): 256^2 at 12 PPW
    err12, info12, _, _, _ = _disc_case(256, 40, 32, 12.0, "fp32_refine", 1e-7)
    assert err12 <= err / 2.0


def _sphere_error(n, radius, n_abs, src_offset, ppw):
    from paper_2507_16087_gb300 import cbs

    shape = (n, n, n)
    p = W.inclusion_medium(shape, radius, 2200.0, 1600.0, 2.0, ppw=ppw, n_abs=n_abs)
    c = p.meta["centre"]
    pos = (n_abs + src_offset, c[1], c[2])
    src = W.point_source(shape, pos)
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max,
                          precision="fp32_refine", tol=1e-6)
    field = torch.zeros(s.field_shape, dtype=torch.complex128, device=DEV)
    info = s.solve_forward(T(src), field)
    s.destroy()
    # central z-slice through the sphere and the source, outside 1 wavelength of the source and the layer
    k = c[2]
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    pts = np.stack([xx * p.dx, yy * p.dx, np.full_like(xx, k * p.dx)], -1)
    cen = np.array(c, float) * p.dx
    sp = np.array(pos, float) * p.dx
    amp = 1j * p.omega * p.dx ** 3 / 1500.0 ** 2  # single-voxel source normalisation
    ref = A.sphere_field(pts, cen, sp, p.omega, radius * p.dx, 1500.0, 1000.0, 2200.0, 1600.0, p.meta["alpha_in"],
                         amp, m_max=120)
    lam = 1500.0 / W.F0 / p.dx
    dsrc = np.hypot(xx - pos[0], yy - pos[1])
    inner = (xx >= n_abs) & (xx < n - n_abs) & (yy >= n_abs) & (yy < n - n_abs)
    mask = inner & (dsrc > lam)
    got = field[3, k].cpu().numpy()
    return np.linalg.norm(got[mask] - ref[mask]) / np.linalg.norm(ref[mask]), info


def test_sphere_128_against_series_and_refinement():
    err6, info = _sphere_error(128, 24, 20, 10, 6.0)
    assert info["rel_residual"] <= 1e-6
    assert err6 <= 0.35
    err12, _ = _sphere_error(256, 48, 40, 20, 12.0)
    assert err12 <= err6 / 2.0
