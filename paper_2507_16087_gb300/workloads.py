"""Seeded synthetic inputs for the Born solver (media, sources, grid units).

This module only builds inputs: sound speed c0 (m/s), density rho (kg/m^3),
absorption alpha (Np/m), grid step, angular frequency, absorbing-layer
parameters and sources.  It holds none of the solver's arithmetic, so both the
CUDA path and the FP64 CPU oracle can take their inputs from it.

Units (the paper's experiments run at 500 kHz in water, Sec. 3):
  f = 500 kHz, background c = 1500 m/s, grid step dx = c_bg / (f * PPW),
  alpha [Np/m] = alpha0 [dB/cm/MHz] * f[MHz] * 100 / (20 log10 e)
  (linear frequency power law).
Absorbing layer: n_abs cells inside the grid on every side, quadratic profile,
gamma_max = 3 c_ref ln(1/R) / (2 n_abs dx) with R = 1e-4, the nominal
normal-incidence round-trip reflection of a quadratic layer.

Arrays are numpy float64 with shape (n[D-1], ..., n[0]) (x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F0 = 5.0e5
C_WATER = 1500.0
RHO_WATER = 1000.0
NEPER_PER_DB = 1.0 / (20.0 * math.log10(math.e))


def db_cm_mhz_to_np_m(alpha0: float, f_hz: float = F0) -> float:
    """Absorption in dB/(cm MHz) -> Np/m at frequency f (linear power law)."""
    return alpha0 * (f_hz / 1e6) * 100.0 * NEPER_PER_DB


def grid_step(ppw: float, f_hz: float = F0, c_bg: float = C_WATER) -> float:
    return c_bg / (f_hz * ppw)


def layer_gamma_max(n_abs: int, dx: float, c_ref: float = C_WATER, refl: float = 1e-4) -> float:
    """Peak absorption of a quadratic layer of n_abs cells with round-trip reflection ``refl``."""
    return 3.0 * c_ref * math.log(1.0 / refl) / (2.0 * n_abs * dx)


@dataclass
class Problem:
    """One solve's inputs.  ``source`` has shape (D+1, *shape): (s_u..., s_p)."""

    name: str
    c0: np.ndarray
    rho: np.ndarray
    alpha: np.ndarray
    dx: float
    omega: float
    nabs: list
    gamma_max: float
    power: float = 2.0
    source: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.c0.shape

    @property
    def ndim(self):
        return self.c0.ndim

    @property
    def n_voxels(self):
        return int(np.prod(self.c0.shape))


def _centre_dist(shape, centre):
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    # grids are in numpy axis order (..., y, x); centre is given in (x, y, z) order
    r2 = np.zeros(shape)
    for ax in range(len(shape)):
        r2 += (grids[ax] - centre[len(shape) - 1 - ax]) ** 2
    return np.sqrt(r2)


def inclusion_medium(shape, radius, c_in, rho_in, alpha_in_db, centre=None, ppw=6.0, n_abs=16,
                     f_hz=F0, c_bg=C_WATER, rho_bg=RHO_WATER):
    """Water with one centred disc (2D) or sphere (3D); inside = cell-centre distance < radius."""
    if centre is None:
        centre = tuple(s // 2 for s in shape[::-1])
    dx = grid_step(ppw, f_hz, c_bg)
    r = _centre_dist(shape, centre)
    inside = r < radius
    c0 = np.where(inside, c_in, c_bg).astype(np.float64)
    rho = np.where(inside, rho_in, rho_bg).astype(np.float64)
    alpha = np.where(inside, db_cm_mhz_to_np_m(alpha_in_db, f_hz), 0.0).astype(np.float64)
    nabs = [[n_abs, n_abs] for _ in shape]
    return Problem(name="inclusion", c0=c0, rho=rho, alpha=alpha, dx=dx, omega=2 * math.pi * f_hz, nabs=nabs,
                   gamma_max=layer_gamma_max(n_abs, dx, c_bg) if n_abs > 0 else 0.0,
                   meta=dict(radius=radius, centre=centre, c_in=c_in, rho_in=rho_in,
                             alpha_in=db_cm_mhz_to_np_m(alpha_in_db, f_hz), c_bg=c_bg, rho_bg=rho_bg, ppw=ppw,
                             n_abs=n_abs, f=f_hz))


def point_source(shape, pos_xyz, amplitude=1.0 + 0j):
    """Single-voxel pressure source s_p at cell pos (x, y, z order); zero velocity sources."""
    src = np.zeros((len(shape) + 1,) + tuple(shape), dtype=np.complex128)
    idx = tuple(pos_xyz[::-1])
    src[(len(shape),) + idx] = amplitude
    return src


def disc_128():
    """2D 128x128: water, disc radius 20 cells (c 2500, rho 1800, 1 dB/cm/MHz), 6 PPW, 16-cell layer."""
    p = inclusion_medium((128, 128), 20, 2500.0, 1800.0, 1.0, ppw=6.0, n_abs=16)
    p.name = "disc2d_128"
    return p


def sphere_128(n=128, radius=24, n_abs=20, src_offset=10):
    """3D n^3: water, sphere radius 24 (c 2200, rho 1600, 2 dB/cm/MHz), 6 PPW, 20-cell layer, point source
    ``src_offset`` cells inside the layer's inner edge on the -x side, on the sphere's axis."""
    shape = (n, n, n)
    p = inclusion_medium(shape, radius, 2200.0, 1600.0, 2.0, ppw=6.0, n_abs=n_abs)
    c = p.meta["centre"]
    pos = (n_abs + src_offset, c[1], c[2])
    p.source = point_source(shape, pos)
    p.meta["source_pos"] = pos
    p.name = f"sphere3d_{n}"
    return p


def smooth_random_medium(shape, seed, c_range=(1400.0, 2800.0), rho_range=(900.0, 1900.0),
                         alpha_db_range=(0.0, 5.0), sigma_frac=1.0 / 16, ppw=6.0, n_abs=16, f_hz=F0):
    """Uniform noise smoothed by a periodic Gaussian (sigma = sigma_frac * n), affinely mapped to ranges."""
    rng = np.random.default_rng(seed)

    def smooth():
        a = rng.random(shape)
        A = np.fft.fftn(a)
        g = np.ones(shape)
        for ax, n in enumerate(shape):
            k = np.fft.fftfreq(n)
            s = sigma_frac * n
            sh = [1] * len(shape)
            sh[ax] = n
            g = g * np.exp(-2.0 * (math.pi * k * s) ** 2).reshape(sh)
        b = np.real(np.fft.ifftn(A * g))
        lo, hi = b.min(), b.max()
        return (b - lo) / (hi - lo if hi > lo else 1.0)

    c0 = c_range[0] + (c_range[1] - c_range[0]) * smooth()
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * smooth()
    al = alpha_db_range[0] + (alpha_db_range[1] - alpha_db_range[0]) * smooth()
    alpha = al * db_cm_mhz_to_np_m(1.0, f_hz)
    dx = grid_step(ppw, f_hz)
    nabs = [[n_abs, n_abs] for _ in shape]
    return Problem(name=f"random{len(shape)}d", c0=c0, rho=rho, alpha=alpha, dx=dx, omega=2 * math.pi * f_hz,
                   nabs=nabs, gamma_max=layer_gamma_max(n_abs, dx) if n_abs > 0 else 0.0, meta=dict(seed=seed))


def random_source(shape, seed, velocity=True):
    """Dense complex Gaussian source in every component (parity-test input)."""
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((len(shape) + 1,) + tuple(shape)) + 1j * rng.standard_normal((len(shape) + 1,) + tuple(shape))
    if not velocity:
        s[:-1] = 0
    return s


def layered_inversion(n=128, n_abs=20, seed=3, n_slabs=5, pert=0.03, sigma=4.0, ppw=6.0, f_hz=F0,
                      src_grid=(4, 2), rec_grid=(8, 8), n_fd=20, fd_seed=33):
    """Adjoint / gradient workload: 5 random-thickness slabs along z (c ~ U(1400, 3000), rho ~ U(900, 2000),
    alpha = 0) plus a 3 % periodic-Gaussian-smoothed (sigma cells) random perturbation; point pressure sources
    on a 4 x 2 grid and receivers on an 8 x 8 grid, all on the plane z = n_abs + 2.  Returns a dict with the
    layered (data) medium, the perturbed medium, sources (S, 4, n, n, n), receiver index arrays and seeded
    interior voxels for finite-difference checks."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    lo, hi = n_abs, n - n_abs
    depth = hi - lo
    min_thick = max(1, min(4, depth // n_slabs))  # 4 cells when the interior allows it
    for _ in range(10000):
        cuts = np.sort(rng.uniform(0, depth, n_slabs - 1))
        edges = np.concatenate([[0.0], cuts, [float(depth)]]).round().astype(int)
        if np.all(np.diff(edges) >= min_thick):
            break
    else:  # equal slabs
        edges = np.linspace(0, depth, n_slabs + 1).round().astype(int)
    c_s = rng.uniform(1400.0, 3000.0, n_slabs)
    r_s = rng.uniform(900.0, 2000.0, n_slabs)
    zc = np.clip(np.arange(n) - lo, 0, depth - 1)
    slab = np.searchsorted(edges[1:], zc, side="right")
    slab = np.clip(slab, 0, n_slabs - 1)
    c_lay = np.broadcast_to(c_s[slab][:, None, None], shape).astype(np.float64).copy()
    r_lay = np.broadcast_to(r_s[slab][:, None, None], shape).astype(np.float64).copy()

    def smooth_noise():
        a = rng.standard_normal(shape)
        A = np.fft.fftn(a)
        g = np.ones(shape)
        for ax in range(3):
            k = np.fft.fftfreq(n)
            sh = [1, 1, 1]
            sh[ax] = n
            g = g * np.exp(-2.0 * (math.pi * k * sigma) ** 2).reshape(sh)
        b = np.real(np.fft.ifftn(A * g))
        return b / b.std()

    c_pert = c_lay * (1.0 + pert * smooth_noise())
    r_pert = r_lay * (1.0 + pert * smooth_noise())
    dx = grid_step(ppw, f_hz)
    z = n_abs + 2
    sx = np.linspace(lo + 8, hi - 8, src_grid[0]).round().astype(int)
    sy = np.linspace(lo + 8, hi - 8, src_grid[1]).round().astype(int)
    srcs = []
    for yy in sy:
        for xx in sx:
            srcs.append(point_source(shape, (int(xx), int(yy), z))[None])
    sources = np.concatenate(srcs, axis=0)
    rx = np.linspace(lo + 4, hi - 4, rec_grid[0]).round().astype(int)
    ry = np.linspace(lo + 4, hi - 4, rec_grid[1]).round().astype(int)
    RY, RX = np.meshgrid(ry, rx, indexing="ij")
    rec = (np.full(RX.size, z), RY.ravel(), RX.ravel())  # numpy (z, y, x) order
    frng = np.random.default_rng(fd_seed)
    fd = frng.integers(lo + 2, hi - 2, size=(n_fd, 3))  # (z, y, x)
    return dict(shape=shape, dx=dx, omega=2 * math.pi * f_hz, nabs=[[n_abs, n_abs]] * 3,
                gamma_max=layer_gamma_max(n_abs, dx), c_layered=c_lay, rho_layered=r_lay, c0=c_pert, rho=r_pert,
                alpha=np.zeros(shape), sources=sources, receivers=rec, fd_voxels=fd)


def _smooth_noise(shape, sigma, rng, dtype=np.float32):
    """Unit-std white noise smoothed by a periodic Gaussian of width sigma cells (separable, per axis)."""
    a = rng.standard_normal(shape).astype(dtype)
    for ax, n in enumerate(shape):
        k = np.fft.rfftfreq(n) if ax == len(shape) - 1 else np.fft.fftfreq(n)
        g = np.exp(-2.0 * (math.pi * k * sigma) ** 2).astype(dtype)
        sh = [1] * len(shape)
        sh[ax] = g.size
        if ax == len(shape) - 1:
            a = np.fft.irfft(np.fft.rfft(a, axis=ax) * g.reshape(sh), n=n, axis=ax).astype(dtype)
        else:
            a = np.real(np.fft.ifft(np.fft.fft(a, axis=ax) * g.reshape(sh), axis=ax)).astype(dtype)
    return a / a.std()


def skull_shell(n=512, n_abs=24, seed=5, r_in=180.0, r_out=200.0, mod_amp=6.0, mod_sigma=8.0, var=0.02,
                var_sigma=4.0, aperture=300.0, roc=300.0, ppw=6.0, f_hz=F0):
    """Transcranial-like stand-in: a spherical shell (c 2800, rho 1850, 8 dB/cm/MHz) between radii r_in and
    r_out (outer radius modulated by smoothed noise, |mod| <= mod_amp cells) in water, with a 2 % smoothed
    variation of c and rho inside the shell; a focused bowl pressure source (spherical cap of radius of
    curvature `roc`, aperture `aperture` cells, apex on the -x face at x = n_abs + 2, axis +x), uniform
    amplitude on the cap voxels.  Synthetic: the paper's benchmark skull mesh is not available."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    c = (n - 1) / 2.0
    ax = np.arange(n, dtype=np.float32) - c
    z2 = (ax ** 2)[:, None, None]
    y2 = (ax ** 2)[None, :, None]
    x2 = (ax ** 2)[None, None, :]
    r = np.sqrt(z2 + y2 + x2, dtype=np.float32)
    mod = _smooth_noise(shape, mod_sigma, rng)
    mod = np.clip(mod / max(float(np.abs(mod).max()), 1e-30) * mod_amp, -mod_amp, mod_amp)
    shell = (r >= r_in) & (r < r_out + mod)
    del mod
    inner = r < r_in
    del r
    vc = _smooth_noise(shape, var_sigma, rng)
    vr = _smooth_noise(shape, var_sigma, rng)
    c0 = np.where(inner, C_WATER * (1.0 + var * vc), C_WATER).astype(np.float64)
    rho = np.where(inner, RHO_WATER * (1.0 + var * vr), RHO_WATER).astype(np.float64)
    del vc, vr
    c0[shell] = 2800.0
    rho[shell] = 1850.0
    alpha = np.zeros(shape)
    alpha[shell] = db_cm_mhz_to_np_m(8.0, f_hz)
    del shell, inner
    # bowl: voxels within half a cell of the sphere of radius roc centred at (apex + roc, c, c), lateral
    # distance <= aperture / 2, on the apex side
    x_apex = n_abs + 2
    xs = np.arange(n, dtype=np.float64)
    depth = roc - math.sqrt(roc ** 2 - (aperture / 2) ** 2)
    xmax = int(math.ceil(x_apex + depth)) + 2
    sub = np.zeros((n, n, xmax), dtype=bool)
    lat2 = ((xs[:, None] - c) ** 2 + (xs[None, :] - c) ** 2)[:, :, None]
    dist = np.sqrt(lat2 + (xs[None, None, :xmax] - (x_apex + roc)) ** 2)
    sub[:] = (np.abs(dist - roc) < 0.5) & (lat2 <= (aperture / 2) ** 2) & (xs[None, None, :xmax] <= x_apex + roc)
    src = np.zeros((4,) + shape, dtype=np.complex128)
    src[3, :, :, :xmax][sub] = 1.0
    dx = grid_step(ppw, f_hz)
    return Problem(name=f"skull3d_{n}", c0=c0, rho=rho, alpha=alpha, dx=dx, omega=2 * math.pi * f_hz,
                   nabs=[[n_abs, n_abs]] * 3, gamma_max=layer_gamma_max(n_abs, dx), source=src,
                   meta=dict(bowl_voxels=int(sub.sum()), r_in=r_in, r_out=r_out))


def smooth_random_medium_torch(shape, seed, c_range=(1400.0, 2800.0), rho_range=(900.0, 1900.0),
                               alpha_db_range=(0.0, 5.0), sigma_frac=1.0 / 16, ppw=6.0, n_abs=16, f_hz=F0,
                               device=None):
    """The smooth_random_medium recipe generated on a torch device (seeded torch generator, torch.fft):
    c0, rho, alpha are float64 device tensors.  Not bit-identical to the numpy version (other generator)."""
    import torch

    dev = torch.device("cuda", 0) if device is None else torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))

    def smooth():
        a = torch.rand(shape, generator=g, device=dev, dtype=torch.float64)
        A = torch.fft.fftn(a)
        for ax, n in enumerate(shape):
            k = torch.fft.fftfreq(n, device=dev, dtype=torch.float64)
            sh = [1] * len(shape)
            sh[ax] = n
            A = A * torch.exp(-2.0 * (math.pi * k * sigma_frac * n) ** 2).reshape(sh)
        b = torch.fft.ifftn(A).real
        lo, hi = b.min(), b.max()
        return (b - lo) / torch.clamp(hi - lo, min=1e-300)

    c0 = (c_range[0] + (c_range[1] - c_range[0]) * smooth()).contiguous()
    rho = (rho_range[0] + (rho_range[1] - rho_range[0]) * smooth()).contiguous()
    alpha = ((alpha_db_range[0] + (alpha_db_range[1] - alpha_db_range[0]) * smooth())
             * db_cm_mhz_to_np_m(1.0, f_hz)).contiguous()
    dx = grid_step(ppw, f_hz)
    return Problem(name=f"random{len(shape)}d_dev", c0=c0, rho=rho, alpha=alpha, dx=dx, omega=2 * math.pi * f_hz,
                   nabs=[[n_abs, n_abs] for _ in shape], gamma_max=layer_gamma_max(n_abs, dx) if n_abs > 0 else 0.0,
                   meta=dict(seed=seed))


def line_source(shape, y_row, amplitude=1.0 + 0j, margin=0):
    """2D planar line source: s_p = amplitude on every cell of row y_row (x in [margin, n0 - margin))."""
    src = np.zeros((3,) + tuple(shape), dtype=np.complex128)
    n0 = shape[1]
    src[2, y_row, margin:n0 - margin] = amplitude
    return src


def disc_perturbation(n=256, radius=32, dc=0.0, drho=0.0, n_abs=16, ppw=6.0, f_hz=F0):
    """Convergence-versus-contrast case: water (1500 m/s, 1000 kg/m^3) with a central disc of c = 1500 + dc,
    rho = 1000 + drho; planar line source near the top (inside the layer's inner edge)."""
    p = inclusion_medium((n, n), radius, C_WATER + dc, RHO_WATER + drho, 0.0, ppw=ppw, n_abs=n_abs, f_hz=f_hz)
    p.source = line_source((n, n), n_abs + 2, margin=n_abs)
    p.name = f"disc_dc{dc:g}_drho{drho:g}"
    return p


def three_discs(n=256, dx=0.5e-3, f_hz=F0, n_abs=16, radius=24):
    """Strongly heterogeneous 2D example (256 x 256, 0.5 mm, 500 kHz): water with three disc inclusions,
    one in sound speed (3500 m/s), one in density (3000 kg/m^3), one in attenuation (10 dB/cm), and a planar
    line source at the top."""
    shape = (n, n)
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    c0 = np.full(shape, C_WATER)
    rho = np.full(shape, RHO_WATER)
    alpha = np.zeros(shape)
    centres = [(n * 0.3, n * 0.45), (n * 0.7, n * 0.45), (n * 0.5, n * 0.72)]
    masks = [(xx - cx) ** 2 + (yy - cy) ** 2 < radius ** 2 for cx, cy in centres]
    c0[masks[0]] = 3500.0
    rho[masks[1]] = 3000.0
    alpha[masks[2]] = 10.0 * NEPER_PER_DB * 100.0  # 10 dB/cm in Np/m
    p = Problem(name="three_discs_256", c0=c0, rho=rho, alpha=alpha, dx=dx, omega=2 * math.pi * f_hz,
                nabs=[[n_abs, n_abs]] * 2, gamma_max=layer_gamma_max(n_abs, dx))
    p.source = line_source(shape, n_abs + 2, margin=n_abs)
    return p
