"""Pin for the adjoint-state misfit gradient (oracle/gradient.py): central finite
differences of J computed with dense LAPACK solves of the plain system."""
import numpy as np
import pytest

from oracle import dense, gradient
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W


def _setup(shape=(10, 12), seed=5):
    p = W.smooth_random_medium(shape, seed=seed, n_abs=2)
    p.gamma_max = 0.5 * p.omega
    rng = np.random.default_rng(seed + 1)
    S = 2
    src = np.zeros((S, len(shape) + 1) + shape, dtype=np.complex128)
    src[0, -1, 3, 4] = 1.0
    src[1, -1, 7, 8] = 1.0 - 0.5j
    src[1, 0] = 0.1 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    rec = (np.array([2, 5, 8, 8]), np.array([2, 9, 3, 10]))
    data = rng.standard_normal((S, 4)) + 1j * rng.standard_normal((S, 4))
    return p, src, rec, data


def _J(p, c0, rho, src, rec, data):
    f = np.stack([dense.solve(s, c0, rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power) for s in src])
    return gradient.receiver_misfit(f, data, rec)


@pytest.mark.parametrize("which", ["c0", "rho"])
def test_gradient_matches_central_differences_dense(which):
    p, src, rec, data = _setup()
    J, g = _J(p, p.c0, p.rho, src, rec, data)
    fields = np.stack([dense.solve(s, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power) for s in src])
    adj = np.stack([dense.solve_adjoint(gs, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
                    for gs in g])
    gc, gr = gradient.medium_gradient(p.c0, p.rho, p.alpha, p.omega, p.nabs, p.gamma_max, src, fields, adj)
    grad = gc if which == "c0" else gr
    rng = np.random.default_rng(9)
    for _ in range(6):
        iy, ix = rng.integers(0, p.shape[0]), rng.integers(0, p.shape[1])
        m = (p.c0 if which == "c0" else p.rho).copy()
        h = 1e-6 * m[iy, ix]
        mp, mm = m.copy(), m.copy()
        mp[iy, ix] += h
        mm[iy, ix] -= h
        if which == "c0":
            Jp, _ = _J(p, mp, p.rho, src, rec, data)
            Jm, _ = _J(p, mm, p.rho, src, rec, data)
        else:
            Jp, _ = _J(p, p.c0, mp, src, rec, data)
            Jm, _ = _J(p, p.c0, mm, src, rec, data)
        fd = (Jp - Jm) / (2 * h)
        assert abs(grad[iy, ix] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (which, iy, ix, grad[iy, ix], fd)


def test_gradient_with_born_solves_equals_dense_version():
    p, src, rec, data = _setup()
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    fields = np.stack([P.solve_field(s, 1e-12, check_every=25)[0] for s in src])
    J, g = gradient.receiver_misfit(fields, data, rec)
    adj = np.stack([P.unscale(P.solve(P.scale_source(gs, adjoint=True), 1e-12, check_every=25, adjoint=True)[0])
                    for gs in g])
    gc, gr = gradient.medium_gradient(p.c0, p.rho, p.alpha, p.omega, p.nabs, p.gamma_max, src, fields, adj)
    fd_ = np.stack([dense.solve(s, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power) for s in src])
    _, gd = gradient.receiver_misfit(fd_, data, rec)
    ad_ = np.stack([dense.solve_adjoint(x, p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
                    for x in gd])
    gc2, gr2 = gradient.medium_gradient(p.c0, p.rho, p.alpha, p.omega, p.nabs, p.gamma_max, src, fd_, ad_)
    assert np.linalg.norm(gc - gc2) <= 1e-9 * np.linalg.norm(gc2)
    assert np.linalg.norm(gr - gr2) <= 1e-9 * np.linalg.norm(gr2)
