"""Plain definition of the discrete system, assembled densely (tiny grids only).

TEST INFRASTRUCTURE.  The Born iteration converges to the solution of one
linear system: the row-scaled first-order system on the staggered grid
(eq. HH1stOrderSH with App. B.1's staggering).  Written out, with
``N = prod(n)`` unknowns per component:

    [ diag(d_eta)      S+ d_eta   ] [ u ]   [ (S+ rho) s_u      ]
    [ d_eta S-         diag(q)    ] [ p ] = [ s_p / (rho c^2)   ]

    d_eta = (S+ rho)_eta (S+ gamma_eta + i omega)     (App. B.1)
    q     = (i omega + gamma) / (rho c^2)               (eq. HH1stOrderSH)
    c^2   = c0^2 / (1 - 2 i alpha c0 / omega)           (eq. 118)
    (S+ rho)_eta = (rho(x) + rho(x + dx e_eta)) / 2     (App. B.1)
    S+ d_eta = F^H diag(i k_eta e^{+i k_eta dx/2}) F,  d_eta S- = F^H diag(i k_eta e^{-i k_eta dx/2}) F
                                                        (shift theorem, App. B.1)

The DFT matrices here are built explicitly from exp(-2 pi i jk/n), not through
any FFT, and the whole set-up is retyped from the paper in numpy, so this
module shares no arithmetic with ``cbs_oracle.c``.  The solution does not
depend on the shifts, the scaling C or nu, which is what makes it a pin for
the iteration.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int) -> np.ndarray:
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def wavenumbers(n: int, dx: float) -> np.ndarray:
    f = np.array([j if j < (n + 1) // 2 else j - n for j in range(n)], dtype=np.float64)
    return 2 * np.pi * f / (n * dx)


def layer_profile(n: int, lo: int, hi: int, gamma_max: float, power: float, offset: float) -> np.ndarray:
    """gamma contribution of one axis at cell coordinates j + offset (quadratic layer inside the grid)."""
    xi = np.arange(n) + offset
    d = np.zeros(n)
    if lo > 0:
        d = np.maximum(d, (lo - xi) / lo)
    if hi > 0:
        d = np.maximum(d, (xi - (n - 1 - hi)) / hi)
    d = np.clip(d, 0.0, 1.0)
    return gamma_max * d ** power


def axis_operator(shape, axis_xyz: int, one_d: np.ndarray) -> np.ndarray:
    """Kronecker embedding of a 1-D operator acting along axis x/y/z (numpy C order)."""
    D = len(shape)
    np_axis = D - 1 - axis_xyz
    M = np.ones((1, 1))
    for ax in range(D):
        M = np.kron(M, one_d if ax == np_axis else np.eye(shape[ax]))
    return M


def diagonals(c0, rho, alpha, dx, omega, nabs, gamma_max, power=2.0, collocated=False):
    """d_eta (D arrays) and q at every voxel, from the formulas in the module docstring (collocated grid of
    App. B: velocity at the cell centres, so rho and gamma are not shifted)."""
    shape = c0.shape
    D = len(shape)
    c2 = c0 ** 2 / (1 - 2j * alpha * c0 / omega)
    per_axis_c = []
    per_axis_s = []
    for a in range(D):
        n = shape[D - 1 - a]
        lo, hi = nabs[a]
        sh = [1] * D
        sh[D - 1 - a] = n
        per_axis_c.append(layer_profile(n, lo, hi, gamma_max, power, 0.0).reshape(sh))
        per_axis_s.append(layer_profile(n, lo, hi, gamma_max, power, 0.0 if collocated else 0.5).reshape(sh))
    gamma = sum(np.broadcast_to(g, shape) for g in per_axis_c)
    q = (1j * omega + gamma) / (rho * c2)
    d = []
    rho_s = []
    for eta in range(D):
        g_s = sum(np.broadcast_to(per_axis_s[a] if a == eta else per_axis_c[a], shape) for a in range(D))
        r_s = rho if collocated else 0.5 * (rho + np.roll(rho, -1, axis=D - 1 - eta))
        rho_s.append(r_s)
        d.append(r_s * (g_s + 1j * omega))
    return d, q, rho_s, c2


def assemble(c0, rho, alpha, dx, omega, nabs, gamma_max, power=2.0, adjoint=False, collocated=False):
    """Dense row-scaled operator A (C*N x C*N).  adjoint=True gives A^H.  collocated: derivative symbol i k
    (App. B) instead of the staggered i k e^{+-i k dx/2}."""
    shape = c0.shape
    D = len(shape)
    N = int(np.prod(shape))
    d, q, _, _ = diagonals(c0, rho, alpha, dx, omega, nabs, gamma_max, power, collocated)
    A = np.zeros(((D + 1) * N, (D + 1) * N), dtype=np.complex128)
    for eta in range(D):
        n = shape[D - 1 - eta]
        F = dft_matrix(n)
        Fi = np.conj(F).T / n
        k = wavenumbers(n, dx)
        sh = 0.0 if collocated else dx / 2
        dplus = Fi @ np.diag(1j * k * np.exp(1j * k * sh)) @ F
        dminus = Fi @ np.diag(1j * k * np.exp(-1j * k * sh)) @ F
        A[eta * N:(eta + 1) * N, eta * N:(eta + 1) * N] = np.diag(d[eta].ravel())
        A[eta * N:(eta + 1) * N, D * N:] = axis_operator(shape, eta, dplus)
        A[D * N:, eta * N:(eta + 1) * N] = axis_operator(shape, eta, dminus)
    A[D * N:, D * N:] = np.diag(q.ravel())
    return np.conj(A).T if adjoint else A


def scaled_rhs(src, c0, rho, alpha, dx, omega, nabs, gamma_max, power=2.0, collocated=False):
    """Row-scaled right-hand side ((S+ rho) s_u, s_p / (rho c^2))."""
    D = c0.ndim
    _, _, rho_s, c2 = diagonals(c0, rho, alpha, dx, omega, nabs, gamma_max, power, collocated)
    out = np.empty_like(np.asarray(src, dtype=np.complex128))
    for eta in range(D):
        out[eta] = rho_s[eta] * src[eta]
    out[D] = src[D] / (rho * c2)
    return out


def solve(src, c0, rho, alpha, dx, omega, nabs, gamma_max, power=2.0, collocated=False):
    """Physical (u, p) from physical (s_u, s_p) by LAPACK on the dense system."""
    A = assemble(c0, rho, alpha, dx, omega, nabs, gamma_max, power, collocated=collocated)
    b = scaled_rhs(src, c0, rho, alpha, dx, omega, nabs, gamma_max, power, collocated).ravel()
    return np.linalg.solve(A, b).reshape(np.shape(src))


def solve_adjoint(g, c0, rho, alpha, dx, omega, nabs, gamma_max, power=2.0):
    """lambda with A^H lambda = g (g taken as given: the adjoint right-hand side)."""
    A = assemble(c0, rho, alpha, dx, omega, nabs, gamma_max, power, adjoint=True)
    return np.linalg.solve(A, np.asarray(g, dtype=np.complex128).ravel()).reshape(np.shape(g))


def second_order_pressure(src_p, c0, alpha, dx, omega):
    """Constant density, no layer: (lap + omega^2/c^2) p = -i omega s_p / c^2 (App. A), with the spectral
    Laplacian -|k|^2 (the product of the two staggered derivative symbols)."""
    shape = c0.shape
    D = len(shape)
    N = int(np.prod(shape))
    c2 = c0 ** 2 / (1 - 2j * alpha * c0 / omega)
    lap = np.zeros((N, N), dtype=np.complex128)
    for eta in range(D):
        n = shape[D - 1 - eta]
        F = dft_matrix(n)
        Fi = np.conj(F).T / n
        k = wavenumbers(n, dx)
        lap += axis_operator(shape, eta, Fi @ np.diag(-(k ** 2)) @ F)
    H = lap + np.diag((omega ** 2 / c2).ravel())
    b = (-1j * omega * src_p / c2).ravel()
    return np.linalg.solve(H, b).reshape(shape)


def uniform_solve(src, c0: float, rho: float, alpha: float, dx: float, omega: float):
    """Uniform medium, no absorbing layer: the staggered system has constant coefficients, so the DFT
    diagonalises it and each wavenumber is an independent (D+1)x(D+1) solve
        [[ d I , i k S ], [ i k^T S^, q ]] (u^, p^) = (rho s_u^, s_p^ / (rho c^2))
    with d = i omega rho, q = i omega / (rho c^2), S_eta = e^{i k_eta dx/2} (App. B.1).  Uses numpy.fft as
    a library step; valid at any grid size."""
    src = np.asarray(src, dtype=np.complex128)
    D = src.ndim - 1
    shape = src.shape[1:]
    c2 = c0 ** 2 / (1 - 2j * alpha * c0 / omega)
    d = 1j * omega * rho
    q = 1j * omega / (rho * c2)
    rhs = np.empty_like(src)
    rhs[:D] = rho * src[:D]
    rhs[D] = src[D] / (rho * c2)
    R = np.stack([np.fft.fftn(rhs[c]) for c in range(D + 1)], axis=-1)  # (*shape, C)
    ks = np.meshgrid(*[wavenumbers(shape[D - 1 - a], dx) for a in range(D)][::-1], indexing="ij")[::-1]
    M = np.zeros(shape + (D + 1, D + 1), dtype=np.complex128)
    for e in range(D):
        M[..., e, e] = d
        M[..., e, D] = 1j * ks[e] * np.exp(1j * ks[e] * dx / 2)
        M[..., D, e] = 1j * ks[e] * np.exp(-1j * ks[e] * dx / 2)
    M[..., D, D] = q
    X = np.linalg.solve(M, R[..., None])[..., 0]
    return np.stack([np.fft.ifftn(X[..., c]) for c in range(D + 1)], axis=0)
