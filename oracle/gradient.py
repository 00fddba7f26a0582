"""Adjoint-state gradient of a field misfit with respect to sound speed and
density (FP64, numpy) -- the oracle for the GPU gradient.

TEST INFRASTRUCTURE.

The solved system is the row-scaled staggered system A(m) X = b(m) of the
paper (eq. HH1stOrderSH with App. B.1), with A = L0 + diag(d_eta, q):
    d_eta = (S+ rho)_eta (S+ gamma_eta + i omega),  (S+ rho)_eta(x) = (rho(x) + rho(x + e_eta)) / 2
    q     = (i omega + gamma) / (rho c^2),          c^2 = c0^2 / (1 - 2 i alpha c0 / omega)   (eq. 118)
    b     = ((S+ rho) s_u, s_p / (rho c^2))
For a real misfit J(X) with dJ = Re<g, dX>, the adjoint field lambda solves
A^H lambda = g (Sec. 2.3 notes A^H is accretive, so the same iteration applies)
and dJ/dm = Re <lambda, db/dm - (dA/dm) X>, pointwise in m because A's
m-dependence is diagonal:
    dq/dc0   = (i omega + gamma) (-2/c0^3 + 2 i alpha / (omega c0^2)) / rho,  db_p/dc0 = s_p (same factor) / rho
    dq/drho  = -q / rho,                                                     db_p/drho = -b_p / rho
    d d_eta(x')/drho(x) = (S+ gamma_eta(x') + i omega)/2 for x' = x and x' = x - e_eta,
    d b_eta(x')/drho(x) = s_u,eta(x') / 2 for the same x'.
"""
from __future__ import annotations

import numpy as np

from . import dense


def layer_fields(shape, nabs, gamma_max, power=2.0):
    """gamma at the cell centres and at each staggered point (same profile as the solver)."""
    D = len(shape)
    cen, stag = [], []
    for a in range(D):
        n = shape[D - 1 - a]
        sh = [1] * D
        sh[D - 1 - a] = n
        cen.append(dense.layer_profile(n, nabs[a][0], nabs[a][1], gamma_max, power, 0.0).reshape(sh))
        stag.append(dense.layer_profile(n, nabs[a][0], nabs[a][1], gamma_max, power, 0.5).reshape(sh))
    g = sum(np.broadcast_to(x, shape) for x in cen)
    gs = [sum(np.broadcast_to(stag[a] if a == e else cen[a], shape) for a in range(D)) for e in range(D)]
    return g, gs


def medium_gradient(c0, rho, alpha, omega, nabs, gamma_max, src, field, adj, power=2.0):
    """Re <lambda, db/dm - dA/dm X> for m = c0 and m = rho, summed over sources.
    src, field, adj: (S, D+1, *shape) physical source, forward field and adjoint field."""
    shape = c0.shape
    D = len(shape)
    g, gs = layer_fields(shape, nabs, gamma_max, power)
    fac = -2.0 / c0 ** 3 + 2j * alpha / (omega * c0 ** 2)
    c2 = c0 ** 2 / (1 - 2j * alpha * c0 / omega)
    q = (1j * omega + g) / (rho * c2)
    grad_c = np.zeros(shape)
    grad_r = np.zeros(shape)
    for s in range(src.shape[0]):
        sp, p, lp = src[s, D], field[s, D], adj[s, D]
        grad_c += np.real(np.conj(lp) * (sp * fac / rho - (1j * omega + g) * fac / rho * p))
        bp = sp / (rho * c2)
        grad_r += np.real(np.conj(lp) * (-bp / rho + q / rho * p))
        for e in range(D):
            ax = D - 1 - e
            term = np.conj(adj[s, e]) * 0.5 * (src[s, e] - (gs[e] + 1j * omega) * field[s, e])
            grad_r += np.real(term + np.roll(term, 1, axis=ax))
    return grad_c, grad_r


def receiver_misfit(fields, data, rec_idx):
    """J = 1/2 sum_s sum_r |p_s(x_r) - d_s(r)|^2 and its adjoint source g (dJ = Re<g, dX>).
    rec_idx: tuple of index arrays into one component's grid."""
    D = fields.shape[1] - 1
    r = fields[:, D][(slice(None),) + tuple(rec_idx)] - data
    J = 0.5 * float(np.sum(np.abs(r) ** 2))
    g = np.zeros_like(fields)
    g[(slice(None), D) + tuple(rec_idx)] = r
    return J, g
