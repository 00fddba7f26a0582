"""Pins for the oracle's operators.

* The (L+I)^-1 symbol (typed from App. B.1's matrix) inverts L + I, with L
  typed separately from eq. LV and the shift-theorem derivative symbols.
* L + V matches the plain definition assembled densely with explicit DFT
  matrices (C^-1/2 A C^-1/2 with the oracle's own scaling).
* The adjoint operators are the Hermitian transposes (dot-product tests).
"""
import numpy as np
import pytest

from oracle import dense
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W


def _problem(shape, seed, n_abs=2, gamma_scale=0.5):
    p = W.smooth_random_medium(shape, seed=seed, n_abs=n_abs)
    p.gamma_max = gamma_scale * p.omega
    return p


def _oracle(p, **kw):
    return O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power, **kw)


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape", [(16, 16), (9, 12), (15, 8), (8, 8, 8), (6, 5, 4)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_green_inverts_L_plus_I(shape, adjoint):
    p = _problem(shape, seed=len(shape) * 7 + shape[0])
    P = _oracle(p)
    x = _rand(P.field_shape, 3)
    v = P.v()
    Lx = P.apply(x, adjoint) - (np.conj(v) if adjoint else v) * x   # L x alone
    back = P.green(Lx + x, adjoint)                                # (L+I)^-1 (L+I) x
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x)) * 10


@pytest.mark.parametrize("shape", [(8, 6), (6, 4, 4)])
def test_apply_matches_dense_plain_definition(shape):
    p = _problem(shape, seed=11)
    P = _oracle(p)
    sc = P.scalars()
    A = dense.assemble(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power)
    D = len(shape)
    N = int(np.prod(shape))
    cinv = np.concatenate([np.full(D * N, sc["lambda1"] ** -0.5), np.full(N, sc["lambda2"] ** -0.5)])
    As = cinv[:, None] * A * cinv[None, :]
    x = _rand(P.field_shape, 5)
    ref = (As @ x.ravel()).reshape(x.shape)
    got = P.apply(x)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # the adjoint apply is the Hermitian transpose of the same matrix
    ref_h = (np.conj(As).T @ x.ravel()).reshape(x.shape)
    assert np.linalg.norm(P.apply(x, adjoint=True) - ref_h) <= 1e-13 * np.linalg.norm(ref_h)


@pytest.mark.parametrize("shape", [(16, 12), (8, 8, 6)])
def test_adjoint_dot_products(shape):
    p = _problem(shape, seed=21)
    P = _oracle(p)
    a = _rand(P.field_shape, 1)
    b = _rand(P.field_shape, 2)
    # <G a, b> = <a, G^H b> and <A a, b> = <a, A^H b>
    lhs = np.vdot(b, P.green(a))
    rhs = np.vdot(P.green(b, adjoint=True), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = np.vdot(b, P.apply(a))
    rhs = np.vdot(P.apply(b, adjoint=True), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_green_uniform_symbol_diagonal_in_k():
    """(L+I)^-1 is translation invariant: it commutes with a circular shift of every component."""
    p = _problem((12, 16), seed=2)
    P = _oracle(p)
    x = _rand(P.field_shape, 9)
    g1 = np.roll(P.green(x), (3, 5), axis=(1, 2))
    g2 = P.green(np.roll(x, (3, 5), axis=(1, 2)))
    assert np.max(np.abs(g1 - g2)) <= 1e-13 * np.max(np.abs(g1)) * 10


@pytest.mark.parametrize("shape", [(12, 10), (6, 8, 6)])
def test_collocated_adjoint_operators_are_hermitian_transposes(shape):
    """App. B's collocated grid: the adjoint (L+I)^-1 and A_s are the Hermitian transposes of the forward ones
    (dot products), and the adjoint apply equals the conjugate transpose of the densely assembled matrix."""
    p = _problem(shape, seed=52)
    P = _oracle(p, collocated=True)
    a = _rand(P.field_shape, 53)
    b = _rand(P.field_shape, 54)
    lhs = np.vdot(b, P.green(a))
    rhs = np.vdot(P.green(b, adjoint=True), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = np.vdot(b, P.apply(a))
    rhs = np.vdot(P.apply(b, adjoint=True), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    sc = P.scalars()
    A = dense.assemble(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, p.power, collocated=True)
    D = len(shape)
    N = int(np.prod(shape))
    cinv = np.concatenate([np.full(D * N, sc["lambda1"] ** -0.5), np.full(N, sc["lambda2"] ** -0.5)])
    As = cinv[:, None] * A * cinv[None, :]
    ref_h = (np.conj(As).T @ a.ravel()).reshape(a.shape)
    assert np.linalg.norm(P.apply(a, adjoint=True) - ref_h) <= 1e-13 * np.linalg.norm(ref_h)
