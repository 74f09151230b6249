"""Pins of the oracle's eigendecomposition adjoint (the reference gradient of the
differentiation workload) against facts independent of its own formula:

  * Hellmann-Feynman: with U_bar = 0, <H_bar, E> = sum_i lambda_bar_i u_i^T E u_i for every
    symmetric direction E (eigenvalue derivatives of a simple spectrum);
  * diagonal H: with U_bar = 0 the adjoint is diag(lambda_bar) placed on the diagonal positions
    of the sorted eigenvalues;
  * central finite differences of a loss that uses eigenvectors (sign-invariant), with the
    forward map computed by LAPACK (numpy.linalg.eigh, test-only), in FP64;
  * a mutation of the oracle (transposed U^T U_bar) fails the finite-difference pin.
"""
import numpy as np
import pytest

import oracle


def _sym(n, g):
    A = g.standard_normal((n, n))
    return (A + A.T) / 2


def _loss_parts(n, g, k):
    w = g.standard_normal(n)
    C = g.standard_normal((n, 2))
    return w, C, k


def _loss(H, w, C, k):
    lam, U = np.linalg.eigh(H)
    return float(w @ lam + np.sum((U[:, :k].T @ C) ** 2))


def _grads(H, w, C, k):
    lam, U = np.linalg.eigh(H)
    lam_bar = w.copy()
    U_bar = np.zeros_like(U)
    U_bar[:, :k] = 2.0 * C @ (C.T @ U[:, :k])
    return lam, U, lam_bar, U_bar


@pytest.mark.parametrize("n", [3, 6, 11])
def test_backward_hellmann_feynman(n):
    g = np.random.default_rng(500 + n)
    H = _sym(n, g)
    lam, U = np.linalg.eigh(H)
    lam_bar = g.standard_normal(n)
    Hb = oracle.eig_backward(lam, U, lam_bar, None)
    assert np.allclose(Hb, Hb.T, rtol=0, atol=0)
    for _ in range(4):
        E = _sym(n, g)
        want = sum(lam_bar[i] * U[:, i] @ E @ U[:, i] for i in range(n))
        got = np.sum(Hb * E)
        assert abs(got - want) <= 1e-13 * (1 + abs(want))


def test_backward_diagonal_closed_form():
    d = np.array([3.0, -1.0, 7.5, 0.25, -4.0])
    H = np.diag(d)
    order = np.argsort(d)
    lam = d[order]
    U = np.eye(5)[:, order]
    lam_bar = np.array([0.5, -2.0, 1.0, 3.0, -0.75])
    Hb = oracle.eig_backward(lam, U, lam_bar, None)
    want = np.zeros((5, 5))
    for i, p in enumerate(order):
        want[p, p] = lam_bar[i]
    assert np.array_equal(Hb, want)


@pytest.mark.parametrize("n,k", [(4, 1), (8, 2), (12, 3)])
def test_backward_finite_differences(n, k):
    g = np.random.default_rng(700 + n)
    H = _sym(n, g)
    w, C, _ = _loss_parts(n, g, k)
    lam, U, lam_bar, U_bar = _grads(H, w, C, k)
    Hb = oracle.eig_backward(lam, U, lam_bar, U_bar)
    h = 1e-6
    for _ in range(5):
        E = _sym(n, g)
        E /= np.linalg.norm(E)
        fd = (_loss(H + h * E, w, C, k) - _loss(H - h * E, w, C, k)) / (2 * h)
        got = np.sum(Hb * E)
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (got, fd)


def test_backward_mutation_detected():
    """Planting a transposed product in the oracle makes the finite-difference pin fail."""
    n, k = 8, 2
    g = np.random.default_rng(708)
    H = _sym(n, g)
    w, C, _ = _loss_parts(n, g, k)
    lam, U, lam_bar, U_bar = _grads(H, w, C, k)
    oracle.set_mutation(6)
    try:
        Hb = oracle.eig_backward(lam, U, lam_bar, U_bar)
    finally:
        oracle.set_mutation(0)
    E = _sym(n, g)
    E /= np.linalg.norm(E)
    h = 1e-6
    fd = (_loss(H + h * E, w, C, k) - _loss(H - h * E, w, C, k)) / (2 * h)
    assert abs(np.sum(Hb * E) - fd) > 1e-4 * max(1.0, abs(fd))
