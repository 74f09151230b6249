"""Pins of the oracle's wide-precision checkers against exact rational arithmetic (-m "not gpu").

Every GPU parity decision on the off-norm, the J-unitarity of V and the factor residual comes
from oracle_check_offdiag, oracle_check_vjv and oracle_check_factor_residual.  These tests feed
them matrices with known NONZERO answers -- small integer (and Gaussian-integer) matrices whose
Gram entries, V^* J V - J and G0 V - G are exact rationals -- and compare with a plain
fractions.Fraction evaluation of the definitions:
  off_F(G^* G) / ||G||_F^2 = sqrt(2 sum_{i<j} |a_ij|^2) / sum_i a_ii,
  max_{i != j} |a_ij| / sqrt(a_ii a_jj)                       (Sec. 2.1: A = G^* G),
  ||V^* J_row V - J_col||_F                                   (Sec. 1: V^* J V = J),
  ||G0 V - G||_F / ||G0||_F                                   (G = G0 V, Sec. 2.3).
Hand-worked closed forms come first; planted mistakes in each checker (mutations 7-12 of the
oracle) must fail at least one of them.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle


# ------------------------------------------------------------------ exact references
def _cols(G):
    """Columns of an integer / Gaussian-integer matrix as lists of (re, im) Fractions."""
    G = np.asarray(G)
    m, n = G.shape
    out = []
    for j in range(n):
        col = []
        for r in range(m):
            z = complex(G[r, j])
            col.append((Fr(int(round(z.real))), Fr(int(round(z.imag)))))
        out.append(col)
    return out


def _dot(x, y):
    """x^* y exactly."""
    re = sum(a * c + b * d for (a, b), (c, d) in zip(x, y))
    im = sum(a * d - b * c for (a, b), (c, d) in zip(x, y))
    return re, im


def exact_offdiag(G):
    cols = _cols(G)
    n = len(cols)
    diag = [_dot(c, c)[0] for c in cols]
    off2 = Fr(0)
    mx = Fr(0)
    for i in range(n):
        for j in range(i + 1, n):
            re, im = _dot(cols[i], cols[j])
            b2 = re * re + im * im
            off2 += 2 * b2
            if diag[i] * diag[j] > 0:
                mx = max(mx, b2 / (diag[i] * diag[j]))
    tr = sum(diag)
    return math.sqrt(off2) / float(tr), math.sqrt(mx)


def exact_vjv(V, Jr, Jc):
    cols = _cols(V)
    n = len(cols)
    acc = Fr(0)
    for i in range(n):
        for j in range(n):
            re = sum(int(Jr[r]) * (a * c + b * d) for r, ((a, b), (c, d)) in enumerate(zip(cols[i], cols[j])))
            im = sum(int(Jr[r]) * (a * d - b * c) for r, ((a, b), (c, d)) in enumerate(zip(cols[i], cols[j])))
            if i == j:
                re -= int(Jc[i])
            acc += re * re + im * im
    return math.sqrt(acc)


def exact_residual(G0, V, G):
    A = _cols(G0)
    B = _cols(V)
    C = _cols(G)
    m, n = len(A[0]), len(A)
    num = Fr(0)
    for c in range(n):
        for r in range(m):
            sr = sum(A[k][r][0] * B[c][k][0] - A[k][r][1] * B[c][k][1] for k in range(n))
            si = sum(A[k][r][0] * B[c][k][1] + A[k][r][1] * B[c][k][0] for k in range(n))
            dr, di = sr - C[c][r][0], si - C[c][r][1]
            num += dr * dr + di * di
    den = sum(a * a + b * b for col in A for (a, b) in col)
    return math.sqrt(num / den)


def close(a, b, rel=1e-14):
    return abs(a - b) <= rel * max(abs(b), 1e-300)


# ------------------------------------------------------------------ pins
def pin_offdiag_closed_form():
    # columns (3,0,0), (0,4,0), (2,0,1): a11 = 9, a22 = 16, a33 = 5, a13 = 6, rest 0
    G = np.array([[3.0, 0, 2], [0, 4, 0], [0, 0, 1]])
    off, mx = oracle.check_offdiag(G)
    return close(off, math.sqrt(72.0) / 30.0) and close(mx, 6.0 / math.sqrt(45.0))


def pin_offdiag_complex_closed_form():
    # g1 = (1, i), g2 = (i, 0): a11 = 2, a22 = 1, a12 = conj(1)*i + conj(i)*0 = i (purely imaginary)
    G = np.array([[1.0, 1j], [1j, 0.0]])
    off, mx = oracle.check_offdiag(G)
    return close(off, math.sqrt(2.0) / 3.0) and close(mx, 1.0 / math.sqrt(2.0))


def pin_offdiag_orthogonal_zero():
    Q = np.array([[1.0, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]]) * np.array([1, 2, 3, 4])
    off, mx = oracle.check_offdiag(Q)
    return off == 0.0 and mx == 0.0


def pin_offdiag_random(seed, cplx):
    g = np.random.default_rng(seed)
    G = g.integers(-5, 6, size=(7, 5)).astype(float)
    if cplx:
        G = G + 1j * g.integers(-5, 6, size=(7, 5))
    off, mx = oracle.check_offdiag(G)
    eo, em = exact_offdiag(G)
    return close(off, eo) and close(mx, em)


def pin_vjv_closed_form():
    # shear V = [[1, 1], [0, 1]], J = diag(1, -1): V^T J V - J = [[0, 1], [1, 1]], norm sqrt(3)
    V = np.array([[1.0, 1.0], [0.0, 1.0]])
    J = np.array([1, -1], dtype=np.int8)
    return close(oracle.check_vjv(V, J), math.sqrt(3.0))


def pin_vjv_row_col_signs():
    # V = swap, J_row = diag(1, -1), J_col = diag(-1, 1): V^T J_row V = J_col exactly
    V = np.array([[0.0, 1.0], [1.0, 0.0]])
    Jr = np.array([1, -1], dtype=np.int8)
    Jc = np.array([-1, 1], dtype=np.int8)
    return oracle.check_vjv(V, Jr, Jc) == 0.0 and close(oracle.check_vjv(V, Jr, Jr), math.sqrt(8.0))


def pin_vjv_random(seed, cplx):
    g = np.random.default_rng(seed)
    n = 5
    V = g.integers(-3, 4, size=(n, n)).astype(float)
    if cplx:
        V = V + 1j * g.integers(-3, 4, size=(n, n))
    Jr = np.where(g.random(n) < 0.5, -1, 1).astype(np.int8)
    Jc = np.where(g.random(n) < 0.5, -1, 1).astype(np.int8)
    return close(oracle.check_vjv(V, Jr, Jc), exact_vjv(V, Jr, Jc))


def pin_residual_closed_form():
    # G0 = [[1, 2], [3, 4]], V = [[1, 2], [0, 1]]: G0 V = [[1, 4], [3, 10]]; G differs by 1 in one
    # entry, ||G0||_F^2 = 30
    G0 = np.array([[1.0, 2.0], [3.0, 4.0]])
    V = np.array([[1.0, 2.0], [0.0, 1.0]])
    G = np.array([[1.0, 4.0], [3.0, 9.0]])
    return close(oracle.check_factor_residual(G0, V, G), 1.0 / math.sqrt(30.0))


def pin_residual_random(seed, cplx):
    g = np.random.default_rng(seed)
    m, n = 6, 4
    G0 = g.integers(-4, 5, size=(m, n)).astype(float)
    V = g.integers(-3, 4, size=(n, n)).astype(float)
    E = g.integers(-2, 3, size=(m, n)).astype(float)
    if cplx:
        G0 = G0 + 1j * g.integers(-4, 5, size=(m, n))
        V = V + 1j * g.integers(-3, 4, size=(n, n))
        E = E + 1j * g.integers(-2, 3, size=(m, n))
    G = G0 @ V + E  # exact in double (small integers)
    return close(oracle.check_factor_residual(G0, V, G), exact_residual(G0, V, G))


CHECKER_PINS = {
    "offdiag_closed_form": pin_offdiag_closed_form,
    "offdiag_complex_closed_form": pin_offdiag_complex_closed_form,
    "offdiag_orthogonal_zero": pin_offdiag_orthogonal_zero,
    "offdiag_random_real": lambda: all(pin_offdiag_random(s, False) for s in (1, 2, 3)),
    "offdiag_random_complex": lambda: all(pin_offdiag_random(s, True) for s in (4, 5, 6)),
    "vjv_closed_form": pin_vjv_closed_form,
    "vjv_row_col_signs": pin_vjv_row_col_signs,
    "vjv_random_real": lambda: all(pin_vjv_random(s, False) for s in (7, 8, 9)),
    "vjv_random_complex": lambda: all(pin_vjv_random(s, True) for s in (10, 11, 12)),
    "residual_closed_form": pin_residual_closed_form,
    "residual_random_real": lambda: all(pin_residual_random(s, False) for s in (13, 14)),
    "residual_random_complex": lambda: all(pin_residual_random(s, True) for s in (15, 16)),
}


@pytest.mark.parametrize("name", sorted(CHECKER_PINS))
def test_checker_pin(name):
    oracle.set_mutation(0)
    assert CHECKER_PINS[name](), name


def test_exact_references_are_independent():
    """The Fraction references themselves on the hand-worked cases (no oracle call)."""
    o, m = exact_offdiag(np.array([[3.0, 0, 2], [0, 4, 0], [0, 0, 1]]))
    assert close(o, math.sqrt(72.0) / 30.0) and close(m, 6.0 / math.sqrt(45.0))
    assert close(exact_vjv(np.array([[1.0, 1.0], [0.0, 1.0]]), [1, -1], [1, -1]), math.sqrt(3.0))
    assert close(exact_residual(np.array([[1.0, 2.0], [3.0, 4.0]]), np.array([[1.0, 2.0], [0.0, 1.0]]),
                                np.array([[1.0, 4.0], [3.0, 9.0]])), 1.0 / math.sqrt(30.0))


@pytest.mark.parametrize("mutation", [7, 8, 9, 10, 11, 12])
def test_checker_mutations_are_caught(mutation):
    """Plant mistake k in a checker: at least one checker pin must fail."""
    try:
        oracle.set_mutation(mutation)
        failed = [name for name, f in CHECKER_PINS.items() if not f()]
    finally:
        oracle.set_mutation(0)
    assert failed, "mutation %d not caught by any checker pin" % mutation
