"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each pin is independent of the oracle's own formulas: Example 1 of Sec. 3.1 (printed values),
closed-form 2x2 eigenvalues, rotation angles from library atan/atanh, exact characteristic
polynomial roots (rational arithmetic), prescribed spectra Q diag(sigma) W, LAPACK SVD for
J = I, and the invariants V^T J V = J, G0 V = G, G^T G diagonal.  The mutation tests plant a
mistake in the oracle and check that some pin fails.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact_charpoly import eigenvalues_exact

EPS = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_example1():
    sec = {}
    cur = None
    s, t = np.sqrt(3.0) / np.sqrt(2.0), 1.0 / np.sqrt(2.0)
    with open(os.path.join(GOLDEN, "example1.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                sec[cur] = []
                continue
            vals = [s if v == "s" else (-s if v == "-s" else (t if v == "t" else (-t if v == "-t" else float(v))))
                    for v in line.split()]
            sec[cur].append(vals)
    return (np.array(sec["H"]), np.array(sec["R"]), np.array(sec["J"][0], dtype=np.int8),
            np.array(sec["eigenvalues"][0]))


# ------------------------------------------------------------------ individual pins (bool)

def pin_example1():
    H, R, J, ev = load_example1()
    G = R.T.copy()
    ok = np.allclose(G @ np.diag(J.astype(float)) @ G.T, H, atol=4 * EPS)
    r = oracle.solve(G, J)
    ok &= r["status"] == 0
    ok &= bool(np.allclose(r["lam"], ev, rtol=0, atol=16 * EPS))
    # eigenvectors: lambda = 3 -> (1,1,1,1)/2, lambda = -1 -> (1,1,-1,-1)/2; lambda = 1 double:
    # compare the projector on the eigenspace (the vectors inside it are not unique)
    U = r["U"]
    v3 = np.ones(4) / 2
    vm = np.array([1, 1, -1, -1]) / 2
    ok &= abs(abs(U[:, 3] @ v3) - 1) < 1e-14 and abs(abs(U[:, 0] @ vm) - 1) < 1e-14
    P1 = np.eye(4) - np.outer(v3, v3) - np.outer(vm, vm)
    U1 = U[:, 1:3]
    ok &= np.linalg.norm(U1 @ U1.T - P1) < 1e-14
    return bool(ok)


def pin_two_column(hyperbolic, seed, cplx=False):
    """One rotation on an m x 2 factor: the two nonzero eigenvalues of H = G J_P G^* in closed form."""
    g = np.random.default_rng(seed)
    G = g.standard_normal((7, 2))
    if cplx:
        G = G + 1j * g.standard_normal((7, 2))
    J = np.array([1, -1] if hyperbolic else [1, 1], dtype=np.int8)
    a = np.vdot(G[:, 0], G[:, 0]).real
    d = np.vdot(G[:, 1], G[:, 1]).real
    b = abs(np.vdot(G[:, 0], G[:, 1]))
    if not hyperbolic:
        disc = np.sqrt((a - d) ** 2 + 4 * b * b)
        ev = np.sort([(a + d - disc) / 2, (a + d + disc) / 2])
    else:
        # nonzero eigenvalues of g1 g1^* - g2 g2^*: those of [[a, b], [-conj b, -d]]
        disc = np.sqrt((a + d) ** 2 - 4 * b * b)
        ev = np.sort([(a - d - disc) / 2, (a - d + disc) / 2])
    r = oracle.solve(G, J)
    return bool(r["status"] == 0 and np.allclose(r["lam"], ev, rtol=64 * EPS, atol=0))


def pin_rotation_angles(seed):
    """t = tan(phi) / tanh(phi) against the angle from library atan / atanh."""
    g = np.random.default_rng(seed)
    ok = True
    for _ in range(200):
        a, d = g.uniform(0.1, 10.0, 2)
        b = g.uniform(0.01, 0.99) * np.sqrt(a * d)
        _, _, t = oracle.rotation_params(a, d, b, 0)
        # cot 2phi = (d - a)/(2b), |phi| <= pi/4
        phi = 0.5 * np.arctan2(2 * b, d - a) if d != a else np.pi / 4
        if phi > np.pi / 4:
            phi -= np.pi / 2
        ok &= abs(t - np.tan(phi)) <= 8 * EPS * max(1.0, abs(t))
        _, _, th = oracle.rotation_params(a, d, b, 1)
        # coth 2phi = -(a + d)/(2b)
        ok &= abs(th - np.tanh(0.5 * np.arctanh(-2 * b / (a + d)))) <= 64 * EPS
    # special cases: equal diagonals give tan(phi) = 1; the hyperbolic guard caps |tanh| at 0.9
    _, _, t = oracle.rotation_params(2.0, 2.0, 1.0, 0)
    ok &= t == 1.0
    _, _, th = oracle.rotation_params(1.0, 1.0, 1.0, 1)
    ok &= abs(th) == 0.9
    return bool(ok)


def pin_charpoly(seed, n, hyperbolic, m_extra=0):
    g = np.random.default_rng(seed)
    G = g.standard_normal((n + m_extra, n))
    J = np.ones(n, dtype=np.int8)
    if hyperbolic:
        J[n // 2:] = -1
    Gf = [[Fraction(float(v)) for v in row] for row in G]
    H = [[sum(Gf[i][k] * J[k] * Gf[j][k] for k in range(n)) for j in range(n + m_extra)] for i in range(n + m_extra)]
    ev = [float(x) for x in eigenvalues_exact(H)]
    # H (m x m) has m - n zero eigenvalues beyond the n of the factor
    ev = sorted(ev, key=abs)[m_extra:] if m_extra else ev
    ev = np.sort(ev)
    r = oracle.solve(G, J)
    B = G / np.linalg.norm(G, axis=0)
    kap = np.linalg.cond(B) ** 2
    return bool(r["status"] == 0 and np.all(np.abs(r["lam"] - ev) <= 50 * n * EPS * kap * np.abs(ev)))


def prescribed(n, npos, seed):
    """G = Q diag(sigma) W in long double: Q orthogonal, W J-orthogonal; eig(G J G^T) = j sigma^2."""
    g = np.random.default_rng(seed)
    L = np.longdouble
    Q, Rq = np.linalg.qr(g.standard_normal((n, n)))
    Q = Q * np.sign(np.diag(Rq))
    Q = Q.astype(L)
    # re-orthogonalize Q in long double (one Gram-Schmidt pass)
    for c in range(n):
        v = Q[:, c].copy()
        for k in range(c):
            v -= (Q[:, k] @ v) * Q[:, k]
        Q[:, c] = v / np.sqrt(v @ v)
    J = np.array([1] * npos + [-1] * (n - npos), dtype=np.int8)
    W = np.eye(n, dtype=L)
    for _ in range(3 * n):
        i, j = g.choice(n, 2, replace=False)
        if J[i] == J[j]:
            th = L(g.uniform(-np.pi, np.pi))
            c, s = np.cos(th), np.sin(th)
            R = np.array([[c, s], [-s, c]], dtype=L)
        else:
            th = L(np.arctanh(g.uniform(-0.5, 0.5)))
            c, s = np.cosh(th), np.sinh(th)
            R = np.array([[c, s], [s, c]], dtype=L)
        W[:, [i, j]] = W[:, [i, j]] @ R
    sigma = g.uniform(1.0, 10.0, n).astype(L)
    G = (Q * sigma) @ W
    lam = np.sort((J * sigma.astype(np.float64) ** 2))
    return G.astype(np.float64), J, lam


def pin_prescribed(seed, n, npos):
    G, J, lam = prescribed(n, npos, seed)
    r = oracle.solve(G, J)
    return bool(r["status"] == 0 and np.max(np.abs(r["lam"] - lam) / np.abs(lam)) <= 1e-12)


def pin_svd(seed, n):
    G = np.random.default_rng(seed).standard_normal((n + 3, n))
    s = np.linalg.svd(G, compute_uv=False)
    r = oracle.solve(G, np.ones(n, dtype=np.int8))
    return bool(r["status"] == 0 and np.max(np.abs(r["lam"] - np.sort(s ** 2)) / np.sort(s ** 2)) <= 1e-12)


def pin_invariants(seed, n, hyperbolic, cplx):
    g = np.random.default_rng(seed)
    G = g.standard_normal((n + 5, n))
    if cplx:
        G = G + 1j * g.standard_normal((n + 5, n))
    J = np.ones(n, dtype=np.int8)
    if hyperbolic:
        J[g.choice(n, n // 3, replace=False)] = -1
    r = oracle.solve(G, J)
    off, mxs = oracle.check_offdiag(r["Gf"])
    vjv = oracle.check_vjv(r["V"], J, r["J"])
    res = oracle.check_factor_residual(G, r["V"], r["Gf"])
    return bool(r["status"] == 0 and off <= n * EPS and mxs <= n * EPS and vjv <= 100 * n * EPS
                and res <= 100 * n * EPS and np.all(np.sign(r["lam"]) == r["J"]))


def pin_complex_hermitian(seed, n):
    g = np.random.default_rng(seed)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    J = np.array([1] * (n - n // 3) + [-1] * (n // 3), dtype=np.int8)
    H = (G * J) @ G.conj().T
    ev = np.linalg.eigvalsh(H)
    r = oracle.solve(G, J)
    return bool(r["status"] == 0 and np.max(np.abs(r["lam"] - ev) / np.abs(ev)) <= 1e-9)


PINS = {
    "example1": pin_example1,
    "two_column_trig": lambda: pin_two_column(False, 3),
    "two_column_hyp": lambda: pin_two_column(True, 4),
    "two_column_complex": lambda: pin_two_column(True, 5, cplx=True) and pin_two_column(False, 6, cplx=True),
    "angles": lambda: pin_rotation_angles(7),
    "charpoly": lambda: all(pin_charpoly(100 + n, n, h) for n in (2, 3, 5) for h in (False, True)),
    "prescribed": lambda: pin_prescribed(8, 24, 10) and pin_prescribed(9, 30, 30),
    "svd": lambda: pin_svd(10, 25),
    "invariants": lambda: all(pin_invariants(11 + k, 20, h, c) for k, (h, c) in
                              enumerate([(False, False), (True, False), (True, True)])),
    "complex_hermitian": lambda: pin_complex_hermitian(12, 16),
}


@pytest.mark.parametrize("name", sorted(PINS))
def test_pin(name):
    oracle.set_mutation(0)
    assert PINS[name](), name


@pytest.mark.parametrize("n,h", [(2, False), (4, True), (6, False), (6, True)])
def test_charpoly_sizes(n, h):
    assert pin_charpoly(200 + n, n, h)


def test_charpoly_tall_factor():
    assert pin_charpoly(300, 3, True, m_extra=1)


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5])
def test_mutations_are_caught(mutation):
    """Plant mistake k in the oracle: at least one pin must fail."""
    try:
        oracle.set_mutation(mutation)
        failed = [name for name, f in PINS.items() if not f()]
    finally:
        oracle.set_mutation(0)
    assert failed, "mutation %d not caught by any pin" % mutation


def test_trivial_sizes():
    # one column: no rotation, lambda = j ||g||^2
    r = oracle.solve(np.array([[3.0], [4.0]]), np.array([-1], dtype=np.int8))
    assert r["status"] == 0 and r["sweeps"] == 0 and r["lam"][0] == -25.0
    # orthogonal columns: one sweep without rotation
    r = oracle.solve(np.diag([3.0, 1.0, 2.0]), np.array([1, -1, 1], dtype=np.int8))
    assert r["status"] == 0 and r["sweeps"] == 1 and r["rotations"] == 0
    assert np.array_equal(r["lam"], [-1.0, 4.0, 9.0])


def test_inputs_are_seeded():
    from paper_1008_0201_gb300 import inputs

    a, Ja = inputs.config2_hyperbolic(n=64)
    b, Jb = inputs.config2_hyperbolic(n=64)
    assert np.array_equal(a, b) and np.array_equal(Ja, Jb)
    assert np.sum(Ja > 0) == 32
    Gs, Js = inputs.config4_batched(count=20)
    assert all(8 <= g.shape[0] <= 128 and g.shape[0] == g.shape[1] for g in Gs)
    assert all(np.sum(j < 0) == int(round(0.3 * len(j))) for j in Js)
    G3, J3 = inputs.config3_graded_complex(n=32)
    col = np.linalg.norm(G3, axis=0)
    assert col[0] > 100 * col[-1]
