"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the tests, the bench and the smoke check; holds random draws and sign patterns only
(none of the method's arithmetic).  The paper's own test matrices (Sec. 4: symmetric, entries
uniform in [-5, 5] drawn by LAPACK's dlarnd, then Bunch-Parlett factored) are not reproducible
here; these generators stand in for them with the shapes of the benchmark configurations.
"""
import numpy as np

SEED_BASE = 10080201


def rng(config, salt=0):
    return np.random.default_rng(SEED_BASE + int(config) + 1000 * int(salt))


def gaussian_factor(m, n, seed):
    """G (m x n), i.i.d. N(0, 1) float64."""
    return np.random.default_rng(seed).standard_normal((m, n))


def signature(n, npos):
    """J = diag(+1 x npos, -1 x (n - npos)) as int8."""
    J = -np.ones(n, dtype=np.int8)
    J[:npos] = 1
    return J


def random_signature(n, frac_neg, g):
    """J with round(frac_neg * n) entries -1 at random positions (generator g)."""
    J = np.ones(n, dtype=np.int8)
    k = int(round(frac_neg * n))
    J[g.choice(n, size=k, replace=False)] = -1
    return J


def config1_pd(n=64, salt=0):
    """Plain trigonometric case: G n x n Gaussian, H = G G^T positive definite, J = I."""
    g = rng(1, salt)
    return g.standard_normal((n, n)), np.ones(n, dtype=np.int8)


def config2_hyperbolic(n=512, salt=0):
    """Hyperbolic SVD case: G n x n Gaussian, J = diag(+1 x n/2, -1 x n/2)."""
    g = rng(2, salt)
    return g.standard_normal((n, n)), signature(n, n // 2)


def config3_graded_complex(n=4096, salt=0):
    """Graded complex case: G = B D, B complex Gaussian (re, im i.i.d. N(0, 1/2)),
    D = diag(10^(-8 i / n)), J = I."""
    g = rng(3, salt)
    B = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * np.sqrt(0.5)
    d = 10.0 ** (-8.0 * np.arange(n) / n)
    return B * d[None, :], np.ones(n, dtype=np.int8)


def config4_batched(count=10000, lo=8, hi=128, frac_neg=0.3, salt=0):
    """Batched uneven orders n_b ~ U{lo..hi}, m_b = n_b, G Gaussian, J with 30% -1 entries."""
    g = rng(4, salt)
    sizes = g.integers(lo, hi + 1, size=count)
    Gs, Js = [], []
    for n in sizes:
        Gs.append(g.standard_normal((int(n), int(n))))
        Js.append(random_signature(int(n), frac_neg, g))
    return Gs, Js


def config5_backward(batch=256, n=256, salt=0):
    """Differentiation case: G (batch, n, n) Gaussian, H = G G^T + 0.1 I; loss weights w (n)
    and C (n x 4), seeded."""
    g = rng(5, salt)
    G = g.standard_normal((batch, n, n))
    w = g.standard_normal(n)
    C = g.standard_normal((n, 4))
    return G, w, C
