"""Host-side Bunch-Parlett preparation of the paper-shaped workload (symmetric, entries uniform
in [-5, 5]): H = G J G^T to rounding, 2x2 pivots exercised, the spectrum of H reproduced by the
oracle run on (G, J).  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1008_0201_gb300 import preprocess


@pytest.mark.parametrize("n,seed", [(6, 1), (50, 2), (200, 3)])
def test_bunch_parlett_reconstructs(n, seed):
    H = preprocess.uniform_symmetric(n, seed)
    perm, L, blocks = preprocess.bunch_parlett(H)
    assert np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.diag(L), 1.0)
    D = np.zeros((n, n))
    for s, size, Db in blocks:
        D[s:s + size, s:s + size] = Db
    assert sum(b[1] for b in blocks) == n
    Hp = H[np.ix_(perm, perm)]
    assert np.linalg.norm(L @ D @ L.T - Hp) <= 1e-12 * np.linalg.norm(H)
    # complete pivoting bounds the multipliers
    assert np.abs(L).max() <= 1.0 / preprocess.ALPHA + 1e-12 or n <= 2
    G, J = preprocess.factor_gjgt(H)
    assert set(np.unique(J)) <= {-1, 1}
    assert np.linalg.norm(G @ np.diag(J.astype(float)) @ G.T - H) <= 1e-12 * np.linalg.norm(H)


def test_two_by_two_pivots_occur():
    sizes = [b[1] for seed in range(4) for b in preprocess.bunch_parlett(preprocess.uniform_symmetric(60, seed))[2]]
    assert 2 in sizes and 1 in sizes


def test_oracle_on_factor_reproduces_spectrum():
    H = preprocess.uniform_symmetric(40, 7)
    G, J = preprocess.factor_gjgt(H)
    r = oracle.solve(G, J)
    assert r["status"] == 0
    ev = np.linalg.eigvalsh(H)
    assert np.allclose(np.sort(r["lam"]), ev, rtol=1e-11, atol=1e-11 * np.abs(ev).max())
