"""Host-side preparation of a symmetric matrix for the one-sided solver: H -> (G, J).

The paper's experiments factor the symmetric input H before the hyperbolic Jacobi method
(Sec. 4): a symmetric indefinite factorization with complete pivoting (Bunch-Parlett),
H = P L D L^T P^T with D block diagonal (1x1 and 2x2 blocks), turned into H = G J G^T by
diagonalizing each 2x2 block of D.  This module writes that step in numpy for the paper-shaped
workload (entries uniform in [-5, 5]).  It is set-up outside the hot path: the solver takes G and
J; nothing in the library calls this module.
"""
import numpy as np

ALPHA = (1.0 + np.sqrt(17.0)) / 8.0  # Bunch-Parlett growth-balancing constant


def bunch_parlett(H):
    """Symmetric indefinite factorization with complete pivoting (Bunch and Parlett, 1971).

    Returns (perm, L, blocks) with H[perm][:, perm] = L D L^T, L unit lower triangular, and
    blocks a list of (start, size, D_block) for the 1x1 and 2x2 diagonal blocks of D.
    At step k, with mu0 = max |a_ij| over the trailing matrix and mu1 = max |a_ii| over its
    diagonal, a 1x1 pivot (the largest diagonal) is taken when mu1 >= ALPHA mu0, else a 2x2
    pivot on the rows / columns of the largest off-diagonal entry."""
    A = np.array(H, dtype=np.float64, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    L = np.eye(n)
    blocks = []

    def swap(i, j):
        if i == j:
            return
        A[[i, j], :] = A[[j, i], :]
        A[:, [i, j]] = A[:, [j, i]]
        perm[[i, j]] = perm[[j, i]]
        L[[i, j], :k] = L[[j, i], :k]

    k = 0
    while k < n:
        T = A[k:, k:]
        d = np.abs(np.diag(T))
        q = int(np.argmax(d))
        mu1 = d[q]
        if n - k > 1:
            off = np.abs(T)
            np.fill_diagonal(off, 0.0)
            rs = int(np.argmax(off))
            r, s = divmod(rs, n - k)
            mu0 = off[r, s]
        else:
            mu0, r, s = 0.0, 0, 0
        if mu1 >= ALPHA * mu0 or n - k == 1:
            swap(k, k + q)
            d11 = A[k, k]
            if d11 == 0.0:
                raise ValueError("singular matrix")
            l = A[k + 1:, k] / d11
            L[k + 1:, k] = l
            A[k + 1:, k + 1:] -= np.outer(l, A[k, k + 1:])
            A[k + 1:, k] = 0.0
            A[k, k + 1:] = 0.0
            blocks.append((k, 1, np.array([[d11]])))
            k += 1
        else:
            r, s = min(r, s), max(r, s)
            swap(k, k + r)
            swap(k + 1, k + s)
            E = A[k:k + 2, k:k + 2].copy()
            Einv = np.linalg.inv(E)
            C = A[k + 2:, k:k + 2]
            Lb = C @ Einv
            L[k + 2:, k:k + 2] = Lb
            A[k + 2:, k + 2:] -= Lb @ C.T
            A[k + 2:, k:k + 2] = 0.0
            A[k:k + 2, k + 2:] = 0.0
            blocks.append((k, 2, E))
            k += 2
    return perm, L, blocks


def factor_gjgt(H):
    """(G, J) with H = G J G^T: G = P L B, where B diagonalizes each block of D,
    D_b = Q diag(l) Q^T  ->  B_b = Q diag(sqrt|l|), J_b = sign(l)."""
    n = H.shape[0]
    perm, L, blocks = bunch_parlett(H)
    B = np.zeros((n, n))
    J = np.ones(n, dtype=np.int8)
    for start, size, D in blocks:
        if size == 1:
            B[start, start] = np.sqrt(abs(D[0, 0]))
            J[start] = 1 if D[0, 0] > 0 else -1
        else:
            lam, Q = np.linalg.eigh(D)
            B[start:start + 2, start:start + 2] = Q * np.sqrt(np.abs(lam))[None, :]
            J[start:start + 2] = np.where(lam > 0, 1, -1)
    G = np.empty((n, n))
    G[perm, :] = L @ B  # rows back to the input order: H = G J G^T
    return G, J


def uniform_symmetric(n, seed, lo=-5.0, hi=5.0):
    """Symmetric matrix with entries uniform in [lo, hi] (upper triangle drawn, mirrored), the
    shape of the paper's test matrices (Sec. 4)."""
    g = np.random.default_rng(seed)
    A = g.uniform(lo, hi, size=(n, n))
    return np.triu(A) + np.triu(A, 1).T
