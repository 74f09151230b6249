"""FP64 accuracy of the rotation angles on nearly diagonal, graded pivot blocks (-m gpu).

The pivot kernel computes its 2x2 rotation parameters in FP32 on the shifted representation
A_P = D (I + E) D, R = D_P + F, V_P = I + W (F, W small, stored in FP32), and makes each V_P
J-unitary in FP64 afterwards.  The case where FP32 parameters could cost FP64 accuracy is a
block whose scaled off-diagonal entries |a_ij| / sqrt(a_ii a_jj) lie between 2^-53 and 2^-24:
each still needs a rotation (they exceed tol = n 2^-53), the angles are tiny, and the diagonal
is graded over many decades.  These factors are G = Q (I + E) diag(d): Q with orthonormal
columns, E with zero diagonal and entries of size 2^-k, d spanning 10 decades in shuffled
order.  kappa_2(A) is ~1, so the eigenvalue bound 50 n eps kappa_2(A) asks for FP64 accuracy
relative to each eigenvalue; off-norm, J-unitarity and residual are checked as everywhere.
"""
import numpy as np
import pytest

from checks import compare, to_np
from oracle import oracle

pytestmark = pytest.mark.gpu


def _factor(m, n, k, hyperbolic, seed):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((m, n)))
    E = g.standard_normal((n, n)) * 2.0 ** -k
    np.fill_diagonal(E, 0.0)
    d = 10.0 ** (-10.0 * g.permutation(n) / n)
    G = (Q @ (np.eye(n) + E)) * d[None, :]
    J = np.ones(n, dtype=np.int8)
    if hyperbolic:
        J[g.choice(n, n // 3, replace=False)] = -1
    return np.ascontiguousarray(G), J


@pytest.mark.parametrize("k", [44, 36, 30, 25])
@pytest.mark.parametrize("hyperbolic", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiny_graded_rotations(cuda_dev, k, hyperbolic, precision):
    import torch

    from paper_1008_0201_gb300 import binding

    m, n = 160, 96
    G, J = _factor(m, n, k, hyperbolic, 900 + k)
    ref = oracle.solve(G, J)
    scaled0 = oracle.check_offdiag(G)[1]
    assert n * 2.0 ** -53 < scaled0 < 2.0 ** -20  # every block needs tiny rotations
    opts = binding.default_opts(block_w=16, ordering="round_robin", factor="chol_signpiv", precision=precision)
    out = binding.jacobi_hsvd(torch.from_numpy(G).to(cuda_dev), torch.from_numpy(J).to(cuda_dev), opts,
                              raise_on_error=False)
    torch.cuda.synchronize()
    out = to_np(out)
    assert out["status"] == 0, out["info"]
    assert out["info"]["rotations"] > 0
    r = compare(G, J, out, ref=ref)
    assert r["eig_bound"] < 1e-10  # the test demands FP64-level eigenvalues
    print("tiny", k, hyperbolic, precision, r)
