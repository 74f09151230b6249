"""The paper-shaped input class on the GPU against the oracle (-m gpu, through the C ABI).

Sec. 4's test matrices are symmetric with entries uniform in [-5, 5], factored by Bunch-Parlett
with complete pivoting before the hyperbolic Jacobi method.  The factor G = P L |D|^(1/2) (2x2
blocks of D diagonalized) is lower triangular up to the pivot permutation, with signs J in
pivot order: a different input class from the Gaussian factors of the other tests (structured
zeros, 2x2 pivot blocks, a sign pattern that is not sorted).  The GPU solve (hyperbolic HBSC and
HFSC, FP64 and mixed) is held to the oracle on the same (G, J) within the stated tolerances.
"""
import numpy as np
import pytest

from checks import compare, to_np
from oracle import oracle

pytestmark = pytest.mark.gpu


def _factor(n, seed):
    from paper_1008_0201_gb300 import preprocess

    H = preprocess.uniform_symmetric(n, seed)
    G, J = preprocess.factor_gjgt(H)
    return H, np.ascontiguousarray(G), np.ascontiguousarray(J, dtype=np.int8)


@pytest.mark.parametrize("n,seed", [(200, 41), (333, 42), (480, 43)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("block_mode", ["oriented", "full"])
def test_bunch_parlett_factor_vs_oracle(cuda_dev, n, seed, precision, block_mode):
    import torch

    from paper_1008_0201_gb300 import binding

    H, G, J = _factor(n, seed)
    assert 0 < np.sum(J < 0) < n
    ref = oracle.solve(G, J)
    opts = binding.default_opts(block_w=32, ordering="round_robin", factor="chol_signpiv",
                                block_mode=block_mode, precision=precision)
    out = binding.jacobi_hsvd(torch.from_numpy(G).to(cuda_dev), torch.from_numpy(J).to(cuda_dev), opts,
                              raise_on_error=False)
    torch.cuda.synchronize()
    out = to_np(out)
    assert out["status"] == 0, out["info"]
    r = compare(G, J, out, ref=ref)
    # the spectrum of H itself (LAPACK, a cross-check of the factorization, not of the solver)
    ev = np.linalg.eigvalsh(H)
    assert np.max(np.abs(out["lam"] - ev) / np.abs(ev)) <= 1e-8
    print("BP", n, precision, block_mode, out["info"]["sweeps"], r)
