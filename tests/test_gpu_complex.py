"""Complex Hermitian problems (dtype JAC_C128) through the C ABI against the complex oracle.

Inputs are seeded complex Gaussian factors, positive definite and indefinite, and scaled-down
copies of the graded workload G = B D (B complex Gaussian, D = diag(10^(-8 i / n))); every
result is held to the same tolerances as the real problems (tests/checks.py).
"""
import numpy as np
import pytest

from checks import compare, to_np

pytestmark = pytest.mark.gpu


def run(G, J, dev, **kw):
    import torch

    from paper_1008_0201_gb300 import binding

    opts = binding.default_opts(**kw)
    Gd = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
    if J is None:
        out = binding.jacobi_eig_pd(Gd, opts, raise_on_error=False)
    else:
        out = binding.jacobi_hsvd(Gd, torch.from_numpy(J).to(dev), opts, raise_on_error=False)
    torch.cuda.synchronize()
    return to_np(out)


def cgauss(g, m, n):
    return (g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))) * np.sqrt(0.5)


@pytest.mark.parametrize("m,n,w", [(24, 24, 4), (48, 48, 8), (70, 45, 8)])
def test_complex_pd(cuda_dev, m, n, w):
    g = np.random.default_rng(300 + n)
    G = cgauss(g, m, n)
    out = run(G, None, cuda_dev, block_w=w)
    assert out["status"] == 0, out["info"]
    assert out["G"].dtype == np.complex128 and out["V"].dtype == np.complex128
    compare(G, np.ones(n, dtype=np.int8), out)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("block_mode", ["full", "oriented"])
def test_complex_hyperbolic(cuda_dev, precision, block_mode):
    g = np.random.default_rng(311)
    m, n = 60, 40
    G = cgauss(g, m, n)
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=15, replace=False)] = -1
    out = run(G, J, cuda_dev, block_w=8, precision=precision, block_mode=block_mode)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("n,w", [(64, 16), (128, 32)])
def test_complex_graded(cuda_dev, n, w):
    """The graded workload at reduced order: column norms from 1 down to 1e-8."""
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config3_graded_complex(n=n, salt=1)
    out = run(G, None, cuda_dev, block_w=w, precision="fp32")
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


def test_complex_errors(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(5)
    G = cgauss(g, 12, 12)
    Gn = G.copy()
    Gn[2, 3] = np.nan
    assert run(Gn, None, cuda_dev, block_w=4)["status"] == binding.JAC_ENONFINITE
    J = np.ones(12, dtype=np.int8)
    J[4] = 3
    with pytest.raises(binding.JacobiError) as e:
        binding.jacobi_hsvd(torch.from_numpy(G).to(cuda_dev), torch.from_numpy(J).to(cuda_dev),
                            binding.default_opts(block_w=4))
    assert e.value.code == -6


def test_complex_graded_full_size_properties(cuda_dev):
    """The graded workload at full size (n = 4096, mixed precision).  The oracle cannot run at
    this order, so the test checks what holds at any size, on 64 sampled columns: the scaled
    off-diagonals are within tol = n eps, V is unitary to 100 n eps, G_out = G_in V to 100 n eps.
    It also checks that the eigenvalues are positive and ascending."""
    import torch

    from paper_1008_0201_gb300 import binding, inputs

    G, _ = inputs.config3_graded_complex()
    n = G.shape[1]
    out = binding.jacobi_eig_pd(torch.from_numpy(G).to(cuda_dev),
                                binding.default_opts(block_w=32, ordering="round_robin", block_mode="oriented",
                                                     precision="fp32"), want_u=False)
    torch.cuda.synchronize()
    assert out["status"] == 0, out["info"]
    lam = out["lam"].cpu().numpy()
    assert np.all(lam > 0) and np.all(np.diff(lam) >= 0)
    Go, V = out["G"].cpu().numpy(), out["V"].cpu().numpy()
    idx = np.random.default_rng(9).choice(n, size=64, replace=False)
    Gs = Go[:, idx]
    nr = np.linalg.norm(Gs, axis=0)
    C = np.abs(Gs.conj().T @ Gs) / np.outer(nr, nr)
    np.fill_diagonal(C, 0.0)
    eps = 2.0 ** -53
    assert C.max() <= n * eps, C.max()
    Vs = V[:, idx]
    assert np.abs(Vs.conj().T @ Vs - np.eye(64)).max() <= 100 * n * eps
    assert np.linalg.norm(G @ Vs - Gs) / np.linalg.norm(G) <= 100 * n * eps


def _read_golden(path):
    meta, lam, in_lam = {}, [], False
    with open(path) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            if ln == "lambda":
                in_lam = True
            elif in_lam:
                lam.append(float(ln))
            else:
                k, v = ln.split(None, 1)
                meta[k] = v
    return meta, np.array(lam)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_complex_graded_full_size_vs_oracle(cuda_dev, precision):
    """The graded workload at full size (n = 4096) against the oracle's eigenvalues for the same
    draws (tests/golden/c3_graded_complex_n4096.txt, written by make_c3_golden.py from the oracle
    alone and keyed by a hash of the Gaussian draws), element by element, within the stated bound
    50 n eps kappa_2(A), kappa_2(A) = kappa_2(B_hat)^2, and within the tighter 50 n eps kappa_2(B_hat)."""
    import hashlib
    import os

    import torch

    from paper_1008_0201_gb300 import binding, inputs

    meta, ref = _read_golden(os.path.join(os.path.dirname(__file__), "golden", "c3_graded_complex_n4096.txt"))
    n = int(meta["n"])
    g = inputs.rng(3, 0)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.standard_normal((n, n))).tobytes())
    h.update(np.ascontiguousarray(g.standard_normal((n, n))).tobytes())
    assert h.hexdigest() == meta["draws_sha256"], "the seeded draws differ from those the oracle solved"
    G, _ = inputs.config3_graded_complex(n)
    out = binding.jacobi_eig_pd(torch.from_numpy(G).to(cuda_dev),
                                binding.default_opts(block_w=32, ordering="round_robin", block_mode="oriented",
                                                     precision=precision), want_u=False)
    torch.cuda.synchronize()
    assert out["status"] == 0, out["info"]
    lam = out["lam"].cpu().numpy()
    kb = float(meta["kappa2_bhat"])
    eps = 2.0 ** -53
    rel = np.max(np.abs(lam - ref) / np.abs(ref))
    assert rel <= 50 * n * eps * kb * kb, (rel, 50 * n * eps * kb * kb)
    assert rel <= 50 * n * eps * kb, (rel, 50 * n * eps * kb)
    print("C3 full size", precision, "max rel err %.3e" % rel, "bound(kappa_bhat) %.3e" % (50 * n * eps * kb),
          "sweeps", out["info"]["sweeps"])
