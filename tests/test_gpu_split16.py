"""The FP64 product paths vs the CPU oracle: exact FP16 digit products (f64_products =
"split16", the default: update on the tcgen05 tensor cores, Gram on the warp-level FP16 mma;
"split16_tc": Gram on tcgen05 too) and FP64 tensor-core mma ("mma").

The Gram, update and V_P residual products of the FP64 sweeps run as sums of exact FP16 x FP16
tensor-core products of 7-bit digit slices (error-free splitting after Ozaki et al.); each
product term is exact to 2^-53 of its operand group bounds, so every result is held to the same
tolerances as the FP64 mma path (tests/checks.py).  The cases cover the scale groups of both
products: tall factors (several 128-row Gram stages per CTA), graded columns (a small column
next to a large one in the update), nearly parallel columns, ragged block widths, both
precisions, the batched and the complex entry points.
"""
import numpy as np
import pytest

from checks import EPS, compare, to_np
from test_gpu_batched import check_all, run_batched, small_batch
from test_gpu_parity import run

pytestmark = pytest.mark.gpu

S16 = dict(f64_products="split16")
PRODUCTS = ["split16", "split16_tc"]


@pytest.mark.parametrize("factor", ["chol", "chol_diagpiv", "chol_signpiv"])
def test_split16_config1_pd(cuda_dev, factor):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config1_pd()
    out = run(G, None, cuda_dev, block_w=8, factor=factor, **S16)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("precision,block_mode", [("fp64", "full"), ("fp64", "oriented"), ("fp32", "full"),
                                                  ("fp32", "oriented")])
@pytest.mark.parametrize("prod", PRODUCTS)
def test_split16_config2(cuda_dev, prod, precision, block_mode):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic()
    out = run(G, J, cuda_dev, block_w=32, precision=precision, block_mode=block_mode, f64_products=prod)
    assert out["status"] == 0, out["info"]
    r = compare(G, J, out)
    print("C2-split16", precision, block_mode, out["info"]["sweeps"], r)


@pytest.mark.parametrize("m,n,w,frac", [(130, 100, 16, 0.4), (37, 37, 5, 0.5), (200, 61, 7, 0.0),
                                        (48, 33, 32, 0.3), (17, 3, 1, 0.34), (4500, 40, 8, 0.3)])
@pytest.mark.parametrize("prod", PRODUCTS)
def test_split16_ragged_and_tall(cuda_dev, prod, m, n, w, frac):
    g = np.random.default_rng(5000 + m * 7 + n)
    G = g.standard_normal((m, n))
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=int(round(frac * n)), replace=False)] = -1
    out = run(G, J, cuda_dev, block_w=w, ordering="round_robin", f64_products=prod)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("span", [4, 12])
@pytest.mark.parametrize("prod", PRODUCTS)
def test_split16_graded_columns(cuda_dev, prod, span):
    """G = B D with column scales 10^(-span/2 .. span/2) in shuffled order: every pivot block mixes
    columns of very different size, the case the per-column scaling of the update is for."""
    g = np.random.default_rng(5100 + span)
    m, n = 160, 96
    d = 10.0 ** np.linspace(-span / 2, span / 2, n)
    G = g.standard_normal((m, n)) * g.permutation(d)[None, :]
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=40, replace=False)] = -1
    for prec in ("fp64", "fp32"):
        out = run(G, J, cuda_dev, block_w=16, precision=prec, f64_products=prod)
        assert out["status"] == 0, (prec, out["info"])
        compare(G, J, out)


@pytest.mark.parametrize("signs", ["same", "opposite"])
def test_split16_ill_conditioned_block(cuda_dev, signs):
    g = np.random.default_rng(4242)
    m, n = 80, 40
    G = g.standard_normal((m, n))
    G[:, 7] = G[:, 2] + 1e-4 * g.standard_normal(m)
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=12, replace=False)] = -1
    J[2] = 1
    J[7] = 1 if signs == "same" else -1
    for prec in ("fp64", "fp32"):
        out = run(G, J, cuda_dev, block_w=20, precision=prec, **S16)
        assert out["status"] == 0, (prec, out["info"])
        compare(G, J, out)


def test_split16_agrees_with_mma(cuda_dev):
    """Both product paths solve the same problem to the oracle's tolerance, so their eigenvalues
    agree to twice that bound."""
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic(n=256, salt=5)
    a = run(G, J, cuda_dev, block_w=32, **S16)
    b = run(G, J, cuda_dev, block_w=32, f64_products="mma")
    assert a["status"] == 0 and b["status"] == 0
    B = G / np.linalg.norm(G, axis=0)
    kappa = np.linalg.cond(B) ** 2
    n = G.shape[1]
    rel = np.max(np.abs(a["lam"] - b["lam"]) / np.abs(b["lam"]))
    assert rel <= 2 * 50 * n * EPS * kappa, rel


def test_split16_deterministic(cuda_dev):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic(n=192, salt=3)
    a = run(G, J, cuda_dev, block_w=32, **S16)
    b = run(G, J, cuda_dev, block_w=32, **S16)
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["V"], b["V"])


def test_split16_batched(cuda_dev):
    Gs, Js = small_batch(16, salt=21, pd_every=4)
    outs, rc = run_batched(Gs, Js, cuda_dev, **S16)
    assert rc == 0
    check_all(Gs, Js, outs)


def _complex_graded(dev, **kw):
    import torch

    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(5200)
    m, n = 60, 40
    G = (g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))) * np.sqrt(0.5)
    G = G * (10.0 ** np.linspace(0, -3, n))[None, :]
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=15, replace=False)] = -1
    opts = binding.default_opts(block_w=8, **kw)
    out = binding.jacobi_hsvd(torch.from_numpy(G).to(dev), torch.from_numpy(J).to(dev), opts, raise_on_error=False)
    torch.cuda.synchronize()
    out = to_np(out)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


def test_split16_complex(cuda_dev):
    _complex_graded(cuda_dev, **S16)


MMA = dict(f64_products="mma")


@pytest.mark.parametrize("precision,block_mode", [("fp64", "full"), ("fp64", "oriented"), ("fp32", "oriented")])
def test_mma_products_config2(cuda_dev, precision, block_mode):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic()
    out = run(G, J, cuda_dev, block_w=32, precision=precision, block_mode=block_mode, **MMA)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("m,n,w,frac", [(130, 100, 16, 0.4), (37, 37, 5, 0.5), (4500, 40, 8, 0.3)])
def test_mma_products_ragged(cuda_dev, m, n, w, frac):
    g = np.random.default_rng(5300 + m * 7 + n)
    G = g.standard_normal((m, n))
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=int(round(frac * n)), replace=False)] = -1
    out = run(G, J, cuda_dev, block_w=w, **MMA)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


def test_mma_products_batched_and_complex(cuda_dev):
    Gs, Js = small_batch(8, salt=22, pd_every=3)
    outs, rc = run_batched(Gs, Js, cuda_dev, **MMA)
    assert rc == 0
    check_all(Gs, Js, outs)
    _complex_graded(cuda_dev, **MMA)
