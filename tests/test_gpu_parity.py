"""GPU path (through the C ABI) vs the CPU oracle on the same seeded inputs."""
import ctypes

import numpy as np
import pytest

from checks import EPS, compare, to_np

pytestmark = pytest.mark.gpu


def run(G, J, dev, **kw):
    import torch

    from paper_1008_0201_gb300 import binding

    opts = binding.default_opts(**kw)
    Gd = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
    if J is None or np.all(J > 0):
        out = binding.jacobi_eig_pd(Gd, opts, raise_on_error=False) if J is None else \
            binding.jacobi_hsvd(Gd, torch.from_numpy(J).to(dev), opts, raise_on_error=False)
    else:
        out = binding.jacobi_hsvd(Gd, torch.from_numpy(J).to(dev), opts, raise_on_error=False)
    torch.cuda.synchronize()
    return to_np(out)


@pytest.mark.parametrize("ordering", ["modulus", "modulus_mod", "round_robin", "cycle_weight"])
@pytest.mark.parametrize("factor", ["chol", "chol_diagpiv", "chol_signpiv"])
def test_config1_pd_64(cuda_dev, ordering, factor):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config1_pd()
    out = run(G, None, cuda_dev, block_w=8, ordering=ordering, factor=factor)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("ordering", ["round_robin", "cycle_weight", "modulus"])
@pytest.mark.parametrize("factor", ["chol", "chol_diagpiv", "chol_signpiv"])
def test_config2_hyperbolic_512(cuda_dev, ordering, factor):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic()
    out = run(G, J, cuda_dev, block_w=32, ordering=ordering, factor=factor)
    assert out["status"] == 0, out["info"]
    r = compare(G, J, out)
    print("C2", ordering, factor, out["info"], r)


@pytest.mark.parametrize("ordering", ["round_robin", "cycle_weight", "modulus"])
@pytest.mark.parametrize("factor", ["chol", "chol_signpiv"])
def test_config2_mixed_precision(cuda_dev, ordering, factor):
    """FP32 sweeps, FP64 J-orthogonalization of V, FP64 polish: same tolerances as FP64."""
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic()
    out = run(G, J, cuda_dev, block_w=32, ordering=ordering, factor=factor, precision="fp32")
    assert out["status"] == 0, out["info"]
    assert out["info"]["lowp_sweeps"] >= 1
    r = compare(G, J, out)
    print("C2-mixed", ordering, factor, out["info"], r)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ordering", ["round_robin", "cycle_weight", "modulus_mod"])
def test_block_oriented(cuda_dev, precision, ordering):
    """Block-oriented HB/HBSC (Sec. 2.2, Algorithm 3.4): one inner sweep per pivot block, the
    cross block only after the first step of a sweep; same tolerances."""
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic()
    out = run(G, J, cuda_dev, block_w=32, ordering=ordering, block_mode="oriented", precision=precision)
    assert out["status"] == 0, out["info"]
    r = compare(G, J, out)
    print("C2-oriented", ordering, precision, out["info"]["sweeps"], r)
    G1, J1 = inputs.config1_pd()
    out1 = run(G1, None, cuda_dev, block_w=8, ordering=ordering, block_mode="oriented", precision=precision)
    assert out1["status"] == 0, out1["info"]
    compare(G1, J1, out1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config1_precisions(cuda_dev, precision):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config1_pd()
    out = run(G, None, cuda_dev, block_w=8, precision=precision)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("m,n,w,frac,prec", [(130, 100, 16, 0.4, "fp32"), (37, 37, 5, 0.5, "fp32"),
                                             (200, 61, 7, 0.0, "fp32")])
def test_ragged_mixed(cuda_dev, m, n, w, frac, prec):
    g = np.random.default_rng(2000 + m * 7 + n)
    G = g.standard_normal((m, n))
    J = np.ones(n, dtype=np.int8)
    k = int(round(frac * n))
    J[g.choice(n, size=k, replace=False)] = -1
    out = run(G, J, cuda_dev, block_w=w, ordering="cycle_weight", precision=prec)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


@pytest.mark.parametrize("m,n,w,frac", [(130, 100, 16, 0.4), (37, 37, 5, 0.5), (200, 61, 7, 0.0),
                                        (48, 33, 32, 0.3), (17, 3, 1, 0.34), (64, 2, 1, 0.5)])
def test_ragged_shapes(cuda_dev, m, n, w, frac):
    g = np.random.default_rng(1000 + m * 7 + n)
    G = g.standard_normal((m, n))
    J = np.ones(n, dtype=np.int8)
    k = int(round(frac * n))
    J[g.choice(n, size=k, replace=False)] = -1  # unsorted signs: exercises the internal sort
    out = run(G, J, cuda_dev, block_w=w, ordering="round_robin")
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


def test_single_column(cuda_dev):
    G = np.array([[3.0], [4.0]])
    out = run(G, np.array([-1], dtype=np.int8), cuda_dev, block_w=4)
    assert out["status"] == 0
    assert out["lam"][0] == -25.0
    assert np.allclose(out["U"][:, 0], [0.6, 0.8], rtol=0, atol=2.3e-16)


def test_already_diagonal(cuda_dev):
    # orthogonal columns with distinct norms: no rotation, exact eigenvalues
    G = np.diag([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    J = np.array([1, -1, 1, -1, 1, -1], dtype=np.int8)
    out = run(G, J, cuda_dev, block_w=2)
    assert out["status"] == 0
    assert out["info"]["rotations"] == 0 and out["info"]["sweeps"] == 1
    assert np.array_equal(out["lam"], np.array([-36.0, -16.0, -4.0, 1.0, 9.0, 25.0]))


@pytest.mark.parametrize("signs", ["same", "opposite"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ill_conditioned_block(cuda_dev, signs, precision):
    """Two nearly parallel columns (angle ~1e-4, kappa(A~) ~ 1e8) inside one pivot block: the
    FP32 Cholesky of the scaled Gram breaks down there, the block is factored and rotated in
    FP64 instead, and the result still meets the oracle tolerances."""
    g = np.random.default_rng(4242)
    m, n = 80, 40
    G = g.standard_normal((m, n))
    G[:, 7] = G[:, 2] + 1e-4 * g.standard_normal(m)
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=12, replace=False)] = -1
    J[2] = 1
    J[7] = 1 if signs == "same" else -1
    out = run(G, J, cuda_dev, block_w=20, precision=precision)
    assert out["status"] == 0, out["info"]
    compare(G, J, out)


def test_deterministic(cuda_dev):
    from paper_1008_0201_gb300 import inputs

    G, J = inputs.config2_hyperbolic(n=192, salt=3)
    a = run(G, J, cuda_dev, block_w=32)
    b = run(G, J, cuda_dev, block_w=32)
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["V"], b["V"])


def test_errors(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(5)
    G = g.standard_normal((40, 40))
    J = np.array([1] * 20 + [-1] * 20, dtype=np.int8)
    # non-finite input
    Gn = G.copy()
    Gn[3, 7] = np.nan
    out = run(Gn, J, cuda_dev, block_w=8)
    assert out["status"] == binding.JAC_ENONFINITE
    # invalid signature entry: argument 6
    Jb = J.copy()
    Jb[4] = 0
    out = run(G, Jb, cuda_dev, block_w=8)
    assert out["status"] == -6
    # rank deficient factor: a repeated column inside one block makes the first pivot block
    # singular (Sec. 3.2 needs full column rank), in the hyperbolic and in the PD path
    Gr = G.copy()
    Gr[:, 1] = Gr[:, 0]
    out = run(Gr, J, cuda_dev, block_w=8)
    assert out["status"] == binding.JAC_ENOTPD
    out = run(Gr, None, cuda_dev, block_w=8)
    assert out["status"] == binding.JAC_ENOTPD
    # sweep cap
    out = run(G, J, cuda_dev, block_w=8, max_sweeps=1)
    assert out["status"] == binding.JAC_ENOTCONV and out["info"]["sweeps"] == 1
    # bad options: block width out of range (argument 7 = opts)
    out = run(G, J, cuda_dev, block_w=33)
    assert out["status"] == -7
    # m < n (argument 2)
    out = run(G[:10, :20], J[:20], cuda_dev, block_w=8)
    assert out["status"] == -2


def test_leading_dimension_and_no_v(cuda_dev):
    """ldg > m through the raw C entry point; want_v = 0 leaves V untouched."""
    import torch

    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(11)
    m, n, ld = 50, 40, 64
    G = g.standard_normal((m, n))
    J = np.array([1] * 25 + [-1] * 15, dtype=np.int8)
    buf = np.zeros((n, ld))
    buf[:, :m] = G.T  # column c at buf[c, :m]
    Gd = torch.from_numpy(buf.copy()).to(cuda_dev)
    Jd = torch.from_numpy(J).to(cuda_dev)
    lam = torch.empty(n, dtype=torch.float64, device=cuda_dev)
    U = torch.empty((n, ld), dtype=torch.float64, device=cuda_dev)
    opts = binding.default_opts(block_w=8, want_v=0)
    rc, info = binding.jacobi_hsvd_raw(m, n, Gd.data_ptr(), ld, Jd.data_ptr(), opts, lam.data_ptr(), U.data_ptr(),
                                       ld, 0, n, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0, info
    Gout = Gd.cpu().numpy()[:, :m].T
    assert np.all(Gd.cpu().numpy()[:, m:] == 0.0)  # padding rows of the caller's buffer untouched
    out = {"lam": lam.cpu().numpy(), "G": Gout, "U": U.cpu().numpy()[:, :m].T, "V": None}
    compare(G, J, out)
