"""The fused FP32 step (Gram, pivot and update of a pair in one kernel) vs the CPU oracle.

The FP32 sweeps of problems with few rows (m <= 96 for pivot blocks of k <= 32 columns, m <= 192
for k <= 64) run one kernel per step that keeps X_P = [G_p G_q] in shared memory from the Gram
block to the update.  Every case runs with the fused step on and off: both results are held to
the oracle tolerances (FP64 after the polish of the mixed mode, eps = 2^-24 for the FP32-only
sweeps), and the kernel timing hooks show which path ran.
"""
import numpy as np
import pytest

from checks import EPS, EPS32, compare, to_np
from test_gpu_batched import check_all, run_batched, small_batch

pytestmark = pytest.mark.gpu

# rows at and around the staging limits (96 rows at k <= 32, 192 rows at k <= 64), ragged
# widths, the J = I and indefinite cases
CASES = [(64, 64, 8, 0.0), (96, 80, 16, 0.3), (37, 37, 5, 0.5), (190, 150, 32, 0.4), (192, 128, 24, 0.0),
         (80, 41, 20, 0.5), (9, 9, 4, 0.34)]


def solve(G, J, dev, fused, **kw):
    import torch

    from paper_1008_0201_gb300 import binding

    opts = binding.default_opts(fused_step=fused, **kw)
    Gd = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
    binding.jacobi_profile_begin(("step_fused", "gram_lowp"))
    try:
        out = binding.jacobi_hsvd(Gd, torch.from_numpy(J).to(dev), opts, raise_on_error=False)
        torch.cuda.synchronize()
        launches = {k: binding.jacobi_profile_read(k)[1] for k in ("step_fused", "gram_lowp")}
    finally:
        binding.jacobi_profile_end()
    return to_np(out), launches


def draw(m, n, frac, salt):
    g = np.random.default_rng(7100 + 13 * m + n + salt)
    G = g.standard_normal((m, n))
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=int(round(frac * n)), replace=False)] = -1
    return G, J


@pytest.mark.parametrize("precision", ["fp32", "fp32_only"])
@pytest.mark.parametrize("m,n,w,frac", CASES)
def test_fused_step_vs_oracle(cuda_dev, m, n, w, frac, precision):
    import oracle

    G, J = draw(m, n, frac, 0)
    ref = oracle.solve(G, J)
    eps = EPS if precision == "fp32" else EPS32
    for fused in (1, 0):
        out, launches = solve(G, J, cuda_dev, fused, block_w=w, precision=precision)
        assert out["status"] == 0, (fused, out["info"])
        if fused:
            assert launches["step_fused"] > 0 and launches["gram_lowp"] == 0, launches
        else:
            assert launches["step_fused"] == 0 and launches["gram_lowp"] > 0, launches
        compare(G, J, out, ref=ref, eps=eps)


def test_fused_step_not_used_above_the_row_limit(cuda_dev):
    # 112 padded rows with blocks of k <= 32 columns: above the 96-row staging limit
    G, J = draw(100, 60, 0.3, 1)
    out, launches = solve(G, J, cuda_dev, 1, block_w=16, precision="fp32_only")
    assert out["status"] == 0
    assert launches["step_fused"] == 0 and launches["gram_lowp"] > 0, launches
    compare(G, J, out, eps=EPS32)


@pytest.mark.parametrize("signs", ["same", "opposite"])
def test_fused_step_hands_over_ill_conditioned_blocks(cuda_dev, signs):
    """Two nearly parallel columns (angle 1.5e-3: scaled Schur pivot ~2e-6, below the 64 eps_32
    the FP32 Cholesky accepts, far above the ~5e-7 error of an FP32 Gram of 80 rows) inside one
    pivot block: the fused kernel hands the block to the FP64 pivot kernel, whose transform the
    plain FP32 update applies in the same step (FP32-only sweeps); both paths agree."""
    import oracle

    g = np.random.default_rng(4343)
    m, n = 80, 40
    G = g.standard_normal((m, n))
    G[:, 7] = G[:, 2] + 1.5e-3 * g.standard_normal(m)
    J = np.ones(n, dtype=np.int8)
    J[g.choice(n, size=12, replace=False)] = -1
    J[2] = 1
    J[7] = 1 if signs == "same" else -1
    ref = oracle.solve(G, J)
    for fused in (1, 0):
        out, launches = solve(G, J, cuda_dev, fused, block_w=20, precision="fp32_only")
        assert out["status"] == 0, (fused, out["info"])
        assert (launches["step_fused"] > 0) == bool(fused)
        compare(G, J, out, ref=ref, eps=EPS32)


def test_fused_step_batched(cuda_dev):
    from paper_1008_0201_gb300 import binding

    Gs, Js = small_batch(24, salt=31, pd_every=6)
    res = {}
    for fused in (1, 0):
        binding.jacobi_profile_begin(("step_fused",))
        try:
            outs, rc = run_batched(Gs, Js, cuda_dev, precision="fp32_only", fused_step=fused)
            n_fused = binding.jacobi_profile_read("step_fused")[1]
        finally:
            binding.jacobi_profile_end()
        assert rc == 0
        assert (n_fused > 0) == bool(fused), n_fused
        check_all(Gs, Js, outs, eps=EPS32)
        res[fused] = outs
    # same convergence decisions up to FP32 rounding of the Gram: equal sweep counts within one
    for a, b in zip(res[1], res[0]):
        assert abs(a["info"]["sweeps"] - b["info"]["sweeps"]) <= 1
