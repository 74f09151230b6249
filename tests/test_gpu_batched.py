"""Batched entry point (jacobi_eig_batched) vs the CPU oracle, problem by problem.

The inputs follow the batched workload (orders uniform in [8, 128], Gaussian G, a random 30% of
the signs -1), in small batches the oracle finishes in seconds; every problem of a batch is held
to the single-solve tolerances (FP64) or to the same bounds at eps = 2^-24 (FP32-only sweeps).
"""
import numpy as np
import pytest

from checks import EPS32, compare, to_np

pytestmark = pytest.mark.gpu


def run_batched(Gs, Js, dev, want_u=True, raise_on_error=False, **kw):
    import torch

    from paper_1008_0201_gb300 import binding

    opts = binding.default_opts(**kw)
    Gd = [torch.from_numpy(np.ascontiguousarray(G)).to(dev) for G in Gs]
    Jd = None if Js is None else [None if J is None else torch.from_numpy(J).to(dev) for J in Js]
    outs, rc = binding.jacobi_eig_batched(Gd, Jd, opts, want_u=want_u, raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    return [to_np(o) for o in outs], rc


def small_batch(count, salt, lo=8, hi=128, pd_every=0):
    from paper_1008_0201_gb300 import inputs

    Gs, Js = inputs.config4_batched(count=count, lo=lo, hi=hi, salt=salt)
    if pd_every:
        Js = [None if i % pd_every == 0 else J for i, J in enumerate(Js)]
    return Gs, Js


def check_all(Gs, Js, outs, eps=None):
    for i, (G, J, o) in enumerate(zip(Gs, Js, outs)):
        assert o["info"]["status"] == 0, (i, G.shape, o["info"])
        Jf = np.ones(G.shape[1], dtype=np.int8) if J is None else J
        if eps is None:
            compare(G, Jf, o)
        else:
            compare(G, Jf, o, eps=eps)


@pytest.mark.parametrize("ordering", ["round_robin", "modulus", "modulus_mod"])
def test_batched_fp64_uneven_orders(cuda_dev, ordering):
    Gs, Js = small_batch(20, salt=11, pd_every=4)
    outs, rc = run_batched(Gs, Js, cuda_dev, ordering=ordering)
    assert rc == 0
    check_all(Gs, Js, outs)


@pytest.mark.parametrize("factor", ["chol", "chol_signpiv"])
def test_batched_fp32_only(cuda_dev, factor):
    Gs, Js = small_batch(20, salt=12, pd_every=5)
    outs, rc = run_batched(Gs, Js, cuda_dev, precision="fp32_only", factor=factor)
    assert rc == 0
    check_all(Gs, Js, outs, eps=EPS32)


def test_batched_size_class_edges(cuda_dev):
    """Orders at the class boundaries (one pivot block up to 64 columns, 32-wide blocks above),
    tall factors (m > n) and the smallest problems."""
    g = np.random.default_rng(77)
    shapes = [(8, 8), (9, 2), (31, 31), (32, 32), (33, 33), (40, 33), (64, 64), (65, 65), (96, 97 - 1),
              (128, 128), (130, 127), (5, 3), (2, 2), (70, 1)]
    Gs, Js = [], []
    for i, (m, n) in enumerate(shapes):
        Gs.append(g.standard_normal((m, n)))
        J = np.ones(n, dtype=np.int8)
        J[g.choice(n, size=int(round(0.3 * n)), replace=False)] = -1
        Js.append(J if i % 3 else None)
    outs, rc = run_batched(Gs, Js, cuda_dev)
    assert rc == 0
    check_all(Gs, Js, outs)
    # a single column needs no sweep
    assert outs[-1]["info"]["sweeps"] == 0


def test_batched_composition_independent(cuda_dev):
    """A problem's result does not depend on the rest of the batch (bit for bit), nor on
    repetition."""
    Gs, Js = small_batch(12, salt=13)
    full, rc = run_batched(Gs, Js, cuda_dev)
    assert rc == 0
    again, _ = run_batched(Gs, Js, cuda_dev)
    for a, b in zip(full, again):
        assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["V"], b["V"])
    for i in (0, 5, 11):
        alone, rc1 = run_batched([Gs[i]], [Js[i]], cuda_dev)
        assert rc1 == 0
        assert np.array_equal(alone[0]["lam"], full[i]["lam"])
        assert np.array_equal(alone[0]["G"], full[i]["G"])
        assert np.array_equal(alone[0]["V"], full[i]["V"])


def test_batched_failures_are_per_problem(cuda_dev):
    """A non-finite input, a sign other than +-1 and a rank-deficient indefinite factor fail
    their own problem only; the other problems are solved to the usual tolerances."""
    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(91)
    Gs = [g.standard_normal((n, n)) for n in (20, 24, 40, 16, 70)]
    Js = [np.where(g.random(G.shape[1]) < 0.3, -1, 1).astype(np.int8) for G in Gs]
    Gs[1][3, 5] = np.inf                       # non-finite
    Js[2] = Js[2].copy()
    Js[2][4] = 0                               # invalid sign
    Gs[3][:, 7] = Gs[3][:, 2]                  # duplicate column in one pivot block: A_P singular
    Js[3][2], Js[3][7] = 1, -1
    G1_before = Gs[1].copy()
    outs, rc = run_batched(Gs, Js, cuda_dev)
    st = [o["info"]["status"] for o in outs]
    assert st[1] == binding.JAC_ENONFINITE
    assert st[2] == -7
    assert st[3] == binding.JAC_ENOTPD
    assert rc == binding.JAC_ENONFINITE        # first failing problem in input order
    for i in (0, 4):
        assert st[i] == 0
        compare(Gs[i], Js[i], outs[i])
    # a problem that failed validation keeps its input
    assert np.array_equal(np.nan_to_num(outs[1]["G"], posinf=1e300), np.nan_to_num(G1_before, posinf=1e300))


def test_batched_argument_errors(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    G = torch.randn(20, 20, dtype=torch.float64, device=cuda_dev)
    with pytest.raises(binding.JacobiError) as e:
        binding.jacobi_eig_batched([G], None, binding.default_opts(ordering="cycle_weight"))
    assert e.value.code == -8
    with pytest.raises(binding.JacobiError) as e:
        binding.jacobi_eig_batched([G], None, binding.default_opts(precision="fp32"))
    assert e.value.code == -8
    wide = torch.randn(10, 12, dtype=torch.float64, device=cuda_dev)  # n > m
    with pytest.raises(binding.JacobiError) as e:
        binding.jacobi_eig_batched([G, wide], None, binding.default_opts())
    assert e.value.code == -3
    outs, rc = binding.jacobi_eig_batched([], None, binding.default_opts())
    assert outs == [] and rc == 0


def test_batched_full_size_sampled(cuda_dev):
    """The batched workload at full size (10 000 problems of order 8..128, FP64): every problem
    converges, and 24 sampled problems match the oracle to the single-solve tolerances."""
    import torch

    from paper_1008_0201_gb300 import binding, inputs

    Gs, Js = inputs.config4_batched()
    ns = np.array([G.shape[1] for G in Gs], dtype=np.int32)
    offs = np.concatenate([[0], np.cumsum(ns.astype(np.int64) ** 2)])
    joffs = np.concatenate([[0], np.cumsum(ns.astype(np.int64))])
    Gw = torch.from_numpy(np.concatenate([np.asfortranarray(G).ravel(order="F") for G in Gs])).to(cuda_dev)
    Jd = torch.from_numpy(np.concatenate(Js).astype(np.int8)).to(cuda_dev)
    lam = torch.empty(int(joffs[-1]), dtype=torch.float64, device=cuda_dev)
    V = torch.empty(int(offs[-1]), dtype=torch.float64, device=cuda_dev)
    ptr = lambda t, o, es: (np.uint64(t.data_ptr()) + o[:-1].astype(np.uint64) * np.uint64(es)).astype(np.uint64)
    rc, infos = binding.jacobi_eig_batched_raw(ns, ns, ptr(Gw, offs, 8), ns, ptr(Jd, joffs, 1),
                                               binding.default_opts(precision="fp64"), ptr(lam, joffs, 8), None,
                                               None, ptr(V, offs, 8), ns, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0
    assert all(infos[i].status == 0 for i in range(len(Gs)))
    lam_h, G_h, V_h = lam.cpu().numpy(), Gw.cpu().numpy(), V.cpu().numpy()
    for i in np.random.default_rng(4).choice(len(Gs), size=24, replace=False):
        n = int(ns[i])
        out = dict(lam=lam_h[joffs[i]:joffs[i + 1]], G=G_h[offs[i]:offs[i + 1]].reshape((n, n), order="F"),
                   V=V_h[offs[i]:offs[i + 1]].reshape((n, n), order="F"), U=None)
        compare(Gs[i], Js[i], out)


def test_batched_autotune(cuda_dev):
    """The width autotuner installs one measured rule per size class; batches solved under the
    tuned widths still match the oracle; count = 0 restores the defaults."""
    from paper_1008_0201_gb300 import binding

    rules = binding.jacobi_autotune_batched(count=48, precision="fp64", device=cuda_dev)
    try:
        for lo, hi, allowed in ((8, 16, {0, 8}), (17, 32, {0, 8}), (33, 48, {0, 16, 8}), (49, 64, {0, 16, 32}),
                                (65, 96, {32, 16}), (97, 128, {32, 16})):
            assert len(set(rules[lo:hi + 1])) == 1 and rules[lo] in allowed, (lo, hi, rules[lo:hi + 1])
        assert np.all(rules[:8] == -1)
        Gs, Js = small_batch(16, salt=21)
        outs, rc = run_batched(Gs, Js, cuda_dev)
        assert rc == 0
        check_all(Gs, Js, outs)
    finally:
        reset = binding.jacobi_autotune_batched(count=0, device=cuda_dev)
    assert np.all(reset == -1)
