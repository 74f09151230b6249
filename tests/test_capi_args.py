"""Argument validation of every C entry point, on the CPU.

Each case breaks one argument of an otherwise valid call and checks the documented return code
(the negative position of the first invalid argument).  All of these return before any CUDA
call, so they run without a GPU.  Device pointers are stand-in addresses that the validation
never dereferences; host arrays (the batched entry's per-problem arrays) are real.
"""
import ctypes

import pytest

FAKE = ctypes.c_void_p(0x100000)  # a non-NULL "device" address, never dereferenced here
FAKE2 = ctypes.c_void_p(0x200000)


@pytest.fixture(scope="module")
def lib(lib_built):
    from paper_1008_0201_gb300 import binding

    return binding.load_library()


def _opts(**kw):
    from paper_1008_0201_gb300 import binding

    o = binding.default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _hsvd(lib, m=4, n=3, dtype=0, G=FAKE, ldg=4, J=FAKE, opts=None, lam=FAKE, U=None, ldu=0, V=FAKE, ldv=3):
    o = opts if opts is not None else _opts()
    return lib.jacobi_hsvd(m, n, dtype, G, ldg, J, ctypes.byref(o), lam, U, ldu, V, ldv, None, None)


@pytest.mark.parametrize("dtype", [0, 1])
def test_hsvd_argument_positions(lib, dtype):
    assert _hsvd(lib, dtype=dtype, m=0) == -1
    assert _hsvd(lib, dtype=dtype, n=5) == -2
    assert _hsvd(lib, dtype=dtype, n=0) == -2
    assert _hsvd(lib, dtype=dtype, G=None) == -4
    assert _hsvd(lib, dtype=dtype, ldg=3) == -5
    assert _hsvd(lib, dtype=dtype, J=None) == -6
    for bad in (dict(block_w=0), dict(block_w=33), dict(ordering=4), dict(block_mode=2), dict(factor=3),
                dict(precision=3), dict(max_sweeps=0), dict(want_v=2), dict(f64_products=3),
                dict(f64_products=-1), dict(fused_step=2), dict(fused_step=-1)):
        assert _hsvd(lib, dtype=dtype, opts=_opts(**bad)) == -7, bad
    assert _hsvd(lib, dtype=dtype, lam=None) == -8
    assert _hsvd(lib, dtype=dtype, U=FAKE2, ldu=3) == -10
    assert _hsvd(lib, dtype=dtype, U=FAKE, ldu=4) == -9  # U aliasing G
    assert _hsvd(lib, dtype=dtype, V=None) == -11
    assert _hsvd(lib, dtype=dtype, ldv=2) == -12


def test_hsvd_bad_dtype(lib):
    assert _hsvd(lib, dtype=7) == -3


def test_eig_pd_argument_positions(lib):
    def call(m=4, n=3, G=FAKE, ldg=4, opts=None, lam=FAKE, U=None, ldu=0, V=FAKE, ldv=3):
        o = opts if opts is not None else _opts()
        return lib.jacobi_eig_pd(m, n, 0, G, ldg, ctypes.byref(o), lam, U, ldu, V, ldv, None, None)

    assert call(m=0) == -1
    assert call(n=5) == -2
    assert call(G=None) == -4
    assert call(ldg=3) == -5
    assert call(opts=_opts(factor=9)) == -6
    assert call(lam=None) == -7
    assert call(U=FAKE, ldu=4) == -8
    assert call(U=FAKE2, ldu=3) == -9
    assert call(V=None) == -10
    assert call(ldv=2) == -11


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


def _batched(lib, batch=2, m=(5, 4), n=(3, 4), dtype=0, G=(0x100000, 0x200000), ldg=(5, 4), J=None, opts=None,
             lam=(0x300000, 0x400000), U=None, ldu=None, V=(0x500000, 0x600000), ldv=(3, 4), drop=()):
    P = ctypes.c_void_p
    args = {
        "m": None if "m" in drop else _arr(ctypes.c_int, m),
        "n": None if "n" in drop else _arr(ctypes.c_int, n),
        "G": None if "G" in drop else _arr(P, G),
        "ldg": None if "ldg" in drop else _arr(ctypes.c_int, ldg),
        "lam": None if "lam" in drop else _arr(P, lam),
        "U": None if U is None else _arr(P, U),
        "ldu": None if ldu is None else _arr(ctypes.c_int, ldu),
        "V": None if (V is None or "V" in drop) else _arr(P, V),
        "ldv": None if "ldv" in drop else _arr(ctypes.c_int, ldv),
    }
    o = opts if opts is not None else _opts()
    return lib.jacobi_eig_batched(batch, args["m"], args["n"], dtype, args["G"], args["ldg"], J, ctypes.byref(o),
                                  args["lam"], args["U"], args["ldu"], args["V"], args["ldv"], None, None)


def test_batched_argument_positions(lib):
    assert _batched(lib, batch=-1) == -1
    assert _batched(lib, batch=0) == 0  # nothing to do, no CUDA call
    assert _batched(lib, drop=("m",)) == -2
    assert _batched(lib, drop=("n",)) == -3
    assert _batched(lib, dtype=1) == -4
    assert _batched(lib, drop=("G",)) == -5
    assert _batched(lib, drop=("ldg",)) == -6
    assert _batched(lib, opts=_opts(ordering=3)) == -8  # per-cycle weight ordering: single solves only
    assert _batched(lib, opts=_opts(precision=1)) == -8  # the mixed mode: single solves only
    assert _batched(lib, opts=_opts(f64_products=3)) == -8
    assert _batched(lib, opts=_opts(fused_step=2)) == -8
    assert _batched(lib, drop=("lam",)) == -9
    assert _batched(lib, U=(0x700000, 0x800000)) == -11  # U without ldu
    assert _batched(lib, drop=("V",)) == -12
    assert _batched(lib, drop=("ldv",)) == -13
    # per problem
    assert _batched(lib, m=(5, 0)) == -2
    assert _batched(lib, n=(3, 5)) == -3
    assert _batched(lib, G=(0x100000, 0)) == -5
    assert _batched(lib, ldg=(5, 3)) == -6
    assert _batched(lib, lam=(0x300000, 0)) == -9
    assert _batched(lib, U=(0x700000, 0x800000), ldu=(5, 3)) == -11
    assert _batched(lib, U=(0x700000, 0x200000), ldu=(5, 4)) == -10  # U[1] aliasing G[1]
    assert _batched(lib, V=(0x500000, 0)) == -12
    assert _batched(lib, ldv=(3, 3)) == -13


def test_backward_argument_positions(lib):
    def call(batch=2, n=4, lam=FAKE, s_lam=4, U=FAKE, ldu=4, s_u=16, lb=FAKE, s_lb=4, Ub=FAKE, ldub=4, s_ub=16,
             deg=1e-12, H=FAKE2, ldh=4, s_h=16, G=FAKE, ldg=4, s_g=16, J=FAKE, s_j=4, Gb=FAKE2, ldgb=4, s_gb=16):
        return lib.jacobi_eig_backward(batch, n, lam, s_lam, U, ldu, s_u, lb, s_lb, Ub, ldub, s_ub, deg, H, ldh,
                                       s_h, G, ldg, s_g, J, s_j, Gb, ldgb, s_gb, None)

    assert call(batch=-1) == -1
    assert call(n=0) == -2
    assert call(lam=None) == -3
    assert call(s_lam=3) == -4
    assert call(U=None) == -5
    assert call(ldu=3) == -6
    assert call(s_u=15) == -7
    assert call(s_lb=3) == -9
    assert call(ldub=3) == -11
    assert call(s_ub=15) == -12
    assert call(deg=-1.0) == -13
    assert call(deg=float("nan")) == -13
    assert call(H=None) == -14
    assert call(ldh=3) == -15
    assert call(s_h=15) == -16
    assert call(G=None) == -17
    assert call(ldg=3) == -18
    assert call(s_g=15) == -19
    assert call(s_j=3) == -21
    assert call(ldgb=3) == -23
    assert call(s_gb=15) == -24
    assert call(batch=0) == 0  # nothing to do, no CUDA call


@pytest.mark.parametrize("noalloc", [False, True])
def test_sched_pairs_argument_positions(lib, noalloc):
    fn = lib.jacobi_sched_pairs_noalloc if noalloc else lib.jacobi_sched_pairs
    ns = ctypes.c_int(-5)

    def call(nb=16, ordering=3, w=FAKE, pairs=FAKE, counts=FAKE2, max_steps=32, nsteps=True):
        return fn(nb, ordering, w, pairs, counts, max_steps, ctypes.byref(ns) if nsteps else None, None)

    assert call(nb=0) == -1
    assert call(nb=1) == -1
    assert call(nb=15) == -1  # odd
    assert call(ordering=-1) == -2
    assert call(ordering=4) == -2
    assert call(w=None) == -3  # the weight ordering needs weights
    assert call(pairs=None) == -4
    assert call(counts=None) == -5
    assert call(max_steps=0) == -6
    assert call(ordering=2, max_steps=14) == -6  # round-robin needs nb - 1 steps
    assert call(ordering=0, max_steps=15) == -6  # modulus needs nb steps
    assert call(nsteps=False) == -7
    # block-count limits: 256 for the allocation-free entry point (its fixed scratch),
    # JAC_CYCLE_WEIGHT_MAX_NB = 512 for the weight ordering, 4096 otherwise
    if noalloc:
        assert call(nb=258) == -1
        assert call(nb=258, ordering=2, max_steps=257) == -1
    else:
        assert call(nb=514) == -1
        assert call(nb=4098, ordering=2, max_steps=4097) == -1
    assert ns.value == -5  # nothing written on an argument error


def test_cycle_weight_block_cap(lib):
    # n = 1100 with w = 1 gives nb = 1100 > 512 blocks: rejected as an invalid opts argument,
    # real (argument 7) and complex (the real problem of order 2n; argument 7)
    o = _opts(ordering=3, block_w=1)
    assert _hsvd(lib, m=1100, n=1100, ldg=1100, ldv=1100, opts=o) == -7
    assert _hsvd(lib, m=300, n=300, ldg=300, ldv=300, dtype=1, opts=o) == -7
    assert lib.jacobi_eig_pd(1100, 1100, 0, FAKE, 1100, ctypes.byref(o), FAKE, None, 0, FAKE2, 1100, None,
                             None) == -6
