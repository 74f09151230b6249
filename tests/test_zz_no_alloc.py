"""jacobi_sched_pairs_noalloc: the scheduler entry point for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Its pair tables must equal those of
jacobi_sched_pairs, which allocates its scratch, on two calls in a row (the shared array keeps
the previous call's contents).  Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tables(steps):
    return [s.numpy().tolist() for s in steps]


def test_noalloc_matches_allocating_scheduler(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    for call in range(2):
        for nb, seed in ((16, 11), (64, 12), (256, 13)):
            g = np.random.default_rng(seed + 100 * call)
            W = torch.from_numpy(g.random((nb, nb)))
            ref = binding.jacobi_sched_pairs(nb, "cycle_weight", W, device=cuda_dev)
            got = binding.jacobi_sched_pairs(nb, "cycle_weight", W, device=cuda_dev, noalloc=True)
            assert _tables(got) == _tables(ref), (call, nb)
        for ordering in ("modulus", "modulus_mod", "round_robin"):
            ref = binding.jacobi_sched_pairs(20, ordering, device=cuda_dev)
            got = binding.jacobi_sched_pairs(20, ordering, device=cuda_dev, noalloc=True)
            assert _tables(got) == _tables(ref)


def test_noalloc_rejects_oversized_problems(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    lib = binding.load_library()
    nb = 258
    W = torch.rand((nb, nb), dtype=torch.float64, device=cuda_dev)
    pairs = torch.zeros(2 * nb * (nb // 2) * 2, dtype=torch.int32, device=cuda_dev)
    counts = torch.zeros(2 * nb, dtype=torch.int32, device=cuda_dev)
    ns = ctypes.c_int(-5)
    rc = lib.jacobi_sched_pairs_noalloc(nb, 3, ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(pairs.data_ptr()),
                                        ctypes.c_void_p(counts.data_ptr()), 2 * nb, ctypes.byref(ns),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and ns.value == -5


def _default_pool_used_high():
    """(reset, read) of the device's default memory pool high-water mark, which every
    cudaMallocAsync of the library draws from (driver API, through ctypes)."""
    lib = ctypes.CDLL("libcuda.so.1")
    pool = ctypes.c_void_p()
    assert lib.cuDeviceGetDefaultMemPool(ctypes.byref(pool), 0) == 0
    used_current, used_high = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def reset():
        zero = ctypes.c_uint64(0)
        assert lib.cuMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0

    def read():
        cur, high = ctypes.c_uint64(0), ctypes.c_uint64(0)
        assert lib.cuMemPoolGetAttribute(pool, used_current, ctypes.byref(cur)) == 0
        assert lib.cuMemPoolGetAttribute(pool, used_high, ctypes.byref(high)) == 0
        return cur.value, high.value

    return reset, read


def test_noalloc_draws_nothing_from_the_pool(cuda_dev):
    """The allocating scheduler raises the pool's high-water mark; the noalloc one does not."""
    import torch

    from paper_1008_0201_gb300 import binding

    reset, read = _default_pool_used_high()
    nb = 128
    W = torch.from_numpy(np.random.default_rng(5).random((nb, nb)))
    binding.jacobi_sched_pairs(nb, "cycle_weight", W, device=cuda_dev, noalloc=True)  # first call: set-up
    torch.cuda.synchronize()
    cur0, _ = read()
    reset()
    for _ in range(2):
        binding.jacobi_sched_pairs(nb, "cycle_weight", W, device=cuda_dev, noalloc=True)
    torch.cuda.synchronize()
    cur1, high1 = read()
    assert high1 == cur0 and cur1 == cur0, (cur0, cur1, high1)
    reset()
    binding.jacobi_sched_pairs(nb, "cycle_weight", W, device=cuda_dev)  # allocates its scratch
    torch.cuda.synchronize()
    _, high2 = read()
    assert high2 > cur0, (cur0, high2)
