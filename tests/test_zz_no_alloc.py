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
