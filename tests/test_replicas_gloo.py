"""The N > 1 path of bench.py on CPU: two gloo ranks (the method has no exchange step, so N GPUs
run independent replicas; the only collective is the max over ranks of the timings).

Checks the host logic that the GPU run relies on: every rank gets its own seeded input, the
slowest rank's time is taken, the whole-job value counts every rank's matrix, and the reference
arm prints from rank 0 only.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [40.0, 55.5][rank]
        slowest = bench.max_over_ranks(local_ms, dist, "cpu")
        G, J = bench.replica_input(rank, n=64)
        q.put((rank, slowest, bench.job_value(world, slowest), float(G[0, 0]), int(J.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0, v0, g0, j0), (r1, s1, v1, g1, j1) = res
    assert (r0, r1) == (0, 1)
    assert s0 == s1 == 55.5                      # max over ranks, seen by every rank
    assert v0 == v1 == pytest.approx(2 * 1000.0 / 55.5)
    assert g0 != g1                              # each replica draws its own matrix
    assert j0 == j1 == 64                        # J = I (positive definite) on every rank


def test_reference_arm_rank_nonzero_is_silent(capsys):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.reference_arm(Args, 1, 2) == 0
    assert capsys.readouterr().out == ""


def test_single_rank_helpers():
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 40.0) == 25.0
    G0, _ = bench.replica_input(0, n=32)
    G0b, _ = bench.replica_input(0, n=32)
    assert np.array_equal(G0, G0b)
    G2, J2 = bench.replica_input(1, workload="c2")
    assert G2.shape == (512, 512) and int(J2.sum()) == 0
