"""Device scheduler against the oracle's orderings, bit for bit (-m gpu, through the C ABI).

The pair tables of one cycle (Sec. 2.4: modulus, modified modulus, round-robin; per-cycle
largest-weight greedy ordering, a build extension) are integer index work, so the device
tables must EQUAL the oracle's: the same steps in the same order, each with the same pairs.
The static orderings must also agree slot by slot (both list a step's pairs by increasing p);
for the weight ordering the oracle lists a step's pairs in the order the greedy scan took them
and the device by increasing p, so its steps are compared as sorted pair lists.  Weight matrices
include many ties (few distinct values), where only the stated tie rule (enumeration order)
makes the table unique.  Non-finite weights (NaN, +inf, -inf) are ranked by the documented
total order (NaN last), which the oracle reproduces on the same weights with NaN replaced by
-inf; every table must also cover each pair exactly once in disjoint steps.
"""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

NBS = (2, 4, 8, 16, 64, 256)


def _dev_tables(nb, ordering, W=None, noalloc=False, dev="cuda:0"):
    import torch

    from paper_1008_0201_gb300 import binding

    w = torch.from_numpy(np.ascontiguousarray(W)) if W is not None else None
    steps = binding.jacobi_sched_pairs(nb, ordering, w, device=dev, noalloc=noalloc)
    return [s.numpy().astype(np.int32) for s in steps]


def _oracle_tables(nb, ordering, W=None):
    if ordering == "modulus":
        return [oracle.pairs_modulus(nb, k) for k in range(nb)]
    if ordering == "modulus_mod":
        return [oracle.pairs_modulus(nb, k, modified=True) for k in range(nb)]
    if ordering == "round_robin":
        return [oracle.pairs_round_robin(nb, s) for s in range(nb - 1)]
    return oracle.pairs_cycle_weight(nb, W)


def _by_p(t):
    return t[np.lexsort((t[:, 1], t[:, 0]))] if len(t) else t


def _assert_equal(got, ref, tag, sort_steps=False):
    assert len(got) == len(ref), (tag, len(got), len(ref))
    for s, (a, b) in enumerate(zip(got, ref)):
        if sort_steps:
            assert np.array_equal(a, _by_p(a)), (tag, s, "device step not listed by p")
            b = _by_p(b)
        assert a.shape == b.shape and np.array_equal(a, b), (tag, s, a.tolist(), b.tolist())


def _assert_cover(tables, nb, tag):
    seen = np.zeros((nb, nb), dtype=np.int64)
    for s, t in enumerate(tables):
        blocks = t.reshape(-1)
        assert len(np.unique(blocks)) == len(blocks), (tag, "step not disjoint", s)
        for p, q in t:
            assert 0 <= p < q < nb, (tag, s, p, q)
            seen[p, q] += 1
    iu = np.triu_indices(nb, 1)
    assert np.all(seen[iu] == 1), (tag, "pair not covered exactly once")


@pytest.mark.parametrize("ordering", ["modulus", "modulus_mod", "round_robin"])
@pytest.mark.parametrize("nb", NBS)
def test_static_orderings_equal_oracle(cuda_dev, ordering, nb):
    _assert_equal(_dev_tables(nb, ordering), _oracle_tables(nb, ordering), (ordering, nb))


def _weights(nb, seed, levels):
    g = np.random.default_rng(seed)
    W = g.integers(0, levels, size=(nb, nb)).astype(np.float64) / levels  # ties everywhere
    return W


@pytest.mark.parametrize("nb", NBS)
@pytest.mark.parametrize("levels", [3, 1000])
def test_cycle_weight_equals_oracle(cuda_dev, nb, levels):
    W = _weights(nb, 500 + nb + levels, levels)
    ref = _oracle_tables(nb, "cycle_weight", W)
    for noalloc in (False, True):
        got = _dev_tables(nb, "cycle_weight", W, noalloc=noalloc)
        _assert_equal(got, ref, ("cycle_weight", nb, levels, noalloc), sort_steps=True)
    _assert_cover(ref, nb, "oracle")


def test_cycle_weight_all_equal_and_max_nb(cuda_dev):
    # all weights equal: the enumeration order alone decides; nb = 512 is the largest accepted
    for nb in (32, 512):
        W = np.full((nb, nb), 0.25)
        got = _dev_tables(nb, "cycle_weight", W)
        _assert_equal(got, _oracle_tables(nb, "cycle_weight", W), ("equal", nb), sort_steps=True)


@pytest.mark.parametrize("noalloc", [False, True])
def test_cycle_weight_non_finite(cuda_dev, noalloc):
    nb = 16
    W = _weights(nb, 77, 10)
    W[0, 5] = np.nan
    W[2, 3] = np.inf
    W[1, 9] = -np.inf
    W[4, 7] = np.nan
    got = _dev_tables(nb, "cycle_weight", W, noalloc=noalloc)
    _assert_cover(got, nb, "non-finite")
    W2 = np.where(np.isnan(W), -np.inf, W)
    _assert_equal(got, _oracle_tables(nb, "cycle_weight", W2), "non-finite vs oracle", sort_steps=True)
