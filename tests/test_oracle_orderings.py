"""Pins of the oracle's block orderings (Sec. 2.4) by exhaustive enumeration (no GPU)."""
import itertools

import numpy as np
import pytest

import oracle

NBS = [2, 4, 6, 8, 10, 16, 32, 64]


def all_pairs(nb):
    return set(itertools.combinations(range(nb), 2))


def disjoint(step):
    idx = [int(x) for x in np.asarray(step).ravel()]
    return len(idx) == len(set(idx))


@pytest.mark.parametrize("nb", NBS)
def test_modulus_exact_cover(nb):
    seen = []
    for k in range(nb):
        st = oracle.pairs_modulus(nb, k)
        assert disjoint(st)
        assert all((p + q) % nb == k and p < q for p, q in st)
        expect = nb // 2 - (1 if (k % 2 == 0) else 0)
        assert len(st) == expect
        assert list(st[:, 0]) == sorted(st[:, 0])
        seen += [tuple(map(int, x)) for x in st]
    assert len(seen) == len(set(seen)) and set(seen) == all_pairs(nb)


@pytest.mark.parametrize("nb", NBS)
def test_modified_modulus(nb):
    seen = set()
    for k in range(nb):
        st = oracle.pairs_modulus(nb, k, modified=True)
        assert disjoint(st) and len(st) == nb // 2
        if k % 2 == 0:
            assert (k // 2, k // 2 + nb // 2) in [tuple(map(int, x)) for x in st]
        seen |= {tuple(map(int, x)) for x in st}
    assert seen == all_pairs(nb)


@pytest.mark.parametrize("nb", NBS)
def test_round_robin_matchings(nb):
    seen = []
    for s in range(nb - 1):
        st = oracle.pairs_round_robin(nb, s)
        assert len(st) == nb // 2 and disjoint(st)
        assert sorted(int(x) for x in st.ravel()) == list(range(nb))
        seen += [tuple(map(int, x)) for x in st]
    assert len(seen) == len(set(seen)) and set(seen) == all_pairs(nb)


@pytest.mark.parametrize("nb,seed", [(4, 0), (8, 1), (16, 2), (16, 3), (32, 4), (64, 5)])
def test_cycle_weight_greedy(nb, seed):
    g = np.random.default_rng(seed)
    W = g.random((nb, nb))
    if seed == 3:
        W = np.round(W * 4) / 4  # many ties
    steps = oracle.pairs_cycle_weight(nb, W)
    flat = [tuple(map(int, x)) for st in steps for x in st]
    assert len(flat) == len(set(flat)) and set(flat) == all_pairs(nb)
    assert all(disjoint(st) for st in steps)
    # greedy order: rank of every pair in the descending-weight order (ties: enumeration order)
    order = sorted(all_pairs(nb), key=lambda pq: (-W[pq[0], pq[1]], pq[0], pq[1]))
    rank = {pq: r for r, pq in enumerate(order)}
    assert max(rank[tuple(map(int, x))] for x in steps[0]) >= 0
    assert tuple(order[0]) in [tuple(map(int, x)) for x in steps[0]]
    done = set()
    for st in steps:
        taken = {tuple(map(int, x)) for x in st}
        used = set(int(v) for x in st for v in x)
        # maximality: every pending pair is blocked by a taken pair that precedes it
        for pq in all_pairs(nb) - done - taken:
            blockers = [t for t in taken if set(t) & set(pq)]
            assert blockers and min(rank[t] for t in blockers) < rank[pq]
        assert len(used) == 2 * len(st)
        done |= taken
    assert len(steps) <= 2 * nb - 3 or nb <= 2


def test_cycle_weight_all_equal_is_enumeration_greedy():
    nb = 6
    steps = oracle.pairs_cycle_weight(nb, np.ones((nb, nb)))
    assert [tuple(map(int, x)) for x in steps[0]] == [(0, 1), (2, 3), (4, 5)]


@pytest.mark.parametrize("n,nb", [(64, 8), (512, 16), (100, 8), (37, 8), (3, 2)])
def test_block_offsets(n, nb):
    off = oracle.block_offsets(n, nb)
    w = np.diff(off)
    assert off[0] == 0 and off[-1] == n and w.max() - w.min() <= 1 and w.min() >= 1
