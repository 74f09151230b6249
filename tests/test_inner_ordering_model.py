"""Model of the pivot kernel's inner ordering (the recursive cross ordering of the KM positions
of a pivot block), restated from the kernel's slot arithmetic, checked for exact cover.

Slot q holds a resident (initially position q) and a traveler (position q + KM/2).  At group
size g = KM/2, KM/4, ..., 1 the travelers of each group of g slots go round the group's ring;
after the ring each group splits: the slots of the second half send their residents to the first
half (which receive them as travelers), and the first half sends its travelers to the second half
(received as residents).  Every step rotates the pair held in each slot, and between steps every
slot passes exactly one column on.  The cyclic inner sweep of Sec. 2 needs each pair of positions
exactly once per sweep; the block-oriented steps after the first of a sweep run only the first
ring level, which must pair every resident with every traveler exactly once.
"""
import itertools

import pytest


def inner_sweep_pairs(KM, cross_only=False):
    P2 = KM // 2
    res = list(range(P2))
    trav = [q + P2 for q in range(P2)]
    met = []
    g_last = P2 if cross_only else 1
    g = P2
    while g >= g_last:
        for st in range(g):
            met.extend(tuple(sorted((res[q], trav[q]))) for q in range(P2))
            if st < g - 1 or g > g_last:
                ring = st < g - 1
                out, dst, give = {}, {}, {}
                for q in range(P2):
                    base, pos = q & ~(g - 1), q - (q & ~(g - 1))
                    give[q] = (not ring) and pos >= g // 2
                    d = base + ((pos + 1) & (g - 1)) if ring else (q + g // 2 if pos < g // 2 else q - g // 2)
                    dst[q] = d
                    out[q] = res[q] if give[q] else trav[q]
                incoming = {}
                for q in range(P2):
                    assert dst[q] not in incoming, "two columns sent to one slot"
                    incoming[dst[q]] = out[q]
                assert sorted(incoming) == list(range(P2)), "a slot receives nothing"
                for q in range(P2):
                    if give[q]:
                        res[q] = incoming[q]
                    else:
                        trav[q] = incoming[q]
        g //= 2
    return met


@pytest.mark.parametrize("KM", [2, 4, 8, 16, 32, 64])
def test_full_inner_sweep_is_an_exact_cover(KM):
    met = inner_sweep_pairs(KM)
    assert len(met) == KM * (KM - 1) // 2  # KM - 1 steps of KM/2 pairs
    assert sorted(met) == sorted(itertools.combinations(range(KM), 2))


@pytest.mark.parametrize("KM", [2, 4, 8, 16, 32, 64])
def test_cross_level_pairs_every_resident_with_every_traveler(KM):
    P2 = KM // 2
    met = inner_sweep_pairs(KM, cross_only=True)
    assert sorted(met) == sorted((a, b) for a in range(P2) for b in range(P2, KM))
