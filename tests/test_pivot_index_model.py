"""Models of the pivot kernel's index arithmetic, checked on the CPU.

- The Cholesky's strictly upper entries (r, c), r < c < KM, are enumerated e = c (c - 1) / 2 + r
  and recovered from e with an FP32 square-root estimate plus integer correction; every entry must
  be recovered exactly once for KM = 32 and 64.
- The mailbox of the inner sweep stores row l R + u of a column at u LPP + l; with a slot stride of
  MBS = 2 KM + 8 floats, the four slots of a warp (8 lanes each) write and read distinct banks for
  every u, and the layout stays inside the slot's F and W halves.
"""
import numpy as np
import pytest


def recover(e):
    c = int(np.float32((np.float32(1.0) + np.sqrt(np.float32(1.0) + np.float32(8.0) * np.float32(e))) * np.float32(0.5)))
    while c * (c - 1) // 2 > e:
        c -= 1
    while (c + 1) * c // 2 <= e:
        c += 1
    return c, e - c * (c - 1) // 2


@pytest.mark.parametrize("KM", [32, 64])
def test_upper_entry_enumeration(KM):
    npair = KM * (KM - 1) // 2
    got = [recover(e) for e in range(npair)]
    assert sorted(got) == sorted((r, c)[::-1] for c in range(KM) for r in range(c))
    assert all(r < c < KM for c, r in got)


@pytest.mark.parametrize("KM", [32, 64])
def test_mailbox_layout_banks(KM):
    LPP = 8
    R, MBS = KM // LPP, 2 * KM + 8
    for base_slot in range(0, KM // 2, 4):  # the 4 slots of one warp
        for u in range(R):
            for half in (0, KM):  # F part, W part
                addr = [(base_slot + s) * MBS + half + u * LPP + l for s in range(4) for l in range(LPP)]
                assert len({a % 32 for a in addr}) == 32  # one wavefront per access
    # every (lane, u) position of a slot is distinct and inside its F half
    pos = sorted(u * LPP + l for u in range(R) for l in range(LPP))
    assert pos == list(range(KM))


@pytest.mark.parametrize("KM", [32, 64])
def test_mailbox_writes_of_every_step_hit_distinct_banks(KM):
    """The slots a warp's four slots send to, at every ring and split step, are distinct mod 4,
    which with MBS = 8 (mod 32) puts their 32-byte rows on distinct banks."""
    P2 = KM // 2
    assert (2 * KM + 8) % 32 == 8
    g = P2
    while g >= 1:
        for st in range(g):
            if not (st < g - 1 or g > 1):
                continue
            ring = st < g - 1
            for w0 in range(0, P2, 4):
                dsts = []
                for q in range(w0, w0 + 4):
                    base, pos = q & ~(g - 1), q - (q & ~(g - 1))
                    dsts.append(base + ((pos + 1) & (g - 1)) if ring else (q + g // 2 if pos < g // 2 else q - g // 2))
                assert len({d % 4 for d in dsts}) == 4, (g, st, dsts)
        g //= 2
