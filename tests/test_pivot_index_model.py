"""Models of the pivot kernel's index arithmetic, checked on the CPU.

- The Cholesky (one row of R~ - I per step): each column c is owned by TPC = NT / KM lanes of one
  warp (lane = t CPW + c mod CPW), whose partial sums over the rows l = t mod TPC the shuffles at
  offsets CPW, 2 CPW, ... combine; the rows of a column's lanes partition 0..KM-1; with a row
  stride of LDC = KM + 8 floats a warp's loads of its own columns hit 32 distinct banks and its
  loads of the pivot column hit distinct banks per distinct address; the KM rows fit in the
  mailboxes they borrow.
- The fused step kernel: the staged rows of X_P and the FP32 V_P fit in the digit-product region
  (m <= 96 rows for KM = 32, 192 for KM = 64); its Gram and update thread maps cover the KM x KM
  tile and the 64-row chunks x KM columns exactly once; a 64-row chunk of V fits in the mailboxes.
- The mailbox of the inner sweep stores row l R + u of a column at u LPP + l; with a slot stride of
  MBS = 2 KM + 8 floats, the four slots of a warp (8 lanes each) write and read distinct banks for
  every u, and the layout stays inside the slot's F and W halves.
"""
import numpy as np
import pytest

LPP = 8
OZ_T = 8


def geometry(KM):
    NT = (KM // 2) * LPP
    return dict(NT=NT, P2=KM // 2, MBS=2 * KM + 8, LDC=KM + 8, LDV=KM + 1, LDD=KM + 8)


@pytest.mark.parametrize("KM", [32, 64])
def test_cholesky_lane_map(KM):
    g = geometry(KM)
    NT, LDC = g["NT"], g["LDC"]
    TPC = NT // KM
    CPW = 32 // TPC
    NU = KM // TPC
    assert TPC * KM == NT and CPW * TPC == 32 and NU % 4 == 0
    owners = {}
    for tid in range(NT):
        warp, lane = divmod(tid, 32)
        ct, cc = lane // CPW, warp * CPW + lane % CPW
        owners.setdefault(cc, []).append((warp, lane, ct))
    assert sorted(owners) == list(range(KM))
    offsets = [CPW << i for i in range(TPC.bit_length() - 1)]
    for cc, own in owners.items():
        assert len(own) == TPC and len({w for w, _, _ in own}) == 1  # one warp per column
        lanes = {l for _, l, _ in own}
        # the xor butterfly over the offsets reaches exactly the column's lanes from any of them
        for _, l0, _ in own:
            reach = {l0}
            for o in offsets:
                reach |= {x ^ o for x in reach}
            assert reach == lanes
        rows = sorted(ct + TPC * u for _, _, ct in own for u in range(NU))
        assert rows == list(range(KM))
    # banks of one load instruction (fixed u) of a warp
    for warp in range(NT // 32):
        for u in range(NU):
            own_col = [((lane // CPW + TPC * u) * LDC + warp * CPW + lane % CPW) % 32 for lane in range(32)]
            assert len(set(own_col)) == 32
            for p in (0, 7, KM - 1):
                addr = [(lane // CPW + TPC * u) * LDC + p for lane in range(32)]
                banks = {}
                for a in addr:
                    banks.setdefault(a % 32, set()).add(a)
                assert all(len(v) == 1 for v in banks.values())
    assert 2 * g["P2"] * g["MBS"] >= KM * LDC  # the rows borrow the mailboxes


@pytest.mark.parametrize("KM,MF", [(32, 96), (64, 192)])
def test_fused_step_layout(KM, MF):
    g = geometry(KM)
    NT = g["NT"]
    region = max(KM * g["LDV"] * 8, OZ_T * KM * g["LDD"] * 2) // 4  # floats of the M / D union
    LDX = LDB = KM + 4
    assert ((region - KM * LDB) // LDX) // 32 * 32 == MF  # the row limit the header states
    assert MF * LDX + KM * LDB <= region
    # update reads of a chunk starting at r0 < m <= MF reach row r0 + 63 of Xs: still inside the region
    last_r0 = ((MF - 1) // 64) * 64
    assert (last_r0 + 63) * LDX + KM <= region
    assert (LDX * 4) % 16 == 0 and (LDB * 4) % 16 == 0  # float4 rows
    assert 2 * g["P2"] * g["MBS"] >= 64 * LDX  # a 64-row chunk of V in the mailboxes
    CT = KM // 4
    assert NT // CT == 16
    RPT = KM // 16
    gram = sorted((RPT * (t // CT) + u, 4 * (t % CT) + v) for t in range(NT) for u in range(RPT) for v in range(4))
    assert gram == [(i, j) for i in range(KM) for j in range(KM)]
    upd = sorted((4 * (t // CT) + u, 4 * (t % CT) + v) for t in range(NT) for u in range(4) for v in range(4))
    assert upd == [(r, j) for r in range(64) for j in range(KM)]
    # staging loads: element e < k m is (row e mod m, column e / m), every entry once, any k, m
    for k, m in ((KM, MF), (KM - 3, MF - 16), (5, 16)):
        seen = sorted((e % m, e // m) for e in range(k * m))
        assert seen == sorted((r, c) for c in range(k) for r in range(m))


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
