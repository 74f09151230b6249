"""Shared-memory addressing of the digit-product kernels (csrc/ozaki.cu, the V_P residual of
csrc/pivot.cu), restated from the kernels' index arithmetic and checked on the CPU: every
ldmatrix row address lies inside its digit array, is 16-byte aligned, and the 8 rows of each
8 x 8 matrix fall on distinct 16-byte bank groups (one wavefront per matrix).
"""
import pytest

T = 8  # digits


def ldsm_rows_A(ti, kk, lanes=range(32)):
    """x4 A fragment: lane -> (row, k offset)."""
    return [(16 * ti + (l & 7) + 8 * ((l >> 3) & 1), kk + 8 * (l >> 4)) for l in lanes]


def ldsm_rows_B2(tj, kk, lanes=range(16)):
    """x2 B fragment (one 8-column tile)."""
    return [(8 * tj + (l & 7), kk + 8 * ((l >> 3) & 1)) for l in lanes]


def ldsm_rows_B4(tj0, kk, lanes=range(32)):
    """x4 B fragment covering column tiles tj0 and tj0 + 1."""
    return [(8 * tj0 + (l & 7) + 8 * (l >> 4), kk + 8 * ((l >> 3) & 1)) for l in lanes]


def check(rows, nrows, pitch, kmax):
    """rows: (row, col) in halves of a [T][nrows][pitch] array; checks bounds, alignment, banks."""
    for t in range(T):
        offs = []
        for r, c in rows:
            assert 0 <= r < nrows and 0 <= c and c + 8 <= kmax <= pitch
            b = ((t * nrows + r) * pitch + c) * 2
            assert b % 16 == 0
            offs.append(b)
        for m in range(0, len(offs), 8):  # each 8 x 8 matrix: rows on distinct 16-byte groups
            groups = {(o // 16) % 8 for o in offs[m:m + 8]}
            assert len(groups) == 8


def test_gram_oz():
    ROWS, P, KM = 128, 136, 64
    for idx in range(20):
        ti = 3 if idx >= 18 else 2 if idx >= 14 else 1 if idx >= 8 else 0
        start = {0: 0, 1: 8, 2: 14, 3: 18}[ti]
        tj = 2 * ti + (idx - start)
        assert 8 * tj + 7 >= 16 * ti and tj < 8
        for kk in range(0, ROWS, 16):
            check(ldsm_rows_A(ti, kk), KM, P, ROWS)
            check(ldsm_rows_B2(tj, kk), KM, P, ROWS)


@pytest.mark.parametrize("KP", [16, 32, 48, 64])
def test_update_oz(KP):
    ROWS, P, KM = 64, 72, 64
    for warp in range(8):
        ti = warp & 3
        for h in range(2):
            tj0 = 4 * (warp >> 2) + 2 * h
            if 8 * tj0 >= KP:
                break
            for kk in range(0, KP, 16):
                check(ldsm_rows_A(ti, kk), ROWS, P, KM)
                check(ldsm_rows_B4(tj0, kk), KM, P, KM)


def test_gemm_oz():
    TI, TJ, P, KC = 64, 32, 72, 64
    for warp in range(8):
        ti, tj0 = warp & 3, 2 * (warp >> 2)
        for kk in range(0, KC, 16):
            check(ldsm_rows_A(ti, kk), TI, P, KC)
            check(ldsm_rows_B4(tj0, kk), TJ, P, KC)


@pytest.mark.parametrize("KM,KP", [(32, 16), (32, 32), (64, 48), (64, 64)])
def test_pivot_residual(KM, KP):
    P = KM + 8
    ntj = KP // 8
    for tile in range((KP // 16) * ntj):
        ti, tj = tile // ntj, tile % ntj
        if 8 * tj + 7 < 16 * ti:
            continue
        for kk in range(0, KP, 16):
            check(ldsm_rows_A(ti, kk), KM, P, KM)
            check(ldsm_rows_B2(tj, kk), KM, P, KM)
            r0 = kk + 2 * 3  # largest J index read for the sign masks: r0 + 9 < KP
            assert r0 + 9 < KP


@pytest.mark.parametrize("mp", [16, 48, 512, 1008, 4512, 8192])
@pytest.mark.parametrize("CS", [1, 2, 4, 8, 16])
def test_gram_row_split_and_loads(mp, CS):
    """k_gram_oz's row split over a cluster (rows per CTA rounded up to 16, 128-row stages): the
    CTAs' ranges tile [0, mp) exactly, every stage is a multiple of 16 rows, and every double2
    load (rows 64 i + 2 lane, 2 lane + 1 of a stage) is 16-byte aligned and inside the stage."""
    rpc = ((mp // CS + 15) // 16) * 16
    covered = []
    for crank in range(CS):
        rb = min(mp, crank * rpc)
        re = min(mp, rb + rpc)
        r0 = rb
        while r0 < re:
            rs = min(128, re - r0)
            assert rs % 16 == 0 and r0 % 16 == 0
            for i in range(2):
                for lane in range(32):
                    r = 64 * i + 2 * lane
                    if r < rs:
                        assert r + 1 < rs and (r0 + r) % 2 == 0  # double2 from a 16-byte aligned column
            covered.extend(range(r0, r0 + rs))
            r0 += 128
    assert covered == list(range(mp))
