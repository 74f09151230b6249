"""CPU model of the FP16 digit-product arithmetic (csrc/ozaki.cuh) in exact integer / rational
arithmetic.  It pins the facts the kernels rely on, independently of the GPU:

- the balanced base-128 split of an integer |V| < 2^55 into 8 digits reconstructs V exactly,
  d_1..d_7 in [-64, 63] and d_0 in [-64, 64] (every digit an FP16 integer);
- digit products are at most 2^12 and a level sum over 256 terms stays below 2^23 (the range in
  which FP32 accumulation of integers is exact);
- the two-int64 gathering of the level sums (hi: levels 0..3, lo: levels 4..NL-1) stays below
  2^51, where the exponent-bias conversion to double is exact;
- with the scale groups of the kernels, a Gram entry is exact to a few 2^-53 of the product of
  its column bounds, and an update entry to 2 eps * sum |x v| even for graded columns (the column
  scaling D of the update), against the exact rational result.

This models the arithmetic; the GPU tests compare the kernels with the oracle.
"""
import math
import random
import struct
from fractions import Fraction

import pytest

T = 8


def bexp(x):
    return (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF


def fixed(x, d):
    """round(m 2^(d + 2)) with the sign of x, m the 53-bit significand; d <= 0."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    if (u >> 52) & 0x7FF == 0:
        return 0
    mant = (u & ((1 << 52) - 1)) | (1 << 52)
    s = d + 2
    assert s <= 2
    if s >= 0:
        a = mant << s
    elif s > -60:
        a = (mant + (1 << (-s - 1))) >> (-s)
    else:
        a = 0
    return -a if u >> 63 else a


def split(V):
    """Balanced digits, most significant first: low 28 bits first, then the high part."""
    lo, hi = V & 0x0FFFFFFF, V >> 28
    d = [0] * T
    for t in range(T - 1, 3, -1):
        dig = lo & 127
        if dig >= 64:
            dig -= 128
        lo = (lo - dig) >> 7
        d[t] = dig
    hi += lo
    for t in range(3, 0, -1):
        dig = hi & 127
        if dig >= 64:
            dig -= 128
        hi = (hi - dig) >> 7
        d[t] = dig
    d[0] = hi
    return d


def levels(da, db, nl):
    return [sum(da[t] * db[L - t] for t in range(max(0, L - T + 1), min(L, T - 1) + 1)) for L in range(nl)]


def value(acc, E):
    """Two-int64 gathering, one rounding (modelled with exact integers then one float rounding)."""
    nl = len(acc)
    hi = 0
    for L in range(4):
        hi = hi * 128 + acc[L]
    lo = 0
    for L in range(4, nl):
        lo = lo * 128 + acc[L]
    assert abs(hi) < 2 ** 51 and abs(lo) < 2 ** 51
    s = float(Fraction(hi * 2 ** (7 * (nl - 4)) + lo))  # fma(hi, 2^k, lo): one rounding
    return math.ldexp(s, E - 7 * (nl - 1))


def test_split_reconstructs_and_bounds():
    g = random.Random(1)
    cases = [2 ** 55 - 1, -(2 ** 55 - 1), 0, 1, -1, 2 ** 28 - 1, -(2 ** 28), 64 * 2 ** 49 - 1]
    cases += [g.randrange(-(2 ** 55) + 1, 2 ** 55) for _ in range(20000)]
    for V in cases:
        d = split(V)
        assert sum(d[t] * 128 ** (T - 1 - t) for t in range(T)) == V
        assert all(-64 <= x <= 63 for x in d[1:]) and -64 <= d[0] <= 64


def test_level_sums_stay_exact_in_fp32():
    worst = [64] * T  # the largest digits in magnitude
    for nl in (8, 9):
        acc = levels(worst, worst, nl)
        assert max(acc) * 256 <= 2 ** 23  # 256 terms: exact FP32 integers


def _gram_entry(x, y, nl=8):
    Ex, Ey = max(bexp(v) for v in x), max(bexp(v) for v in y)
    acc = [0] * nl
    for a, b in zip(x, y):
        lv = levels(split(fixed(a, bexp(a) - Ex)), split(fixed(b, bexp(b) - Ey)), nl)
        acc = [p + q for p, q in zip(acc, lv)]
    assert max(abs(v) for v in acc) < 2 ** 23
    return value(acc, Ex + Ey - 2056)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gram_entry_error(seed):
    g = random.Random(100 + seed)
    for _ in range(20):
        R = 128
        sx, sy = 10 ** g.uniform(-30, 30), 10 ** g.uniform(-30, 30)
        x = [g.gauss(0, 1) * sx for _ in range(R)]
        y = [g.gauss(0, 1) * sy for _ in range(R)]
        got = _gram_entry(x, y)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
        bound = Fraction(max(abs(v) for v in x)) * Fraction(max(abs(v) for v in y))
        # per term <= (2 digit roundings + dropped levels) ~ 2^-54 of the bounds, plus one rounding
        assert abs(Fraction(got) - exact) <= R * Fraction(1, 2 ** 53) * bound + abs(exact) * Fraction(1, 2 ** 52)


def test_update_entry_error_graded_columns():
    """Y[r][c] = sum_k X[r][k] V[k][c] with columns of X spread over 16 decades and V graded the
    opposite way: the column scaling keeps the error within 2 eps sum |x v|."""
    g = random.Random(7)
    K, ROWS, NL = 64, 6, 9
    worst = 0.0
    for _ in range(30):
        cs = [10 ** g.uniform(-8, 8) for _ in range(K)]
        X = [[g.gauss(0, 1) * cs[k] for k in range(K)] for _ in range(ROWS)]
        V = [[g.gauss(0, 1) / cs[k] * 10 ** g.uniform(-2, 2) for k in range(K)] for _ in range(3)]  # V[c][k]
        cexp = [max(bexp(X[r][k]) for r in range(ROWS)) for k in range(K)]
        for r in range(ROWS):
            ea = max(bexp(X[r][k]) - cexp[k] for k in range(K))
            for c in range(3):
                eb = max(bexp(V[c][k]) + cexp[k] for k in range(K))
                acc = [0] * NL
                for k in range(K):
                    lv = levels(split(fixed(X[r][k], bexp(X[r][k]) - cexp[k] - ea)),
                                split(fixed(V[c][k], bexp(V[c][k]) + cexp[k] - eb)), NL)
                    acc = [p + q for p, q in zip(acc, lv)]
                got = value(acc, ea + eb - 2056)
                exact = sum(Fraction(X[r][k]) * Fraction(V[c][k]) for k in range(K))
                scale = sum(abs(Fraction(X[r][k]) * Fraction(V[c][k])) for k in range(K))
                worst = max(worst, float(abs(Fraction(got) - exact) / scale))
    assert worst <= 2 * 2.0 ** -53, worst


def test_update_without_column_scaling_loses_graded_columns():
    """The same graded case with the rows of X as the only scale groups: the error relative to
    sum |x v| grows far past FP64 rounding, which is why the update scales columns first."""
    g = random.Random(8)
    K, NL = 64, 9
    cs = [10 ** g.uniform(-8, 8) for _ in range(K)]
    x = [g.gauss(0, 1) * cs[k] for k in range(K)]
    v = [g.gauss(0, 1) / cs[k] * 1e-3 for k in range(K)]
    ea, eb = max(bexp(a) for a in x), max(bexp(b) for b in v)
    acc = [0] * NL
    for a, b in zip(x, v):
        lv = levels(split(fixed(a, bexp(a) - ea)), split(fixed(b, bexp(b) - eb)), NL)
        acc = [p + q for p, q in zip(acc, lv)]
    got = value(acc, ea + eb - 2056)
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, v))
    scale = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(x, v))
    assert float(abs(Fraction(got) - exact) / scale) > 1e-12


NO_EXP = -100000


def update_slab(X, V, nl=9):
    """Y = X V with the update kernel's scale groups: c_k over the slab's rows, row groups of
    X D^-1 and column groups of D V over k with c_k > 0; zero rows / columns give OZ_NO_EXP."""
    rows, K, cols = len(X), len(X[0]), len(V[0])
    cexp = [max(bexp(X[r][k]) for r in range(rows)) for k in range(K)]
    rexp = []
    for r in range(rows):
        m = [bexp(X[r][k]) - cexp[k] for k in range(K) if bexp(X[r][k]) != 0]
        rexp.append(max(m) if m else NO_EXP)
    vexp = []
    for c in range(cols):
        m = [bexp(V[k][c]) + cexp[k] for k in range(K) if bexp(V[k][c]) != 0 and cexp[k] != 0]
        vexp.append(max(m) if m else NO_EXP)
    Y = [[0.0] * cols for _ in range(rows)]
    for r in range(rows):
        for c in range(cols):
            acc = [0] * nl
            for k in range(K):
                x, v = X[r][k], V[k][c]
                a = fixed(x, bexp(x) - cexp[k] - rexp[r]) if bexp(x) else 0
                b = fixed(v, bexp(v) + cexp[k] - vexp[c]) if (bexp(v) and cexp[k]) else 0
                lv = levels(split(a), split(b), nl)
                acc = [p + q for p, q in zip(acc, lv)]
            Y[r][c] = value(acc, rexp[r] + vexp[c] - 2056) if any(acc) else 0.0
    return Y


def test_update_zero_rows_columns_and_subnormals():
    g = random.Random(11)
    K = 16
    X = [[g.gauss(0, 1) for _ in range(K)] for _ in range(5)]
    for r in range(5):
        X[r][3] = 0.0            # a zero column of the slab (c_k = 0)
    X[2] = [0.0] * K             # a zero row
    X[4][7] = 5e-320             # a subnormal entry: treated as zero
    V = [[g.gauss(0, 1) for _ in range(4)] for _ in range(K)]
    for k in range(K):
        V[k][1] = 0.0            # a zero column of V_P
    V[3][2] = 1e300              # large, but on the zero column of X
    Y = update_slab(X, V)
    for r in range(5):
        for c in range(4):
            xs = [0.0 if bexp(x) == 0 else x for x in X[r]]
            exact = sum(Fraction(xs[k]) * Fraction(V[k][c]) for k in range(K))
            scale = sum(abs(Fraction(xs[k]) * Fraction(V[k][c])) for k in range(K))
            if scale == 0:
                assert Y[r][c] == 0.0
            else:
                assert abs(Fraction(Y[r][c]) - exact) <= 2 * Fraction(1, 2 ** 53) * scale
