"""The integer-only final rounding of the digit-product kernels (csrc/oz_assemble.h), on the CPU.

oz_assemble(hi, lo, sh, e) must return the double nearest to 2^e (hi 2^sh + lo), ties to even,
exactly as one FP64 rounding of the exact sum would (the FP64 route it replaces is
fma(hi, 2^sh, lo) * 2^e).  The header is compiled for the host with g++ and checked bit for bit
against Python's correctly rounded integer-to-float conversion, on random and adversarial inputs
(ties, carries across the 64-bit halves, negative sums, cancellations, rounding up to the next
power of two), and against the kernels' FP64 formula through the C library's fma.
"""
import ctypes
import math
import os
import random
import struct
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include "oz_assemble.h"
extern "C" double assemble(long long hi, long long lo, int sh, int e) { return jac::oz_assemble(hi, lo, sh, e); }
'''


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp()
    cpp = os.path.join(d, "a.cpp")
    so = os.path.join(d, "a.so")
    with open(cpp, "w") as f:
        f.write(SRC)
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++14", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_1008_0201_gb300", "csrc"), "-o", so, cpp], check=True)
    L = ctypes.CDLL(so)
    L.assemble.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, ctypes.c_int]
    L.assemble.restype = ctypes.c_double
    return L


_libm = ctypes.CDLL("libm.so.6")
_libm.fma.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
_libm.fma.restype = ctypes.c_double


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def exact(hi, lo, sh, e):
    s = (hi << sh) + lo
    return math.ldexp(float(s), e) if s else 0.0  # int -> float is correctly rounded; ldexp exact here


def check(lib, hi, lo, sh, e):
    got = lib.assemble(hi, lo, sh, e)
    want = exact(hi, lo, sh, e)
    assert bits(got) == bits(want), (hi, lo, sh, e, got, want)
    if want != 0.0 and abs(hi) < 2 ** 53 and abs(lo) < 2 ** 53:
        # the FP64 route of the kernels: one fused rounding of hi 2^sh + lo, then the exact scale
        assert bits(got) == bits(math.ldexp(_libm.fma(float(hi), 2.0 ** sh, float(lo)), e)), (hi, lo, sh, e)


@pytest.mark.parametrize("sh", [28, 35])
def test_random(lib, sh):
    g = random.Random(sh)
    for _ in range(20000):
        hi = g.randrange(-2 ** 51, 2 ** 51) >> g.randrange(0, 50)
        lo = g.randrange(-2 ** 51, 2 ** 51) >> g.randrange(0, 50)
        check(lib, hi, lo, sh, g.randrange(-1000, 900))


def test_adversarial(lib):
    cases = []
    for sh in (28, 35):
        for hi in (0, 1, -1, 2 ** 50, -(2 ** 50), 2 ** 51 - 1, -(2 ** 51 - 1), 3, 12345):
            for lo in (0, 1, -1, 2 ** (sh - 1), -(2 ** (sh - 1)), 2 ** sh - 1, -(2 ** sh), 2 ** 51 - 1,
                       -(2 ** 51 - 1), 3 * 2 ** (sh - 2)):
                cases.append((hi, lo, sh))
        # exact ties at the 53-bit boundary: odd and even mantissas, below and above 2^64
        for p in (53, 60, 63, 64, 65, 70, 80):
            for m in (2 ** 52 + 1, 2 ** 52 + 2, 2 ** 53 - 1):
                s = (2 * m + 1) << (p - 53)  # halfway between m 2^(p-52) and (m+1) 2^(p-52)
                hi, lo = s >> sh, s & ((1 << sh) - 1)
                cases += [(hi, lo, sh), (-hi, -lo, sh), (hi, lo + 1, sh), (hi, lo - 1, sh)]
        # hi and lo of opposite signs (cancellation, borrow across the halves)
        cases += [(1, -(2 ** sh) + 1, sh), (-1, 2 ** sh - 1, sh), (2 ** 40, -(2 ** 51 - 1), sh)]
    for hi, lo, sh in cases:
        for e in (-1074 + 60, -200, -56, 0, 37, 800):
            check(lib, hi, lo, sh, e)


def test_zero_and_range_fallback(lib):
    assert bits(lib.assemble(0, 0, 35, 10)) == bits(0.0)
    assert bits(lib.assemble(5, -5 * 2 ** 35, 35, 3)) == bits(0.0)
    # subnormal and overflowing results go through ldexp: nearest subnormal / infinity
    assert lib.assemble(0, 3, 35, -1075) == math.ldexp(3.0, -1075)
    assert lib.assemble(1, 0, 35, 1000) == math.inf
