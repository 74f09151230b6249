// oz_assemble.h -- the double nearest to 2^e (hi 2^sh + lo), by integer operations only.
//
// The digit-product kernels gather the exact FP32 level sums of a product into two integers, hi
// and lo, whose weighted sum hi 2^sh + lo, scaled by 2^e, is the FP64-accurate result.  GB300
// issues about 1.6 FP64 operations per clock per SM against 64 integer ones, so the final
// rounding is done here in integer arithmetic: the sum is formed exactly in 128 bits, normalized,
// rounded once to nearest (ties to even) to 53 bits, and the exponent field is written directly.
// The result equals fma(hi, 2^sh, lo) * 2^e in IEEE double whenever that is a normal number
// (both round the exact sum once); subnormal or overflowing results take the FP64 route.
// Host and device code (the host side serves the CPU tests of this arithmetic).
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#include <math.h>
#endif

namespace jac {

OZ_HD int oz_clz64(unsigned long long x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

OZ_HD double oz_bits_to_double(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
#endif
}

OZ_HD double oz_ldexp(double x, int e) {
#if defined(__CUDA_ARCH__)
  return ldexp(x, e);
#else
  return ::ldexp(x, e);
#endif
}

// 0 < sh < 64; |hi| 2^sh + |lo| < 2^126
OZ_HD double oz_assemble(long long hi, long long lo, int sh, int e) {
  // S = hi 2^sh + lo in 128-bit two's complement (H:L)
  unsigned long long L = (unsigned long long)hi << sh;
  long long H = hi >> (64 - sh);
  const unsigned long long L2 = L + (unsigned long long)lo;
  H += (lo < 0 ? -1 : 0) + (L2 < L ? 1 : 0);
  L = L2;
  const bool neg = H < 0;
  unsigned long long uH = (unsigned long long)H;
  if (neg) {  // |S|
    L = ~L + 1ull;
    uH = ~uH + (L == 0 ? 1ull : 0ull);
  }
  if (uH == 0 && L == 0) return 0.0;
  const int lz = uH ? oz_clz64(uH) : 64 + oz_clz64(L);
  int p = 127 - lz;  // |S| in [2^p, 2^(p+1))
  unsigned long long mant;
  if (p <= 52) {
    mant = L << (52 - p);  // exact (p < 64)
  } else {
    const int r = p - 52;  // bits dropped, 1..74
    bool up;
    if (r < 64) {
      mant = (L >> r) | (r ? (uH << (64 - r)) : 0ull);
      const unsigned long long rem = L & ((1ull << r) - 1ull), half = 1ull << (r - 1);
      up = rem > half || (rem == half && (mant & 1ull));
    } else {
      const int r2 = r - 64;  // 0..10
      mant = uH >> r2;
      const unsigned long long rem_hi = r2 ? (uH & ((1ull << r2) - 1ull)) : 0ull;
      if (r2 == 0) {  // half = 2^63 in L
        up = L > (1ull << 63) || (L == (1ull << 63) && (mant & 1ull));
      } else {
        const unsigned long long half_hi = 1ull << (r2 - 1);
        up = rem_hi > half_hi || (rem_hi == half_hi && (L != 0 || (mant & 1ull)));
      }
    }
    if (up) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant = 1ull << 52;
        ++p;
      }
    }
  }
  const int be = p + e + 1023;  // value = mant 2^(p - 52) 2^e
  if (be >= 1 && be <= 2046)
    return oz_bits_to_double(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) |
                             (mant & ((1ull << 52) - 1ull)));
  const double m = neg ? -(double)mant : (double)mant;  // exact: 53 bits
  return oz_ldexp(m, p - 52 + e);
}

}  // namespace jac
