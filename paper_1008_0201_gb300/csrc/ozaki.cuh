// ozaki.cuh -- FP64-accurate products from exact FP16 tensor-core products (error-free splitting
// after Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer. Algorithms 2012).
//
// GB300 runs FP16 mma.sync (FP32 accumulate) ~600x faster than FP64 mma, so the FP64 contractions
// of a step -- the Gram block A_P = G_P^* G_P (Eq. (3.4)), the update G_P V_P (Algorithm 3.4) and
// the J-orthogonality residual of V_P -- are formed from small-integer products:
//   - every value of a scale group (the entries that share one row of A or one column of B of a
//     product A B, so that the scale factors out of the contraction) is written as an integer
//     V = round(x 2^(55 - e)), |V| < 2^55, where 2^e bounds |x| over the group;
//   - V = sum_t d_t 128^(7 - t), t = 0..7, with balanced digits d_1..d_7 in [-64, 63] and
//     d_0 in [-64, 64]: every digit is an FP16 integer;
//   - digit products |d_t d_u| <= 2^12 are exact in FP16 x FP16 -> FP32, and the level sums
//     acc_L = sum over the contraction of sum_{t+u=L} d_t d_u (at most 8 products per term) stay
//     below 2^23 for up to 256 terms, where the tensor-core FP32 accumulation is exact;
//   - levels L = 0..NL-1 are kept: NL = 8 drops at most 7 * 2^-56 of the product of the two
//     group bounds per term, NL = 9 at most 6 * 2^-63;
//   - x . y = 2^(e + e' - 110) sum_L 2^(98 - 7 L) acc_L, summed in FP64.
// So each product is exact to 2^-53 of (row bound of A) x (column bound of B) per term, the
// scale of FP64 rounding itself, and the sum over levels rounds once more in FP64.
#pragma once
#include <cuda_fp16.h>

namespace jac {

#define OZ_T 8  // digits per value

// biased exponent of |x| (0 for zero and subnormals, which the splitting treats as zero)
__device__ __forceinline__ int oz_bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// x with biased exponent ex = oz_bexp(x) as the integer round(m 2^(d + 2)), m the 53-bit
// significand of |x| with its sign, for d = ex - (group bound exponent) <= 0: |result| < 2^55.
__device__ __forceinline__ long long oz_fixed(double x, int d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  if (((u >> 52) & 0x7ff) == 0) return 0;
  const unsigned long long mant = (u & ((1ull << 52) - 1)) | (1ull << 52);
  const int s = d + 2;
  unsigned long long a;
  if (s >= 0) a = mant << s;
  else if (s > -60) a = (mant + (1ull << (-s - 1))) >> (-s);
  else a = 0;
  return (u >> 63) ? -(long long)a : (long long)a;
}

// V (|V| < 2^55) -> 8 digits, most significant first, as FP16 integers.  The low 28 bits give
// d_7..d_4 and a carry in 32-bit arithmetic; the high part gives d_3..d_0.
__device__ __forceinline__ void oz_split(long long V, __half (&d)[OZ_T]) {
  int lo = (int)(V & 0x0FFFFFFFll);
  int hi = (int)(V >> 28);
#pragma unroll
  for (int t = OZ_T - 1; t >= 4; --t) {
    int dig = lo & 127;
    dig -= (dig >= 64) ? 128 : 0;
    lo = (lo - dig) >> 7;
    d[t] = __int2half_rn(dig);
  }
  hi += lo;  // carry 0 or 1
#pragma unroll
  for (int t = 3; t >= 1; --t) {
    int dig = hi & 127;
    dig -= (dig >= 64) ? 128 : 0;
    hi = (hi - dig) >> 7;
    d[t] = __int2half_rn(dig);
  }
  d[0] = __int2half_rn(hi);
}

__device__ __forceinline__ unsigned oz_h2(__half lo, __half hi) {
  return (unsigned)__half_as_ushort(lo) | ((unsigned)__half_as_ushort(hi) << 16);
}

// D += A B, m16n8k16, FP16 operands, FP32 accumulate
__device__ __forceinline__ void oz_mma(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// four 8 x 8 FP16 matrices from shared memory; lane l gives the address of row (l & 7) of
// matrix l >> 3
__device__ __forceinline__ void oz_ldsm4(unsigned (&r)[4], const __half* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void oz_ldsm2(unsigned& r0, unsigned& r1, const __half* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

// The digit products of one 16 x 16 (A) by 16 x 8 (B) piece into the level accumulators
// L = 0..NL-1 (NL = 8: 36 products; NL = 9: 43).
template <int NL>
__device__ __forceinline__ void oz_levels(float (&acc)[NL][4], const unsigned (&fa)[OZ_T][4],
                                          const unsigned (&fb)[OZ_T][2]) {
#pragma unroll
  for (int L = 0; L < NL; ++L)
#pragma unroll
    for (int t = (L >= OZ_T ? L - OZ_T + 1 : 0); t <= (L < OZ_T ? L : OZ_T - 1); ++t)
      oz_mma(acc[L], fa[t], fb[L - t][0], fb[L - t][1]);
}

// GB300 issues ~1.6 FP64 operations per clock per SM (FP32: 128), so the recombination avoids
// FP64 work: the integer level sums are gathered exactly in two int64 (hi: L = 0..3 in units of
// level 3, lo: L = 4..NL-1 in units of level NL-1, both below 2^51 for level sums below 2^23),
// turned into doubles by the exponent-bias trick and joined with one rounding: 4 FP64
// operations per value, against ~25 for a per-level sum and ldexp.

// exact double of an integer |x| < 2^51: the bits of 1.5 * 2^52 + x are those of 1.5 * 2^52
// plus x
__device__ __forceinline__ double oz_i2d(long long x) {
  return __longlong_as_double(0x4338000000000000ll + x) - 6755399441055744.0;
}

// 2^E sum_L acc_L 2^(-7 L), the acc_L exact integers held in FP32
template <int NL>
__device__ __forceinline__ double oz_value(const float (&acc)[NL][4], int v, int E) {
  static_assert(NL > 4 && NL <= 9, "two int64 accumulators");
  long long hi = 0, lo = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) hi = hi * 128 + __float2int_rn(acc[L][v]);
#pragma unroll
  for (int L = 4; L < NL; ++L) lo = lo * 128 + __float2int_rn(acc[L][v]);
  const double s = fma(oz_i2d(hi), (double)(1ll << (7 * (NL - 4))), oz_i2d(lo));
  const int e = E - 7 * (NL - 1);
  return (e >= -1022 && e <= 1023) ? s * __longlong_as_double((long long)(e + 1023) << 52) : ldexp(s, e);
}

// (double)f by integer operations (FP32 subnormals flush to zero)
__device__ __forceinline__ double oz_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu)), (int)(u << 29));
}

// x or -x by the sign bit (no FP64 operation)
__device__ __forceinline__ double oz_neg_if(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

}  // namespace jac
