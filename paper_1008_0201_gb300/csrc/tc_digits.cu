// tc_digits.cu -- the FP64-accurate block update (Algorithm 3.4: [G_p G_q] <- [G_p G_q] V_P, and
// the same for V) from exact FP16 digit products on the fifth-generation tensor cores.
//
// Same arithmetic as k_update_oz (ozaki.cu), rebuilt around tcgen05:
//   - a CTA takes 128-row tiles of Gw (then Vw) of one pair; per tile the columns are brought to
//     a common size (X~ = X D^-1, V~ = D V_P, D = diag(2^c_k), c_k the bound exponent of tile
//     column k), the rows of X~ and the columns of V~ are the scale groups, and every value
//     becomes 8 balanced 7-bit digits (ozaki.cuh), each an FP16 integer;
//   - the digits are written as K-major operands with the 128-byte swizzle (X~: 8 planes of
//     128 rows x 64 K; V~: 8 planes of 64 columns x 64 K) and one thread issues
//     tcgen05.mma kind::f16 (M = 128, N = 64, K = 16) for every digit pair (t, u), t + u <= 8;
//     products are exact and the level sums acc_L = sum_{t+u=L} d_t d_u stay below 2^23 (64-term
//     contraction), where the FP32 accumulation in tensor memory is exact;
//   - levels 0..7 fill the 512 tensor-memory columns (one 64-column block per level); level 8
//     reuses block 0 once level 0 has been read;
//   - each thread reads its row's level sums for 16 output columns, gathers them exactly in two
//     int64 (levels 0..3 and 4..8) and rounds hi 2^35 + lo once to double in integer arithmetic
//     (oz_assemble.h): no FP64 instruction on the path.
// Grid (nx, 1, nprob), 512 threads, ~195 KB of shared memory (one CTA per SM): a persistent CTA
// walks the (pair, tile) items of its problem with stride nx; the items of pairs that did not
// rotate (skip flag of the pivot) cost one flag read.
#include <cooperative_groups.h>

#include "jacobi_common.cuh"
#include "oz_assemble.h"
#include "ozaki.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace jac {

namespace {
__device__ __forceinline__ unsigned char* align1k_d(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}
// an FP32 value that holds an integer of magnitude <= 2^22, as that integer (one FP32 add: the
// integer lands in the low mantissa bits of 1.5 * 2^23 + x)
__device__ __forceinline__ int f32_small_int(float x) { return __float_as_int(x + 12582912.0f) - 0x4B400000; }
__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
}  // namespace

#define TD_XPLANE 16384                       // 128 rows x 128 B
#define TD_VPLANE 8192                        // 64 rows x 128 B
#define TD_XOFF 0
#define TD_VOFF (OZ_T * TD_XPLANE)            // 131072
#define TD_MISC (TD_VOFF + OZ_T * TD_VPLANE)  // 196608: cexp[64], rexp[128], vexp[64], barriers
#define TD_SMEM (1024 + TD_MISC + 1024 + 128)
#define TD_NO_EXP (-100000)

size_t tc_update_oz_smem_bytes() { return TD_SMEM; }

// the integer rounding, called rather than inlined: it runs once per output and keeping it out of
// line keeps the unrolled kernels within the instruction cache
__device__ __noinline__ double oz_assemble_call(long long hi, long long lo, int sh, int e) {
  return oz_assemble(hi, lo, sh, e);
}

__global__ void __launch_bounds__(512, 1) k_update_oz_tc(const JacProb* __restrict__ probs, int s) {
  extern __shared__ unsigned char td_raw[];
  unsigned char* sm = align1k_d(td_raw);
  int* cexp = reinterpret_cast<int*>(sm + TD_MISC);
  int* rexp = cexp + 64;
  int* vexp = rexp + 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(vexp + 64);  // [0] levels 0..7, [1] level 8
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const JacProb& a = probs[blockIdx.z];
  if (!a.active || s >= a.nsteps) return;
  const int gtiles = (a.mp + 127) >> 7;
  const int ntiles = gtiles + (a.Vw ? (a.np + 127) >> 7 : 0);
  const int nitems = a.counts[s] * ntiles;
  if ((int)blockIdx.x >= nitems) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  constexpr uint32_t idesc = tc::idesc_f32acc(tc::FMT_F16, 128, 64, 0, 0);
  const uint32_t xs = tc::smem_u32(sm + TD_XOFF), vs = tc::smem_u32(sm + TD_VOFF);
  // tile row r and output columns 16 cq .. + 15 of this thread, for the loads and digits of X~
  // and for the epilogue (warp w reads TMEM lanes 32 (w & 3) .. + 31: tid & 127 = r)
  const int r = tid & 127, cq = tid >> 7;
  const int vc = tid >> 3, vk0 = 8 * (tid & 7);  // V_P: column vc, rows (slab columns) vk0 .. + 7
  const uint32_t lrow = tb + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * cq;
  bool bad = false;
  int it = 0;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int pair = item / ntiles, t = item - pair * ntiles;
    if (a.skip[pair]) continue;  // uniform over the CTA
    const int* sp = a.pairs + (size_t)s * a.half * 2;
    const int p = sp[2 * pair], q = sp[2 * pair + 1];
    const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
    const int k = wp + wq;
    const double* Vp = a.vp + (size_t)pair * a.apld * a.apld;
    const bool isg = t < gtiles;
    double* base = isg ? a.Gw : a.Vw;
    const int ld = isg ? a.mp : a.np;
    const int r0 = (isg ? t : t - gtiles) << 7;
    const int rows = min(128, (isg ? a.mp : a.np) - r0);
    // ---- loads (all issued before use)
    double x[16], v[8];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = 16 * cq + j;
      x[j] = (c < k && r < rows) ? base[(size_t)(c < wp ? op + c : oq + c - wp) * ld + r0 + r] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (vc < k && vk0 + j < k) ? __ldg(Vp + (size_t)vc * a.apld + vk0 + j) : 0.0;
    if (tid < 64) cexp[tid] = 0;
    if (tid < 128) rexp[tid] = TD_NO_EXP;
    __syncthreads();
    // ---- column bounds c_k of the tile (a warp holds 32 rows of 16 columns)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = warp_max_int(oz_bexp(x[j]));
      if (lane == 0 && e > 0) atomicMax(&cexp[16 * cq + j], e);
    }
    __syncthreads();
    // ---- row groups of X~ and column groups of V~
    {
      int m = TD_NO_EXP;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int ex = oz_bexp(x[j]);
        if (ex != 0) m = max(m, ex - cexp[16 * cq + j]);
      }
      if (m != TD_NO_EXP) atomicMax(&rexp[r], m);
      int mv = TD_NO_EXP;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int ev = oz_bexp(v[j]), ck = cexp[vk0 + j];
        if (ev != 0 && ck != 0) mv = max(mv, ev + ck);
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) mv = max(mv, __shfl_xor_sync(0xffffffffu, mv, o));
      if ((tid & 7) == 0) vexp[vc] = mv;
    }
    // the previous tile's MMAs were waited for before its epilogue: the planes are free
    __syncthreads();
    // ---- digits of X~ (row r) and of V~ (operand row vc): 16-byte stores, 8 K entries each
    {
      const int ea = rexp[r];
#pragma unroll
      for (int j0 = 0; j0 < 16; j0 += 8) {
        unsigned w[OZ_T][4];
#pragma unroll
        for (int jj = 0; jj < 8; jj += 2) {
          __half d0[OZ_T], d1[OZ_T];
          const int c0 = 16 * cq + j0 + jj;
          oz_split(oz_fixed(x[j0 + jj], oz_bexp(x[j0 + jj]) - cexp[c0] - ea), d0);
          oz_split(oz_fixed(x[j0 + jj + 1], oz_bexp(x[j0 + jj + 1]) - cexp[c0 + 1] - ea), d1);
#pragma unroll
          for (int tt = 0; tt < OZ_T; ++tt) w[tt][jj >> 1] = oz_h2(d0[tt], d1[tt]);
        }
        const uint32_t off = tc::sw128_offset(r, 16 * cq + j0, 2);
#pragma unroll
        for (int tt = 0; tt < OZ_T; ++tt)
          *reinterpret_cast<uint4*>(sm + TD_XOFF + tt * TD_XPLANE + off) = make_uint4(w[tt][0], w[tt][1], w[tt][2],
                                                                                      w[tt][3]);
      }
      const int ev = vexp[vc];
      unsigned w[OZ_T][4];
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        __half d0[OZ_T], d1[OZ_T];
        const int ck0 = cexp[vk0 + jj], ck1 = cexp[vk0 + jj + 1];
        oz_split((ck0 != 0 && ev != TD_NO_EXP) ? oz_fixed(v[jj], oz_bexp(v[jj]) + ck0 - ev) : 0ll, d0);
        oz_split((ck1 != 0 && ev != TD_NO_EXP) ? oz_fixed(v[jj + 1], oz_bexp(v[jj + 1]) + ck1 - ev) : 0ll, d1);
#pragma unroll
        for (int tt = 0; tt < OZ_T; ++tt) w[tt][jj >> 1] = oz_h2(d0[tt], d1[tt]);
      }
      const uint32_t off = tc::sw128_offset(vc, vk0, 2);
#pragma unroll
      for (int tt = 0; tt < OZ_T; ++tt)
        *reinterpret_cast<uint4*>(sm + TD_VOFF + tt * TD_VPLANE + off) = make_uint4(w[tt][0], w[tt][1], w[tt][2],
                                                                                    w[tt][3]);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // ---- levels 0..7: block L (TMEM columns 64 L ..) accumulates sum_{t+u=L} X_t V_u
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll 1
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll 1
        for (int L = 0; L < OZ_T; ++L)
          for (int tt = 0; tt <= L; ++tt)
            tc::mma_f16(tb + 64 * L, tc::desc_sw128(xs + tt * TD_XPLANE + kk * 32, 16, 1024),
                        tc::desc_sw128(vs + (L - tt) * TD_VPLANE + kk * 32, 16, 1024), idesc,
                        (kk > 0 || tt > 0) ? 1u : 0u);
      tc::mma_commit(&bar[0]);
    }
    if (__syncthreads_or(!tc::mbar_wait(&bar[0], it & 1))) {
      bad = true;
      break;
    }
    tc::fence_after_sync();
    uint32_t l0[16];
    tc::tmem_ld16(lrow, l0);
    tc::tmem_wait_ld();
    tc::fence_before_sync();
    __syncthreads();  // level 0 read everywhere: block 0 is free for level 8
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll 1
      for (int kk = 0; kk < 4; ++kk)
        for (int tt = 1; tt < OZ_T; ++tt)
          tc::mma_f16(tb, tc::desc_sw128(xs + tt * TD_XPLANE + kk * 32, 16, 1024),
                      tc::desc_sw128(vs + (8 - tt) * TD_VPLANE + kk * 32, 16, 1024), idesc,
                      (kk > 0 || tt > 1) ? 1u : 0u);
      tc::mma_commit(&bar[1]);
    }
    long long hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      hi[j] = f32_small_int(__uint_as_float(l0[j]));
      lo[j] = 0;
    }
#pragma unroll
    for (int L = 1; L < OZ_T; ++L) {
      uint32_t lv[16];
      tc::tmem_ld16(lrow + 64 * L, lv);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const long long iv = f32_small_int(__uint_as_float(lv[j]));
        if (L < 4) hi[j] = hi[j] * 128 + iv;
        else lo[j] = lo[j] * 128 + iv;
      }
    }
    if (__syncthreads_or(!tc::mbar_wait(&bar[1], it & 1))) {
      bad = true;
      break;
    }
    tc::fence_after_sync();
    tc::tmem_ld16(lrow, l0);
    tc::tmem_wait_ld();
    if (r < rows) {
      const int ea = rexp[r];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 16 * cq + j;
        if (c < k) {
          const long long lf = lo[j] * 128 + f32_small_int(__uint_as_float(l0[j]));
          base[(size_t)(c < wp ? op + c : oq + c - wp) * ld + r0 + r] =
              oz_assemble_call(hi[j], lf, 35, ea + vexp[c] - 2056 - 56);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM and the exponent arrays read before the next tile reuses them
    ++it;
  }
  if (bad && tid == 0) {
    atomicOr(a.pflags, JAC_DEVERR_TIMEOUT);
    tc::mbar_wait(&bar[0], it & 1);
    tc::mbar_wait(&bar[1], it & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ------------------------------------------------------------------------------------ Gram
// FP64-accurate Gram block A_P = X^T X (Eq. (3.4)) from exact FP16 digit products, as k_gram_oz:
// grid (half * CS, nprob), cluster (CS, 1, 1), the CTAs of a cluster splitting the rows; per
// group of 128 rows every column is a scale group (bound exponent E_c), its values become 8
// digits, levels 0..7 are kept (36 digit products per multiply-add), and the level sums of a
// group are rounded to FP64 with the group's exponents and added up in FP64 across groups.
//
// tcgen05 layout.  The operand is X^T: 64 rows (the pair's columns) by 128 K (the group's rows),
// as two 64-K chunks; inside a chunk the 8 digit planes follow each other (plane t at t * 8 KB),
// so that one M = 128 operand covers planes a and a + 1.  An MMA with A = [D_a; D_{a+1}] and
// B = D_v (N = 64) puts D_a D_v^T (level a + v) in TMEM lanes 0..63 and D_{a+1} D_v^T (level
// a + v + 1) in lanes 64..127 of the 64-column block L = a + v.  Tiling every column v of the
// (t, v) product table with such pairs of rows (a, a + 1), a = 0, 2, 4, .., covers each product
// with t + v <= 7 exactly once in 20 MMAs per 16 K (instead of 36); the pairs that reach
// t + v = 8 land in the lower half of block 7, which is not read.  Level L is then the upper half
// of block L plus the lower half of block L - 1: the lower lanes gather their share in int64 and
// pass it to the upper lanes through shared memory, which round each entry once (oz_assemble).
// A_P is exactly symmetric (the level sums of (i, j) and (j, i) are the same integers), so only
// entries j >= i are formed.
#define TGD_CHUNK 65536                        // 8 planes x 64 rows x 128 B
#define TGD_TOT (2 * TGD_CHUNK)                // FP64 partial [64][65] after the digits
#define TGD_MISC (TGD_TOT + 64 * 65 * 8)
#define TGD_SMEM (1024 + TGD_MISC + 512 + 128)

size_t tc_gram_oz_smem_bytes() { return TGD_SMEM; }

__global__ void __launch_bounds__(512, 1) k_gram_oz_tc(const JacProb* __restrict__ probs, int s, int CS) {
  extern __shared__ unsigned char tgd_raw[];
  unsigned char* sm = align1k_d(tgd_raw);
  double* tot = reinterpret_cast<double*>(sm + TGD_TOT);  // [64][65], entries j >= i
  int* E = reinterpret_cast<int*>(sm + TGD_MISC);         // [64]
  uint64_t* bar = reinterpret_cast<uint64_t*>(E + 64);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  long long* xch = reinterpret_cast<long long*>(sm);      // [64][64][2], over the digits
  cg::cluster_group cluster = cg::this_cluster();
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x / CS;
  const int crank = (int)cluster.block_rank();
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || (a.cached && a.cached[pair])) return;  // uniform
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rpc = ((a.mp / CS + 15) & ~15);
  const int r_begin = min(a.mp, crank * rpc), r_end = min(a.mp, r_begin + rpc);
  for (int e = tid; e < 64 * 65; e += 512) tot[e] = 0.0;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  constexpr uint32_t idesc = tc::idesc_f32acc(tc::FMT_F16, 128, 64, 0, 0);
  const uint32_t ds = tc::smem_u32(sm);
  // epilogue: warp w reads TMEM lanes 32 (w & 3) .. + 31 (operand rows), columns 16 (w >> 2) .. + 15
  const int lrow = 32 * (warp & 3) + lane, cg16 = warp >> 2;
  const bool upper = (warp & 3) < 2;
  const uint32_t laddr = tb + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * cg16;
  bool bad = false;
  int it = 0;
  for (int g0 = r_begin; g0 < r_end; g0 += 128, ++it) {
    const int rs = min(128, r_end - g0);
    // warp w: columns 4 w .. 4 w + 3; lane l: group rows 4 l .. 4 l + 3 (K-adjacent digits)
    double x[4][4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = 4 * warp + cc;
      const double* col = a.Gw + (size_t)(c < wp ? op + c : oq + c - wp) * a.mp + g0;
#pragma unroll
      for (int i = 0; i < 4; i += 2) {
        const int rr = 4 * lane + i;
        const double2 v = (c < k && rr < rs) ? __ldg(reinterpret_cast<const double2*>(col + rr)) : make_double2(0.0, 0.0);
        x[cc][i] = v.x;
        x[cc][i + 1] = v.y;
      }
    }
    int ec[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      ec[cc] = warp_max_int(max(max(oz_bexp(x[cc][0]), oz_bexp(x[cc][1])), max(oz_bexp(x[cc][2]), oz_bexp(x[cc][3]))));
    if (lane == 0)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) E[4 * warp + cc] = ec[cc];
    // digits: operand row c (pair column), K = group rows 4 lane .. + 3 (chunk lane >> 4)
    {
      unsigned char* base = sm + (lane >> 4) * TGD_CHUNK;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        __half d[4][OZ_T];
#pragma unroll
        for (int i = 0; i < 4; ++i) oz_split(oz_fixed(x[cc][i], oz_bexp(x[cc][i]) - ec[cc]), d[i]);
        const uint32_t off = tc::sw128_offset(4 * warp + cc, (4 * lane) & 63, 2);
#pragma unroll
        for (int tt = 0; tt < OZ_T; ++tt)
          *reinterpret_cast<uint2*>(base + tt * 8192 + off) = make_uint2(oz_h2(d[0][tt], d[1][tt]), oz_h2(d[2][tt], d[3][tt]));
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      unsigned started = 0;
#pragma unroll 1
      for (int kc = 0; kc < 2; ++kc)
#pragma unroll 1
        for (int ks = 0; ks < 4; ++ks)
#pragma unroll 1
          for (int v = 0; v < OZ_T; ++v)
            for (int a0 = 0; a0 + v <= OZ_T - 1; a0 += 2) {
              const int L = a0 + v;
              const uint32_t co = kc * TGD_CHUNK + ks * 32;
              tc::mma_f16(tb + 64 * L, tc::desc_sw128(ds + co + a0 * 8192, 16, 1024),
                          tc::desc_sw128(ds + co + v * 8192, 16, 1024), idesc, (started >> L) & 1u);
              started |= 1u << L;
            }
      tc::mma_commit(&bar[0]);
    }
    if (__syncthreads_or(!tc::mbar_wait(&bar[0], it & 1))) {
      bad = true;
      break;
    }
    tc::fence_after_sync();
    // gather: upper lanes (lrow < 64) hold levels 0..7 of row i = lrow in blocks 0..7, lower
    // lanes levels 1..7 of row i = lrow - 64 in blocks 0..6
    long long hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
#pragma unroll
    for (int B = 0; B < OZ_T; ++B) {
      const int L = upper ? B : B + 1;  // level held by this lane in block B (warp-uniform)
      if (L >= OZ_T) break;
      uint32_t lv[16];
      tc::tmem_ld16(laddr + 64 * B, lv);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const long long iv = f32_small_int(__uint_as_float(lv[j]));
        if (L < 4) hi[j] += iv * (1ll << (7 * (3 - L)));
        else lo[j] += iv * (1ll << (7 * (7 - L)));
      }
    }
    if (!upper) {
      const int i = lrow - 64;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        xch[(i * 64 + 16 * cg16 + j) * 2] = hi[j];
        xch[(i * 64 + 16 * cg16 + j) * 2 + 1] = lo[j];
      }
    }
    __syncthreads();
    if (upper && lrow < k) {
      const int i = lrow;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 16 * cg16 + j;
        if (c >= i && c < k) {
          const long long H = hi[j] + xch[(i * 64 + c) * 2], Lo = lo[j] + xch[(i * 64 + c) * 2 + 1];
          tot[i * 65 + c] += oz_assemble_call(H, Lo, 28, E[i] + E[c] - 2056 - 49);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM, the exchange and E read before the next group overwrites them
  }
  if (bad && tid == 0) {
    atomicOr(a.pflags, JAC_DEVERR_TIMEOUT);
    tc::mbar_wait(&bar[0], it & 1);
  }
  tc::fence_before_sync();
  cluster.sync();
  const int totn = k * k, per = (totn + CS - 1) / CS;
  const int e0 = crank * per, e1 = min(totn, e0 + per);
  double* out = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = e0 + tid; e < e1; e += 512) {
    const int i = e % k, j = e / k;
    const int lo_ = min(i, j), hi_ = max(i, j);
    double part[16];  // all remote loads issued before the fixed-order sum
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) part[rk] = (rk < CS) ? cluster.map_shared_rank(tot, rk)[lo_ * 65 + hi_] : 0.0;
    double sum = 0.0;
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) sum += part[rk];
    out[j * a.apld + i] = sum;
  }
  cluster.sync();  // keep every partial alive until all remote reads are done
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

}  // namespace jac
