// tc_fp32.cu -- Gram block and block update of the FP32 sweeps on the fifth-generation tensor
// cores (tcgen05, accumulators in tensor memory), with the operand tiles staged by TMA.
//
// The FP32 sweeps of the mixed mode (Sec. 4: the outer Jacobi iteration is self-correcting, so
// early sweeps may use less accurate transforms as long as the transforms finally applied to G
// are (J-)unitary to working precision) form A_P = X_P^T X_P (Eq. (3.4)) and apply
// [G_p G_q] <- [G_p G_q] V_P (Algorithm 3.4) on an FP32 copy of G and V.  The tensor cores take
// TF32 operands (the top 19 bits of an FP32 word; the hardware truncates the rest), so each
// operand x is split as x = h + l, h = x with its low 13 bits cleared (exact), l = x - h (exact
// in FP32), and the products are summed as h h' + h l' + l h' (+ l l' in the Gram, where it
// costs nothing): about 2^-21 relative per product, FP32 accumulation in tensor memory.
//
// Gram (k_gram32_tc).  Grid (half * CS, 1), cluster (CS, 1, 1), 128 threads; the CS CTAs of a
//   cluster split the rows of one pair into ranges of multiples of 32.  Per stage of 32 rows, TMA
//   loads two 32 x 32 boxes of G32 (columns op.. and oq.. of the pair; 128-byte swizzle), which
//   are the K-major operand rows 0..63 (S); the threads write T = S - trunc(S) as rows 64..127.
//   One MMA per 8 rows of K with A = B = [S; T] (M = N = 128) accumulates
//   D = [S; T][S; T]^T, and A_P is the sum of its four 64 x 64 quadrants.  Six stage buffers,
//   loads four stages ahead (a refill waits for MMAs committed two stages earlier).  Partials
//   of the cluster are added through distributed shared memory.
// Update (k_update32_tc).  Grid (half, ysplit), 128 threads; a CTA takes consecutive 128-row
//   tiles of G32 (then V32).  TMA stages the raw tile (rows contiguous: eight 32 x 32 boxes);
//   tf32 operands must be K-major, so the threads transpose it into K-major h (X_h) and l
//   (overwriting the staged tile in place); V_P (FP64, from the pivot) is split into V_h, V_l
//   K-major once per CTA.  24 MMAs (M = 128, N = 64, K = 8) accumulate
//   X_h V_h + X_l V_h + X_h V_l, and the epilogue writes the tile back in place.
#include <cooperative_groups.h>

#include "jacobi_common.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace jac {

namespace {

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// operand slot (0..63: 32 columns of block p, then 32 of block q) of pair index c (< wp + wq)
__device__ __forceinline__ int tc_slot(int c, int wp) { return c < wp ? c : 32 + (c - wp); }

}  // namespace

// ------------------------------------------------------------------------------------ Gram
#define TG_NS 6                                  // stage buffers
#define TG_AHEAD (TG_NS - 2)                     // stages loaded ahead of the one consumed
#define TG_STAGE 16384                           // S (p box, q box) + T, 128 rows x 128 B
#define TG_CP_LD 65                              // partial row stride (floats)
#define TG_P1 (128 * TG_CP_LD * 4)                // epilogue column-half sums, over the stages
#define TG_SMEM (1024 + TG_NS * TG_STAGE + 256)      // partial Cp also over the stages (after P1)

size_t tc_gram32_smem_bytes() { return TG_SMEM; }

__global__ void __launch_bounds__(128) k_gram32_tc(const JacProb* __restrict__ probs, int s, int CS,
                                                   const __grid_constant__ CUtensorMap tmG) {
  extern __shared__ unsigned char tg_raw[];
  unsigned char* sm = align1k(tg_raw);
  // [64][TG_CP_LD] partial, read by the cluster's CTAs after the main loop: it lives in the stage
  // buffers (free by then), after the epilogue's P1
  float* Cp = reinterpret_cast<float*>(sm + TG_P1);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TG_NS * TG_STAGE);
  uint64_t* done = full + TG_NS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + TG_NS);
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
  const int rpc = ((a.mp / CS + 31) & ~31);
  const int r_begin = min(a.mp, crank * rpc), r_end = min(a.mp, r_begin + rpc);
  const int nst = (r_end - r_begin + 31) >> 5;
  if (tid == 0) {
    for (int i = 0; i < TG_NS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&done[i], 1);
    }
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmG);
  }
  if (warp == 0) tc::tmem_alloc(tslot, 128);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  auto issue = [&](int j) {
    unsigned char* st = sm + (j % TG_NS) * TG_STAGE;
    tc::mbar_arrive_expect_tx(&full[j % TG_NS], 8192);
    tc::tma_load_2d(st, &tmG, &full[j % TG_NS], r_begin + 32 * j, op);
    tc::tma_load_2d(st + 4096, &tmG, &full[j % TG_NS], r_begin + 32 * j, oq);
  };
  bool bad = false;  // a bounded wait gave up (uniform after each block vote)
  int issued = 0;    // stages whose TMA loads thread 0 has issued
  if (tid == 0)
    for (; issued < TG_AHEAD && issued < nst; ++issued) issue(issued);
  constexpr uint32_t idesc = tc::idesc_f32acc(tc::FMT_TF32, 128, 128, 0, 0);
  int i = 0;
  for (; i < nst; ++i) {
    const int slot = i % TG_NS;
    bool mine = false;
    if (tid == 0 && issued < nst) {  // refill the slot of stage i - 2 (its MMAs are done by now)
      const int j = issued;
      if (j >= TG_NS && !tc::mbar_wait(&done[j % TG_NS], ((j - TG_NS) / TG_NS) & 1)) mine = true;
      if (!mine) {
        issue(j);
        ++issued;
      }
    }
    if (!mine && !tc::mbar_wait(&full[slot], (i / TG_NS) & 1)) mine = true;
    if (!mine) {  // T = S - trunc(S), rows 64..127 of the stage
      const float4* S4 = reinterpret_cast<const float4*>(sm + slot * TG_STAGE);
      float4* T4 = reinterpret_cast<float4*>(sm + slot * TG_STAGE + 8192);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 v = S4[tid + 128 * u];
        T4[tid + 128 * u] = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
      }
    }
    tc::fence_proxy_async_smem();
    if (__syncthreads_or(mine)) {
      bad = true;
      break;
    }
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(sm + slot * TG_STAGE);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t d = tc::desc_sw128(sa + kk * 32, 16, 1024);
        tc::mma_tf32(tb, d, d, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&done[slot]);
    }
  }
  if (!bad && nst > 0) {
    const bool ok = tc::mbar_wait(&done[(nst - 1) % TG_NS], ((nst - 1) / TG_NS) & 1);
    if (__syncthreads_or(!ok)) bad = true;
  }
  if (bad && tid == 0) {  // drain what is still in flight (bounded): loads not consumed, last MMAs
    for (int j = i; j < issued; ++j) tc::mbar_wait(&full[j % TG_NS], (j / TG_NS) & 1);
    if (i > 0) tc::mbar_wait(&done[(i - 1) % TG_NS], ((i - 1) / TG_NS) & 1);
  }
  __syncthreads();  // the stage buffers (P1, Cp below) are quiet
  tc::fence_after_sync();
  if (!bad && nst > 0) {
    // rows i and 64 + i, columns b and 64 + b of D: first the column halves per lane
    float* P1 = reinterpret_cast<float*>(sm);  // [128][TG_CP_LD], over the free stage buffers
    const int row = 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t lo[16], hi[16];
      tc::tmem_ld16(tb + ((uint32_t)(32 * warp) << 16) + c0, lo);
      tc::tmem_ld16(tb + ((uint32_t)(32 * warp) << 16) + 64 + c0, hi);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) P1[row * TG_CP_LD + c0 + j] = __uint_as_float(lo[j]) + __uint_as_float(hi[j]);
    }
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 128) {
      const int i = e >> 6, j = e & 63;
      Cp[i * TG_CP_LD + j] = P1[i * TG_CP_LD + j] + P1[(64 + i) * TG_CP_LD + j];
    }
  } else {
    for (int e = tid; e < 64 * 64; e += 128) Cp[(e >> 6) * TG_CP_LD + (e & 63)] = 0.0f;
    if (bad && tid == 0) atomicOr(a.pflags, JAC_DEVERR_TIMEOUT);
  }
  tc::fence_before_sync();
  cluster.sync();
  const int tot = k * k, per = (tot + CS - 1) / CS;
  const int e0 = crank * per, e1 = min(tot, e0 + per);
  double* out = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = e0 + tid; e < e1; e += 128) {
    const int i = e % k, j = e / k;
    const int si = tc_slot(i, wp), sj = tc_slot(j, wp);
    float part[16];  // all remote loads issued before the fixed-order sum
#pragma unroll
    for (int rk = 0; rk < 16; ++rk)
      part[rk] = (rk < CS) ? cluster.map_shared_rank(Cp, rk)[si * TG_CP_LD + sj] : 0.0f;
    float sum = 0.0f;
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) sum += part[rk];
    out[j * a.apld + i] = (double)sum;
  }
  cluster.sync();  // keep every partial alive until all remote reads are done
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tb, 128);
}

// ---------------------------------------------------------------------------------- update
#define TU_X 32768                                // one 128 x 64 FP32 tile
#define TU_SMEM (1024 + 2 * TU_X + 2 * 16384 + 256)
#define TU_ROWS 128

size_t tc_update32_smem_bytes() { return TU_SMEM; }

__global__ void __launch_bounds__(128) k_update32_tc(const JacProb* __restrict__ probs, int s, int gtiles, int tpc,
                                                     const __grid_constant__ CUtensorMap tmG,
                                                     const __grid_constant__ CUtensorMap tmV) {
  extern __shared__ unsigned char tu_raw[];
  unsigned char* sm = align1k(tu_raw);
  unsigned char* Bst = sm;              // staged tile (TMA), then X_l in place: K-major, chunk c>>5 at 16 KB
  unsigned char* Xh = sm + TU_X;        // X_h, K-major
  unsigned char* Vh = sm + 2 * TU_X;    // V_h: 64 rows (N) x 64 (K), chunk c>>5 at 8 KB
  unsigned char* Vl = Vh + 16384;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Vl + 16384);  // [0] TMA, [1] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const JacProb& a = probs[blockIdx.z];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || a.skip[pair]) return;
  const int ntiles = gtiles + (a.V32 ? (a.np + TU_ROWS - 1) / TU_ROWS : 0);
  const int t_begin = blockIdx.y * tpc, t_end = min(ntiles, t_begin + tpc);
  if (t_begin >= t_end) return;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmG);
    tc::prefetch_tmap(&tmV);
  }
  if (warp == 0) tc::tmem_alloc(tslot, 64);
  // V_h, V_l: element (N slot j, K slot c) = V_P[c'][j'] for the pair indices c', j' of the
  // slots; zero where either slot is past its block
  {
    const double* V = a.vp + (size_t)pair * a.apld * a.apld;
    for (int e = tid; e < 64 * 64; e += 128) {
      const int j = e >> 6, c = e & 63;  // consecutive threads: consecutive K slots
      const int jp = (j < 32) ? (j < wp ? j : -1) : (j - 32 < wq ? wp + j - 32 : -1);
      const int cp = (c < 32) ? (c < wp ? c : -1) : (c - 32 < wq ? wp + c - 32 : -1);
      const float v = (jp >= 0 && cp >= 0) ? (float)V[(size_t)jp * a.apld + cp] : 0.0f;
      const uint32_t off = (c >> 5) * 8192 + tc::sw128_offset(j, c & 31, 4);
      *reinterpret_cast<float*>(Vh + off) = v;
      *reinterpret_cast<float*>(Vl + off) = v - tf32_hi(v);
    }
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  constexpr uint32_t idesc = tc::idesc_f32acc(tc::FMT_TF32, 128, 64, 0, 0);
  bool bad = false;
  int drain_tma = -1, drain_mma = -1;  // phases still in flight when a wait gave up
  // the staged tile's load: issued for the first tile here, for each next one as soon as the
  // current tile's MMAs (the last readers of the staged buffer) are done, so that it overlaps
  // the current tile's epilogue
  auto load_tile = [&](int t) {
    const bool isg = t < gtiles;
    const int r0 = (isg ? t : t - gtiles) * TU_ROWS;
    tc::mbar_arrive_expect_tx(&bar[0], TU_X);
    for (int cb = 0; cb < 2; ++cb)
      for (int rb = 0; rb < 4; ++rb)
        tc::tma_load_2d(Bst + cb * 16384 + rb * 4096, isg ? &tmG : &tmV, &bar[0], r0 + 32 * rb, cb ? oq : op);
  };
  if (tid == 0) load_tile(t_begin);
  for (int t = t_begin; t < t_end; ++t) {
    const int it = t - t_begin;
    const bool isg = t < gtiles;
    float* base = isg ? a.G32 : a.V32;
    const int ld = isg ? a.mp : a.np;
    const int r0 = (isg ? t : t - gtiles) * TU_ROWS;
    const int rows = min(TU_ROWS, (isg ? a.mp : a.np) - r0);
    bool mine = !tc::mbar_wait(&bar[0], it & 1);
    // thread: row r = tid, all 64 columns; staged element (r, c) of box (rb, cb) is box row
    // c & 31, element r & 31
    float x[64];
    if (!mine) {
      const int rb = tid >> 5, rr = tid & 31;
#pragma unroll
      for (int c = 0; c < 64; ++c)
        x[c] = *reinterpret_cast<const float*>(Bst + (c >> 5) * 16384 + rb * 4096 + tc::sw128_offset(c & 31, rr, 4));
    }
    if (__syncthreads_or(mine)) {
      bad = true;
      drain_tma = it;
      break;
    }
#pragma unroll
    for (int c = 0; c < 64; c += 4) {
      const uint32_t off = (c >> 5) * 16384 + tc::sw128_offset(tid, c & 31, 4);
      const float4 h = make_float4(tf32_hi(x[c]), tf32_hi(x[c + 1]), tf32_hi(x[c + 2]), tf32_hi(x[c + 3]));
      *reinterpret_cast<float4*>(Xh + off) = h;
      *reinterpret_cast<float4*>(Bst + off) = make_float4(x[c] - h.x, x[c + 1] - h.y, x[c + 2] - h.z, x[c + 3] - h.w);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sh = tc::smem_u32(Xh), sl = tc::smem_u32(Bst), vh = tc::smem_u32(Vh), vl = tc::smem_u32(Vl);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t ao = (kk >> 2) * 16384 + (kk & 3) * 32, bo = (kk >> 2) * 8192 + (kk & 3) * 32;
        tc::mma_tf32(tb, tc::desc_sw128(sh + ao, 16, 1024), tc::desc_sw128(vh + bo, 16, 1024), idesc, kk > 0);
        tc::mma_tf32(tb, tc::desc_sw128(sl + ao, 16, 1024), tc::desc_sw128(vh + bo, 16, 1024), idesc, 1u);
        tc::mma_tf32(tb, tc::desc_sw128(sh + ao, 16, 1024), tc::desc_sw128(vl + bo, 16, 1024), idesc, 1u);
      }
      tc::mma_commit(&bar[1]);
    }
    mine = !tc::mbar_wait(&bar[1], it & 1);
    if (__syncthreads_or(mine)) {
      bad = true;
      drain_mma = it;
      break;
    }
    tc::fence_after_sync();
    if (tid == 0 && t + 1 < t_end) load_tile(t + 1);  // the staged buffer is free again
    // epilogue: lane row 32 warp + lane, 64 columns -> the pair's columns of G32 / V32
    const int r = 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t v[16];
      tc::tmem_ld16(tb + ((uint32_t)(32 * warp) << 16) + c0, v);
      tc::tmem_wait_ld();
      if (r < rows) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int sj = c0 + j;
          const bool valid = (sj < 32) ? (sj < wp) : (sj - 32 < wq);
          if (valid) base[(size_t)((sj < 32) ? op + sj : oq + sj - 32) * ld + r0 + r] = __uint_as_float(v[j]);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM read before the next tile's MMAs overwrite it
    tc::fence_after_sync();
  }
  if (bad && tid == 0) {
    atomicOr(a.pflags, JAC_DEVERR_TIMEOUT);
    if (drain_tma >= 0) tc::mbar_wait(&bar[0], drain_tma & 1);
    if (drain_mma >= 0) tc::mbar_wait(&bar[1], drain_mma & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 64);
}

}  // namespace jac
