// ozaki.cu -- the FP64 Gram (Eq. (3.4)) and update (Algorithm 3.4) of a step, and a batched
// GEMM (the precision switch's V^T J V and G_in V, the backward's products), from exact FP16
// tensor-core digit products (ozaki.cuh).  Same grids, work split and results as k_gram /
// k_update (gram_update.cu) and k_gemm64 (dense.cu), to FP64 accuracy.
//
// Scale groups.  Gram X^T X: the columns of X over a stage of rows (each column is one row of
// A = X^T and one column of B = X).  Update Y = X V_P: the columns of X are first brought to a
// common size, X~ = X D^-1 and V~ = D V_P with D = diag(2^(c_k)) over the slab (exact, and only
// in the exponent arithmetic), then the rows of X~ and the columns of V~ are the groups.  A
// small column of G stays accurate relative to itself: its entries of V~ are small too.
#include <cooperative_groups.h>

#include <mutex>

#include "jacobi_common.cuh"
#include "ozaki.cuh"

namespace cg = cooperative_groups;

namespace jac {

__device__ __forceinline__ int oz_pair_col(int c, int wp, int op, int oq) { return c < wp ? op + c : oq + (c - wp); }

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------------------------ Gram
// Grid (half * CS, nprob), cluster (CS, 1, 1), 256 threads; the CS CTAs of a cluster split the
// rows of one pair as in k_gram.  A CTA takes its rows in stages of 128: warp w loads columns
// 8w..8w+7 (lane: rows 2 lane, 2 lane + 1, 64 + 2 lane, 65 + 2 lane), sets each column's bound
// exponent E_c over the stage, and stores the digits D[t][c][row].  The 20 upper 16 x 8 tiles of
// the 64 x 64 block go to the warps (at most 3 each) and are summed in FP64 across stages.
#define OZG_ROWS 128
#define OZG_NL 8  // levels kept: the Gram's groups are its own columns, bounds within ~4x of the terms
#define OZG_P (OZG_ROWS + 8)  // 272-byte digit rows: 16-byte aligned, ldmatrix conflict-free
struct OzGramSmem {
  __half D[OZ_T][JAC_KMAX][OZG_P];
  double C[JAC_KMAX][JAC_KMAX + 1];
  int E[JAC_KMAX];
};

// idx-th upper tile (8 tj + 7 >= 16 ti) of the 4 x 8 tile grid: ti = 0: tj 0..7, 1: 2..7,
// 2: 4..7, 3: 6..7
__device__ __forceinline__ void oz_upper_tile(int idx, int& ti, int& tj) {
  ti = (idx >= 18) ? 3 : (idx >= 14) ? 2 : (idx >= 8) ? 1 : 0;
  const int start = (ti == 0) ? 0 : (ti == 1) ? 8 : (ti == 2) ? 14 : 18;
  tj = 2 * ti + (idx - start);
}

__global__ void __launch_bounds__(256) k_gram_oz(const JacProb* __restrict__ probs, int s, int CS) {
  extern __shared__ __align__(16) unsigned char oz_raw[];
  OzGramSmem& sm = *reinterpret_cast<OzGramSmem*>(oz_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x / CS;
  const int crank = (int)cluster.block_rank();
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || (a.cached && a.cached[pair])) return;  // uniform
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int rpc = ((a.mp / CS + 15) & ~15);
  const int r_begin = min(a.mp, crank * rpc), r_end = min(a.mp, r_begin + rpc);

  double tot[3][4];
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) tot[u][v] = 0.0;

  for (int r0 = r_begin; r0 < r_end; r0 += OZG_ROWS) {
    const int rs = min(OZG_ROWS, r_end - r0);  // multiple of 16
    // ---- load the stage (all loads first), bound exponents, digits
    double2 x[8][2];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int c = 8 * warp + cc;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = 64 * i + 2 * lane;
        x[cc][i] = (c < k && r < rs)
                       ? __ldg(reinterpret_cast<const double2*>(a.Gw + (size_t)oz_pair_col(c, wp, op, oq) * a.mp + r0 + r))
                       : make_double2(0.0, 0.0);
      }
    }
    int ec[8];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      int e = max(max(oz_bexp(x[cc][0].x), oz_bexp(x[cc][0].y)), max(oz_bexp(x[cc][1].x), oz_bexp(x[cc][1].y)));
      ec[cc] = warp_max_i(e);
    }
    __syncthreads();  // the previous stage's digits and exponents are no longer read
    if (lane == 0) {
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) sm.E[8 * warp + cc] = ec[cc];
    }
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int c = 8 * warp + cc;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        __half d0[OZ_T], d1[OZ_T];
        oz_split(oz_fixed(x[cc][i].x, oz_bexp(x[cc][i].x) - ec[cc]), d0);
        oz_split(oz_fixed(x[cc][i].y, oz_bexp(x[cc][i].y) - ec[cc]), d1);
#pragma unroll
        for (int t = 0; t < OZ_T; ++t)
          *reinterpret_cast<unsigned*>(&sm.D[t][c][64 * i + 2 * lane]) = oz_h2(d0[t], d1[t]);
      }
    }
    __syncthreads();
    // ---- digit products of the upper tiles
    const int kend = (rs + 15) & ~15;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int idx = warp + 8 * u;
      if (idx >= 20) break;
      int ti, tj;
      oz_upper_tile(idx, ti, tj);
      float acc[OZG_NL][4];
#pragma unroll
      for (int L = 0; L < OZG_NL; ++L)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[L][v] = 0.0f;
      // ldmatrix rows: A (X^T, rows = columns i of the tile) and B (X, rows = columns j)
      const int arow = 16 * ti + (lane & 7) + 8 * ((lane >> 3) & 1), akof = 8 * (lane >> 4);
      const int brow = 8 * tj + (lane & 7), bkof = 8 * ((lane >> 3) & 1);
#pragma unroll 1
      for (int kk = 0; kk < kend; kk += 16) {
        unsigned fa[OZ_T][4], fb[OZ_T][2];
#pragma unroll
        for (int t = 0; t < OZ_T; ++t) {
          oz_ldsm4(fa[t], &sm.D[t][arow][kk + akof]);
          oz_ldsm2(fb[t][0], fb[t][1], &sm.D[t][brow][kk + bkof]);
        }
        oz_levels(acc, fa, fb);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = 16 * ti + g + 8 * (v >> 1), j = 8 * tj + 2 * t4 + (v & 1);
        tot[u][v] += oz_value(acc, v, sm.E[i] + sm.E[j] - 2056);
      }
    }
  }
  // ---- partial -> own shared memory: (i, j), j >= i, and its mirror
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int idx = warp + 8 * u;
    if (idx < 20) {
      int ti, tj;
      oz_upper_tile(idx, ti, tj);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = 16 * ti + g + 8 * (v >> 1), j = 8 * tj + 2 * t4 + (v & 1);
        if (j >= i) {
          sm.C[i][j] = tot[u][v];
          sm.C[j][i] = tot[u][v];
        }
      }
    }
  }
  cluster.sync();
  const int totn = k * k, per = (totn + CS - 1) / CS;
  const int e0 = crank * per, e1 = min(totn, e0 + per);
  double* out = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = e0 + tid; e < e1; e += 256) {
    const int i = e % k, j = e / k;
    double part[16];  // all remote loads issued before the fixed-order sum
#pragma unroll
    for (int rk = 0; rk < 16; ++rk)
      part[rk] = (rk < CS) ? cluster.map_shared_rank(&sm.C[0][0], rk)[i * (JAC_KMAX + 1) + j] : 0.0;
    double sum = 0.0;
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) sum += part[rk];
    out[j * a.apld + i] = sum;
  }
  cluster.sync();  // keep every partial alive until all remote reads are done
}

// ---------------------------------------------------------------------------------- update
// Grid (half, nslab, nprob), 256 threads; slab y covers 64 rows of Gw (y < gslabs) or of Vw, as
// in k_update: Y = X V_P in place.  Warp w loads slab columns 8w..8w+7 (lane: rows lane and
// lane + 32) and V_P columns 8w..8w+7 (lane: rows lane and lane + 32).
//   c_k  = bound exponent of slab column k (0: zero column),
//   Ea_r = max_k (ex(X[r][k]) - c_k)   (row group of X~),
//   Eb_c = max_k (ex(V[k][c]) + c_k)   (column group of V~, over k with c_k > 0),
//   Y[r][c] = 2^(Ea_r + Eb_c - 2056) sum_L 2^(-7 L) acc_L.
#define OZU_ROWS 64
#define OZU_NL 9  // levels kept: the update's row and column bounds can sit far above a term
#define OZU_P (JAC_KMAX + 8)  // 144-byte digit rows
struct OzUpdSmem {
  __half A[OZ_T][OZU_ROWS][OZU_P];  // digits of X~: [t][row][k]
  __half B[OZ_T][JAC_KMAX][OZU_P];  // digits of V~: [t][column][k]
  int cexp[JAC_KMAX];
  int rexp[OZU_ROWS];
  int vexp[JAC_KMAX];
};

#define OZ_NO_EXP (-100000)

__global__ void __launch_bounds__(256) k_update_oz(const JacProb* __restrict__ probs, int s, int gslabs) {
  extern __shared__ __align__(16) unsigned char oz_raw[];
  OzUpdSmem& sm = *reinterpret_cast<OzUpdSmem*>(oz_raw);
  const JacProb& a = probs[blockIdx.z];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || a.skip[pair]) return;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq, KP = (k + 15) & ~15;
  double* base;
  int ld, r0, rs;
  if ((int)blockIdx.y < gslabs) {
    base = a.Gw;
    ld = a.mp;
    r0 = blockIdx.y * OZU_ROWS;
    rs = min(OZU_ROWS, a.mp - r0);
  } else {
    if (!a.Vw) return;
    base = a.Vw;
    ld = a.np;
    r0 = (blockIdx.y - gslabs) * OZU_ROWS;
    rs = min(OZU_ROWS, a.np - r0);
  }
  if (rs <= 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const double* Vp = a.vp + (size_t)pair * a.apld * a.apld;
  if (tid < OZU_ROWS) sm.rexp[tid] = OZ_NO_EXP;
  // ---- loads (all issued before use)
  double x[8][2], v[8][2];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int c = 8 * warp + cc;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = lane + 32 * i;
      x[cc][i] = (c < k && r < rs) ? base[(size_t)oz_pair_col(c, wp, op, oq) * ld + r0 + r] : 0.0;
      v[cc][i] = (c < k && r < k) ? __ldg(Vp + (size_t)c * a.apld + r) : 0.0;
    }
  }
  // ---- column bounds of the slab (warp-local)
  int ce[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) ce[cc] = warp_max_i(max(oz_bexp(x[cc][0]), oz_bexp(x[cc][1])));
  if (lane == 0) {
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) sm.cexp[8 * warp + cc] = ce[cc];
  }
  __syncthreads();  // cexp and the rexp initialization visible
  // ---- row groups of X~
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    int m = OZ_NO_EXP;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int ex = oz_bexp(x[cc][i]);
      if (ex != 0) m = max(m, ex - ce[cc]);
    }
    if (m != OZ_NO_EXP) atomicMax(&sm.rexp[lane + 32 * i], m);
  }
  // ---- column groups of V~ (warp-local); the row index of V_P is a slab column
  const int ck0 = sm.cexp[lane], ck1 = sm.cexp[lane + 32];
  int eb[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int e0 = oz_bexp(v[cc][0]), e1 = oz_bexp(v[cc][1]);
    int m = OZ_NO_EXP;
    if (e0 != 0 && ck0 != 0) m = e0 + ck0;
    if (e1 != 0 && ck1 != 0) m = max(m, e1 + ck1);
    eb[cc] = warp_max_i(m);
  }
  if (lane == 0) {
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) sm.vexp[8 * warp + cc] = eb[cc];
  }
  __syncthreads();  // rexp complete
  // ---- digits of X~: row r, columns 8w..8w+7 as one 16-byte store per digit
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = lane + 32 * i, ea = sm.rexp[r];
    unsigned w[OZ_T][4];
#pragma unroll
    for (int cc = 0; cc < 8; cc += 2) {
      __half d0[OZ_T], d1[OZ_T];
      const int ex0 = oz_bexp(x[cc][i]), ex1 = oz_bexp(x[cc + 1][i]);
      oz_split(oz_fixed(x[cc][i], ex0 - ce[cc] - ea), d0);
      oz_split(oz_fixed(x[cc + 1][i], ex1 - ce[cc + 1] - ea), d1);
#pragma unroll
      for (int t = 0; t < OZ_T; ++t) w[t][cc >> 1] = oz_h2(d0[t], d1[t]);
    }
#pragma unroll
    for (int t = 0; t < OZ_T; ++t)
      *reinterpret_cast<uint4*>(&sm.A[t][r][8 * warp]) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
  // ---- digits of V~: column c, rows lane and lane + 32 (zero where the slab column is zero)
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int c = 8 * warp + cc;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int kr = lane + 32 * i, ck = i ? ck1 : ck0;
      __half d[OZ_T];
      const long long V = (ck != 0) ? oz_fixed(v[cc][i], oz_bexp(v[cc][i]) + ck - eb[cc]) : 0ll;
      oz_split(V, d);
#pragma unroll
      for (int t = 0; t < OZ_T; ++t) sm.B[t][c][kr] = d[t];
    }
  }
  __syncthreads();
  // ---- products: warp w takes row tile ti = w & 3 and column tiles 4 (w >> 2) .. + 3, two at a
  // time (one ldmatrix.x4 of B per digit covers both)
  const int ti = warp & 3;
  if (16 * ti >= rs) return;
  const int arow = 16 * ti + (lane & 7) + 8 * ((lane >> 3) & 1), akof = 8 * (lane >> 4);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int tj0 = 4 * (warp >> 2) + 2 * h;
    if (8 * tj0 >= KP) break;
    float acc0[OZU_NL][4], acc1[OZU_NL][4];
#pragma unroll
    for (int L = 0; L < OZU_NL; ++L)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc0[L][e] = 0.0f;
        acc1[L][e] = 0.0f;
      }
    const int bcol = 8 * tj0 + (lane & 7) + 8 * (lane >> 4), bkof = 8 * ((lane >> 3) & 1);
#pragma unroll 1
    for (int kk = 0; kk < KP; kk += 16) {
      unsigned fa[OZ_T][4], fb0[OZ_T][2], fb1[OZ_T][2];
#pragma unroll
      for (int t = 0; t < OZ_T; ++t) {
        unsigned r4[4];
        oz_ldsm4(fa[t], &sm.A[t][arow][kk + akof]);
        oz_ldsm4(r4, &sm.B[t][bcol][kk + bkof]);
        fb0[t][0] = r4[0];
        fb0[t][1] = r4[1];
        fb1[t][0] = r4[2];
        fb1[t][1] = r4[3];
      }
      oz_levels(acc0, fa, fb0);
      oz_levels(acc1, fa, fb1);
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 16 * ti + g + 8 * (e >> 1), c = 8 * (tj0 + hh) + 2 * t4 + (e & 1);
        if (r < rs && c < k) {
          const int E = sm.rexp[r] + sm.vexp[c] - 2056;
          base[(size_t)oz_pair_col(c, wp, op, oq) * ld + r0 + r] = hh ? oz_value(acc1, e, E) : oz_value(acc0, e, E);
        }
      }
    }
  }
}

size_t oz_gram_smem_bytes() { return sizeof(OzGramSmem); }
size_t oz_update_smem_bytes() { return sizeof(OzUpdSmem); }

// ------------------------------------------------------------------------------- GEMM
// C = op(A) diag(sb) op(B) - diag(dsub), the contract of k_gemm64 (dense.cu), from FP16 digit
// products: column-major, C is Mr x Nc, batch member blockIdx.z at element strides sa, sbb, sc;
//   transA = 1: op(A)[i][r] = A[i * lda + r], else A[r * lda + i];
//   transB = 1: op(B)[r][j] = B[r * ldb + j], else B[j * ldb + r];
//   sb: optional +-1 per r; dsub: optional, its sign subtracted on the diagonal;
//   sym = 1: C symmetric (Mr == Nc), entries j >= i computed and mirrored.
// K runs in segments of 256 (4 chunks of 64), each an exact FP32 level sum recombined into FP64.
// Per segment the scales are those of k_update_oz: c_r = bound exponent of column r of the CTA's
// op(A) rows, then the rows of op(A) D^-1 and the columns of D op(B) (D = diag(2^c_r)) are the
// scale groups, so a term is exact to 2^-53 of its own row and column sizes even when the columns
// of A (or rows of B) are graded.  Grid (ceil(Mr/64), ceil(Nc/32), batch), 256 threads: warp w
// computes row tile w & 3 (16 rows) and column tiles 2 (w >> 2) + {0, 1}.
#define OZM_TI 64
#define OZM_TJ 32
#define OZM_KC 64
#define OZM_SEG 256
#define OZM_P (OZM_KC + 8)
#define OZM_NL 9
struct OzGemmSmem {
  __half A[OZ_T][OZM_TI][OZM_P];  // digits of op(A) D^-1: [t][row][r]
  __half B[OZ_T][OZM_TJ][OZM_P];  // digits of D op(B): [t][column][r]
  int ck[OZM_SEG];                // c_r of the segment (0: zero column)
  int rexp[OZM_TI];
  int cexp[OZM_TJ];
};

__global__ void __launch_bounds__(256) k_gemm_oz(int Mr, int Nc, int K, const double* __restrict__ A, int lda,
                                                int transA, const double* __restrict__ B, int ldb,
                                                const int8_t* __restrict__ sb, const int8_t* __restrict__ dsub,
                                                double* __restrict__ C, int ldc, int sym, int transB, long long sa,
                                                long long sbb, long long sc) {
  extern __shared__ __align__(16) unsigned char oz_raw[];
  OzGemmSmem& sm = *reinterpret_cast<OzGemmSmem*>(oz_raw);
  A += (size_t)blockIdx.z * sa;
  B += (size_t)blockIdx.z * sbb;
  C += (size_t)blockIdx.z * sc;
  const int i0 = blockIdx.x * OZM_TI, j0 = blockIdx.y * OZM_TJ;
  if (sym && j0 + OZM_TJ - 1 < i0) return;  // no entry with j >= i
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int ai = tid >> 2, ar = tid & 3, bj = tid >> 3, br = tid & 7;  // 4 threads per row, 8 per column
  const bool rowok = i0 + ai < Mr, colok = j0 + bj < Nc;
  const int ti = warp & 3, tj0 = 2 * (warp >> 2);
  const int arow = 16 * ti + (lane & 7) + 8 * ((lane >> 3) & 1), akof = 8 * (lane >> 4);
  const int bcol = 8 * tj0 + (lane & 7) + 8 * (lane >> 4), bkof = 8 * ((lane >> 3) & 1);
  auto a_at = [&](int i, int r) -> double {  // op(A)[i0 + i][r], in range
    return transA ? A[(size_t)(i0 + i) * lda + r] : A[(size_t)r * lda + i0 + i];
  };
  auto b_at = [&](int j, int r) -> double {  // op(B)[r][j0 + j] with the sign sb_r, in range
    const double y = transB ? B[(size_t)r * ldb + j0 + j] : B[(size_t)(j0 + j) * ldb + r];
    return (sb && sb[r] < 0) ? oz_neg_if(y, true) : y;
  };
  float acc0[OZM_NL][4], acc1[OZM_NL][4];
  double res[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int e = 0; e < 4; ++e) res[h][e] = 0.0;
  for (int s0 = 0; s0 < K; s0 += OZM_SEG) {
    const int slen = min(OZM_SEG, K - s0);
    // ---- c_r: thread tid takes column r = s0 + tid of the CTA's op(A) rows
    {
      int c = 0;
      if (tid < slen) {
        const int imax = min(OZM_TI, Mr - i0);
#pragma unroll 16
        for (int i = 0; i < imax; ++i) c = max(c, oz_bexp(a_at(i, s0 + tid)));
      }
      __syncthreads();  // the previous segment's exponents are no longer read
      sm.ck[tid] = c;
    }
    __syncthreads();
    // ---- row groups of op(A) D^-1 and column groups of D op(B)
    {
      int ea = OZ_NO_EXP, eb = OZ_NO_EXP;
      if (rowok) {
#pragma unroll 16
        for (int r = ar; r < slen; r += 4) {
          const int ex = oz_bexp(a_at(ai, s0 + r));
          if (ex != 0) ea = max(ea, ex - sm.ck[r]);
        }
      }
      if (colok) {
#pragma unroll 16
        for (int r = br; r < slen; r += 8) {
          const int ex = oz_bexp(b_at(bj, s0 + r)), c = sm.ck[r];
          if (ex != 0 && c != 0) eb = max(eb, ex + c);
        }
      }
      ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, 1));
      ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, 2));
      eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
      eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
      eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 4));
      if (ar == 0) sm.rexp[ai] = ea;
      if (br == 0) sm.cexp[bj] = eb;
    }
    __syncthreads();
    const int my_ea = sm.rexp[ai], my_eb = sm.cexp[bj];
#pragma unroll
    for (int L = 0; L < OZM_NL; ++L)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc0[L][e] = 0.0f;
        acc1[L][e] = 0.0f;
      }
    for (int kc = 0; kc < slen; kc += OZM_KC) {
      // ---- chunk values (all loads first), digits
      double xa[16], xb[8];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int r = kc + ar + 4 * u;
        xa[u] = (rowok && r < slen) ? a_at(ai, s0 + r) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = kc + br + 8 * u;
        xb[u] = (colok && r < slen) ? b_at(bj, s0 + r) : 0.0;
      }
      __syncthreads();  // the previous chunk's digits are consumed
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int r = kc + ar + 4 * u;
        __half d[OZ_T];
        const int c = (r < slen) ? sm.ck[r] : 0;
        oz_split(oz_fixed(xa[u], oz_bexp(xa[u]) - c - my_ea), d);
#pragma unroll
        for (int t = 0; t < OZ_T; ++t) sm.A[t][ai][ar + 4 * u] = d[t];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = kc + br + 8 * u;
        __half d[OZ_T];
        const int c = (r < slen) ? sm.ck[r] : 0;
        oz_split(c != 0 ? oz_fixed(xb[u], oz_bexp(xb[u]) + c - my_eb) : 0ll, d);
#pragma unroll
        for (int t = 0; t < OZ_T; ++t) sm.B[t][bj][br + 8 * u] = d[t];
      }
      __syncthreads();
#pragma unroll 1
      for (int kk = 0; kk < OZM_KC; kk += 16) {
        unsigned fa[OZ_T][4], fb0[OZ_T][2], fb1[OZ_T][2];
#pragma unroll
        for (int t = 0; t < OZ_T; ++t) {
          unsigned r4[4];
          oz_ldsm4(fa[t], &sm.A[t][arow][kk + akof]);
          oz_ldsm4(r4, &sm.B[t][bcol][kk + bkof]);
          fb0[t][0] = r4[0];
          fb0[t][1] = r4[1];
          fb1[t][0] = r4[2];
          fb1[t][1] = r4[3];
        }
        oz_levels(acc0, fa, fb0);
        oz_levels(acc1, fa, fb1);
      }
    }
    // ---- the segment's exact level sums into FP64
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int il = 16 * ti + g + 8 * (e >> 1);
      const int jl0 = 8 * tj0 + 2 * t4 + (e & 1), jl1 = jl0 + 8;
      res[0][e] += oz_value(acc0, e, sm.rexp[il] + sm.cexp[jl0] - 2056);
      res[1][e] += oz_value(acc1, e, sm.rexp[il] + sm.cexp[jl1] - 2056);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = i0 + 16 * ti + g + 8 * (e >> 1), j = j0 + 8 * (tj0 + h) + 2 * t4 + (e & 1);
      if (i < Mr && j < Nc && (!sym || j >= i)) {
        double v = res[h][e];
        if (dsub && i == j) v -= (dsub[i] < 0) ? -1.0 : 1.0;
        C[(size_t)j * ldc + i] = v;
        if (sym && j > i) C[(size_t)i * ldc + j] = v;
      }
    }
}

size_t oz_gemm_smem_bytes() { return sizeof(OzGemmSmem); }

// Launch with the grid of k_gemm_oz; sets the kernel's shared-memory limit on first use per
// device (outside any stream capture: the solvers call it before capturing).
int oz_gemm_launch(int Mr, int Nc, int K, const double* A, int lda, int transA, const double* B, int ldb,
                   const int8_t* sb, const int8_t* dsub, double* C, int ldc, int sym, int transB, long long sa,
                   long long sbb, long long sc, int batch, cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
      if (cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(OzGemmSmem)) !=
          cudaSuccess)
        return 1;
      done[dev] = true;
    }
  }
  const dim3 grid((Mr + OZM_TI - 1) / OZM_TI, (Nc + OZM_TJ - 1) / OZM_TJ, batch);
  k_gemm_oz<<<grid, 256, sizeof(OzGemmSmem), st>>>(Mr, Nc, K, A, lda, transA, B, ldb, sb, dsub, C, ldc, sym, transB,
                                                    sa, sbb, sc);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace jac
