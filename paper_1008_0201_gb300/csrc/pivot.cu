// pivot.cu -- one pivot block per CTA: the square factor and the inner one-sided Jacobi.
//
// For the pair (p, q) of a step, with X = [G_p G_q] (m x k) and A_P = X^* X (from the gram
// kernel):
//  1. convergence statistics of A_P: rotate the block iff some |a_ij| > tol sqrt(a_ii a_jj);
//  2. the Cholesky factor P^T A_P P = R^* R (Sec. 3.2), unpivoted (HF), with diagonal pivoting
//     over the whole block (HFC) or J_P-sign-pivoted (Algorithm 3.3, HFSC: diagonal pivoting
//     inside the J = +1 part, then inside the Schur complement of the J = -1 part, whose columns
//     are then taken in reverse order);
//  3. the pointwise one-sided Jacobi on the columns of R with respect to J_P (Sec. 2.1, the
//     "one-sided manner" of Sec. 2.2), trigonometric rotations (Eq. (2.1)) for equal signs and
//     hyperbolic ones otherwise, with the tanh = +-1 guard of Sec. 3.2, repeated until an inner
//     sweep rotates nothing (full block algorithm);
//  4. V_P = P W Pi (rows permuted back as Algorithm 3.4 states; Pi = the reversed order of the
//     J = -1 columns of Algorithm 3.3), J_P-unitary to FP64 accuracy when requested.
//
// GB300 placement.  The inner rotations run in FP32, LPP lanes per column pair and every pair of
// an inner step at once, the columns held in registers (see phase 3).  To keep relative precision when A_P is nearly diagonal, the factor is carried as
//     A_P = D (I + E) D,   R = Dp + F,   W = I + Wd,
// where D = diag(fp32(sqrt(a_ii))) is fixed and only the deviations F, Wd are stored in FP32:
// every rotation Q is applied as F <- F Q + Dp (Q - I) and Wd <- Wd Q + (Q - I), so small
// entries keep their own relative precision and the angles need FP32 only.  The transform that
// is applied to G in FP64 must be J-unitary in FP64; it is corrected by Newton-Schulz,
//     V <- V - V J (V^T J V - J) / 2   (quadratic),
// whose residual M = V^T J V - J is formed in FP32 from the small Wd when max|Wd| <= 2^-20 and
// otherwise from FP16 digit products of Wd (oz_residual) or on the FP64 mma path (symmetric
// tiles only); the correction product itself is small and is formed in FP32.
#include "jacobi_common.cuh"
#include "ozaki.cuh"

namespace jac {

// Pivot capacity KM (largest k = w_p + w_q of the class); KM / 2 pair slots of LPP lanes each.
template <int KM, int LPP>
struct PivotSmem {
  static constexpr int LDF = KM;       // F, W column stride (floats)
  static constexpr int LDS = KM + 1;   // Cholesky matrix / FP32 scratch stride (floats)
  static constexpr int LDV = KM + 1;   // FP64 V / M stride
  static constexpr int NT = (KM / 2) * LPP;
  static constexpr int NW = NT / 32;
  static constexpr int P2 = KM / 2;    // pair slots
  static constexpr int MBS = 2 * KM + 8;  // mailbox slot: F and W column; +8 floats spreads banks
  static constexpr int LDD = KM + 8;   // digit rows of W (halves): 16-byte aligned, ldmatrix conflict-free
  static constexpr int LDC = KM + 8;   // Cholesky rows (floats, in the mailboxes): 8 mod 32
  double V[KM * LDV];   // A_P first, then V (physical coordinates), FP64
  union {
    double M[KM * LDV];           // FP64 residual (FP64 mma products)
    __half D[OZ_T][KM][LDD];      // digits of W = V - I by column (digit products)
  };
  double dlo[KM];       // V_ii - 1 - fl(V_ii - 1) (digit products)
  int dexp[KM];         // bound exponent of column c of W (digit products)
  float S[KM * LDS];    // Cholesky working matrix (upper triangle), later FP32 J M
  float F[KM * LDF];
  float W[KM * LDF];
  float Vf[KM * LDS];   // FP32 copy of V for the correction product
  float mb[2][P2 * MBS];  // column mailboxes of the inner sweep (double-buffered)
  int mphys[2][P2];
  float mcn[2][P2];
  float dd[KM];
  float fid[KM];        // fp32(1 / d_i)
  int perm[KM];
  int lpos[KM];
  int jphys[KM];
  int jloc[KM];
  float dg[2][KM];       // shifted Schur diagonal of the Cholesky steps (double-buffered)
  unsigned pkey[2][KM];  // pivot search keys of the Cholesky steps (double-buffered)
  int pres[KM / 2];      // block-oriented cross step: columns of block p (pivot order) per slot
  int ptrav[KM / 2];     // ... and of block q
  float red_f[NW][4];
  int red_i[NW][2];
  double trs[2];
  int piv;
  int bad;
};

template <int KM, int LPP>
__device__ __forceinline__ float block_max_f(float v, PivotSmem<KM, LPP>& sm, int slot) {
  constexpr int NW = PivotSmem<KM, LPP>::NW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sm.red_f[warp][slot] = v;
  __syncthreads();
  float r = 0.0f;
  for (int w = 0; w < NW; ++w) r = fmaxf(r, sm.red_f[w][slot]);
  __syncthreads();
  return r;
}

// sum over the LPP lanes of a pair slot (aligned lane groups)
template <int LPP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// entry r of a register-held column (row l R + u in lane l of the group), broadcast to the group;
// a select chain instead of a dynamic register index
template <int R>
__device__ __forceinline__ float col_entry(const float (&f)[R], int r, int group_lane0) {
  float v = f[0];
#pragma unroll
  for (int u = 1; u < R; ++u) v = ((r & (R - 1)) == u) ? f[u] : v;
  return __shfl_sync(0xffffffffu, v, group_lane0 + r / R);
}

// J-orthogonality residual M = V^T J V - J from digit products (ozaki.cuh).  With W = fl(V - I)
// column by column and l_i = (V_ii - 1) - W_ii exactly (TwoSum), V = I + W + diag(l) and
//   M = W^T J + J W + W^T J W + diag(2 J l) + diag(l) J W + W^T J diag(l)   (+ l^2 terms, dropped)
// The linear and diag(l) terms are elementwise FP64; W^T J W, of size |W|^2, runs on the digit
// path with the columns of W (over the k rows) as scale groups and J_r applied to the A digits
// by their sign bit.  So M is accurate to ~2^-53 |W|^2 + 2^-53 |W|, where the FP64 product
// V^T J V carries ~2^-53 |V|^2.  Writes S = fp32(J M) (zero outside k x k) and returns this
// thread's max |M_ij|.  Warp w prepares columns 8w..8w+7 (lane: rows lane, lane + 32).
template <int KM, int LPP>
__device__ float oz_residual(PivotSmem<KM, LPP>& sm, const double* Vs, int k, int KP) {
  using SM = PivotSmem<KM, LPP>;
  constexpr int NW = SM::NW, LDV = SM::LDV, LDS = SM::LDS;
  constexpr int RI = KM / 32;
  static_assert(NW * 8 == KM, "one warp per 8 columns");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  // ---- W, its column bounds and digits
  double w[8][RI];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int c = 8 * warp + cc;
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const int r = lane + 32 * i;
      double x = (r < k && c < k) ? Vs[c * LDV + r] : 0.0;
      if (r == c && r < k) {  // TwoSum(V_cc, -1)
        const double hi = x - 1.0, bv = hi - x, av = hi - bv;
        sm.dlo[c] = (x - av) + (-1.0 - bv);
        x = hi;
      }
      w[cc][i] = x;
    }
  }
  int ec[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    int e = 0;
#pragma unroll
    for (int i = 0; i < RI; ++i) e = max(e, oz_bexp(w[cc][i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    ec[cc] = e;
  }
  if (lane == 0) {
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) sm.dexp[8 * warp + cc] = ec[cc];
  }
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      __half d[OZ_T];
      oz_split(oz_fixed(w[cc][i], oz_bexp(w[cc][i]) - ec[cc]), d);
#pragma unroll
      for (int t = 0; t < OZ_T; ++t) sm.D[t][8 * warp + cc][lane + 32 * i] = d[t];
    }
  }
  __syncthreads();
  // ---- upper 16 x 8 tiles of W^T J W, then M and S
  float mloc = 0.0f;
  const int ntj = KP / 8, ntiles = (KP / 16) * ntj;
  for (int tile = warp; tile < ntiles; tile += NW) {
    const int ti = tile / ntj, tj = tile % ntj;
    if (8 * tj + 7 < 16 * ti) continue;
    float acc[OZ_T][4];
#pragma unroll
    for (int L = 0; L < OZ_T; ++L)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[L][v] = 0.0f;
    const int arow = 16 * ti + (lane & 7) + 8 * ((lane >> 3) & 1), akof = 8 * (lane >> 4);
    const int brow = 8 * tj + (lane & 7), bkof = 8 * ((lane >> 3) & 1);
    for (int kk = 0; kk < KP; kk += 16) {
      const int r0 = kk + 2 * t4;
      const unsigned slo = (sm.jphys[r0] < 0 ? 0x8000u : 0u) | (sm.jphys[r0 + 1] < 0 ? 0x80000000u : 0u);
      const unsigned shi = (sm.jphys[r0 + 8] < 0 ? 0x8000u : 0u) | (sm.jphys[r0 + 9] < 0 ? 0x80000000u : 0u);
      unsigned fa[OZ_T][4], fb[OZ_T][2];
#pragma unroll
      for (int t = 0; t < OZ_T; ++t) {
        oz_ldsm4(fa[t], &sm.D[t][arow][kk + akof]);
        fa[t][0] ^= slo;
        fa[t][1] ^= slo;
        fa[t][2] ^= shi;
        fa[t][3] ^= shi;
        oz_ldsm2(fb[t][0], fb[t][1], &sm.D[t][brow][kk + bkof]);
      }
      oz_levels(acc, fa, fb);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int x = 16 * ti + g + 8 * (v >> 1), j = 8 * tj + 2 * t4 + (v & 1);
      if (j < x) continue;  // (x, j), j >= x, covers the block; (j, x) is its mirror
      float sxj = 0.0f, sjx = 0.0f;
      if (x < k && j < k) {  // FP64 work kept to ~7 operations per entry (J by sign bits)
        const bool nx = sm.jphys[x] < 0, nj = sm.jphys[j] < 0;
        double m = oz_value(acc, v, sm.dexp[x] + sm.dexp[j] - 2056);
        if (x == j) {
          const double wxx = Vs[x * LDV + x] - 1.0, l = sm.dlo[x];
          m += oz_neg_if(wxx + wxx, nx);
          if (__double_as_longlong(l) << 1) m += oz_neg_if(2.0 * l * (1.0 + wxx), nx);
        } else {
          const double wxj = Vs[j * LDV + x], wjx = Vs[x * LDV + j];  // W[x][j], W[j][x]
          const double lx = sm.dlo[x], lj = sm.dlo[j];
          m += oz_neg_if(wjx, nj) + oz_neg_if(wxj, nx);
          if ((__double_as_longlong(lx) << 1) | (__double_as_longlong(lj) << 1))
            m += oz_neg_if(lx * wxj, nx) + oz_neg_if(lj * wjx, nj);
        }
        const float f = (float)m;
        mloc = fmaxf(mloc, fabsf(f));
        sxj = nx ? -f : f;  // (J M)[x][j]
        sjx = nj ? -f : f;  // (J M)[j][x]
      }
      sm.S[j * LDS + x] = sxj;
      sm.S[x * LDS + j] = sjx;
    }
  }
  return mloc;
}

// The pivot of one pair in one CTA.  Returns 0 when V_P was formed and the pair is to be updated,
// 2 when the block was handed over to the FP64 pivot kernel (A_P still in sm.V), 1 otherwise (no
// rotation, or a reported error); uniform over the CTA.  FUSED = false: A_P is read from the Gram kernel's output and
// V_P written for the update kernel.  FUSED = true (the fused step kernel): A_P is already in
// sm.V and V = I + W stays in shared memory (sm.Vf, sm.perm, sm.lpos) for the caller's update.
template <int KM, int LPP, bool FUSED>
__device__ __forceinline__ int pivot_block(PivotSmem<KM, LPP>& sm, const JacProb& a, int s, int pair,
                                           const PivotParams& pp) {
  using SM = PivotSmem<KM, LPP>;
  constexpr int NT = SM::NT, NW = SM::NW;
  constexpr int LDF = SM::LDF, LDS = SM::LDS, LDV = SM::LDV;
  unsigned* err = a.pflags;
  PairStat* stats = a.stats + (size_t)s * a.half;
  const long long t_start = clock64();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- 1. load A_P, scaled matrix E, statistics ----------------------------------------------
  // The A_P tile's address depends on the pair slot only: its loads (the whole KM x KM tile,
  // entries beyond k unused) are issued first, so that their latency overlaps the dependent
  // lookups of the pair's blocks below (pair table, block offsets: ~10k clocks per pivot when
  // they ran in sequence on GB300)
  constexpr int NLD = KM * KM / NT;
  static_assert(NLD * NT == KM * KM, "whole tile per thread set");
  double av[NLD];
  if constexpr (!FUSED) {
    const double* A = a.Ap + (size_t)pair * a.apld * a.apld;
#pragma unroll
    for (int u = 0; u < NLD; ++u) {
      const int e = tid + u * NT;
      av[u] = __ldg(A + (e / KM) * a.apld + e % KM);
    }
  }
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq, KP = (k + 15) & ~15;
  double* Vs = sm.V;
  if (k > KM) {  // the driver assigns classes by k; reported, never trapped
    if (tid == 0) {
      atomicOr(err, JAC_DEVERR_INNER_LIMIT);
      a.skip[pair] = 1;
    }
    return 1;
  }
  // the sign of this thread's column, needed after the first barrier
  const int jcol = (tid < k) ? a.Js[tid < wp ? op + tid : oq + (tid - wp)] : 0;
  if constexpr (!FUSED) {
#pragma unroll
    for (int u = 0; u < NLD; ++u) {
      const int e = tid + u * NT, r = e % KM, c = e / KM;
      if (r < k && c < k) Vs[c * LDV + r] = av[u];
    }
  }
  if (tid == 0) sm.bad = 0;
  __syncthreads();
  double tr = 0.0;
  if (tid < k) {
    sm.jloc[tid] = jcol;
    const double aii = Vs[tid * LDV + tid];
    if (!(aii > 0.0) || !(aii < 1.0e300)) atomicOr(&sm.bad, 1);
    const float d = sqrtf((float)aii);
    const double d2 = (double)d * (double)d;  // exact
    sm.dd[tid] = d;
    sm.fid[tid] = 1.0f / d;
    sm.perm[tid] = tid;
    // e_ii = a_ii / d_i^2 - 1 = (a_ii - d_i^2) / d_i^2: the difference is exact in FP64 (both
    // agree to FP32 accuracy), so one FP32 division rounds the result (no FP64 division, whose
    // latency is ~650 clocks on GB300)
    sm.S[tid * LDS + tid] = (float)(aii - d2) / (float)d2;
    tr = aii;
  }
  for (int e = tid; e < KM * LDF; e += NT) {
    sm.F[e] = 0.0f;
    sm.W[e] = 0.0f;
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) {
      atomicOr(err, JAC_DEVERR_NOTPD);
      a.skip[pair] = 1;
      PairStat st = {};
      st.evaluated = 1;
      stats[pair] = st;
    }
    return 1;
  }
  // off-diagonal e_ij = a_ij / (d_i d_j) in FP32: it is the scaled off-diagonal entry
  // |a_ij| / sqrt(a_ii a_jj) to FP32 accuracy, so it drives the statistics; only entries within
  // 2^-12 of the threshold are re-decided in FP64.
  const double tol = pp.tol > 0.0 ? pp.tol : fmax((double)a.n, pp.tol_m * sqrt((double)a.mp)) * pp.tol_eps;
  const float tolf = (float)tol;
  float mx = 0.0f, oc = 0.0f, od = 0.0f;
  int cnt = 0;
  // the whole KM x KM tile in a fixed, unrolled pattern (no division by k; the loads of the
  // iterations issue together), entries beyond k skipped
#pragma unroll
  for (int u = 0; u < NLD; ++u) {
    const int e = tid + u * NT, i = e % KM, j = e / KM;
    if (i >= k || j >= k || i == j) continue;
    const float aij = (float)Vs[j * LDV + i];
    const float eij = aij * sm.fid[i] * sm.fid[j];
    sm.S[j * LDS + i] = eij;
    if (i < j) {
      const float r = fabsf(eij);
      mx = fmaxf(mx, r);
      bool hit = r > tolf;
      if (fabsf(r - tolf) <= tolf * 2.44140625e-4f) {
        const double ad = Vs[j * LDV + i];
        hit = ad * ad > tol * tol * Vs[i * LDV + i] * Vs[j * LDV + j];
      }
      cnt += hit ? 1 : 0;
      const float a2 = aij * aij;
      if ((i < wp) != (j < wp)) oc += a2; else od += a2;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    oc += __shfl_xor_sync(0xffffffffu, oc, o);
    od += __shfl_xor_sync(0xffffffffu, od, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (warp < 2) tr = warp_sum_d(tr);  // k <= 64 diagonal entries live in warps 0 and 1
  if (lane == 0) {
    sm.red_f[warp][0] = mx;
    sm.red_f[warp][1] = oc;
    sm.red_f[warp][2] = od;
    sm.red_i[warp][0] = cnt;
    if (warp < 2) sm.trs[warp] = tr;
  }
  __syncthreads();
  mx = oc = od = 0.0f;
  cnt = 0;
  for (int w = 0; w < NW; ++w) {
    mx = fmaxf(mx, sm.red_f[w][0]);
    oc += sm.red_f[w][1];
    od += sm.red_f[w][2];
    cnt += sm.red_i[w][0];
  }
  PairStat st;
  st.max_scaled = (double)mx;
  st.off2_cross = (double)oc;
  st.off2_diag = (double)od;
  st.trace = sm.trs[0] + ((NW > 1 && k > 32) ? sm.trs[1] : 0.0);
  st.rotations = 0;
  st.inner_sweeps = 0;
  st.ns_steps = 0;
  st.active = (cnt > 0) ? 1 : 0;
  st.evaluated = 1;
  const long long t_stats = clock64();
  if (cnt == 0) {
    if (tid == 0) {
      a.skip[pair] = 1;
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = st.cyc[2] = st.cyc[3] = 0;
      stats[pair] = st;
    }
    return 1;
  }
  __syncthreads();  // red_* and the trace slots are reused below

  // ---- 2. scaled, optionally sign-pivoted Cholesky in FP32 -----------------------------------
  int npos = 0;
  for (int c = 0; c < k; ++c) npos += (sm.jloc[c] > 0) ? 1 : 0;  // J sorted: + block first
  __syncthreads();
  const bool signpiv = (pp.factor == 2), diagpiv = (pp.factor == 1);
  // Left-looking Cholesky of I + E with diagonal pivoting inside the sign groups, on unpermuted
  // storage: the pivot of step i is perm[i]; row i of R~ - I is kept by column index in Fr (the
  // scaled entries e_ab stay untouched in S).  Step i forms row i only: for every column c not
  // yet pivoted, (e_pc - sum_{l<i} R~_lp R~_lc) / r_ii, the sum split over TPC lanes of one warp
  // (rows l = t mod TPC) and combined by shuffles; the shifted Schur diagonal s_cc (dg) and the
  // search key of the next step are updated by the column's own thread, both double-buffered,
  // so one block barrier per step suffices.  Every step is a short dependent chain: the loads
  // that do not depend on the pivot are issued before the key reduction, and the sum runs over
  // all rows without predicates (rows >= i of Fr are zero; row i is written in step i only after
  // the shuffles of the warp that reads it, so its products are 0).
  constexpr int TPC = NT / KM, CPW = 32 / TPC, NU = KM / TPC, LDC = SM::LDC;
  static_assert(TPC * KM == NT && CPW * TPC == 32 && NU % 4 == 0, "TPC lanes of one warp per column");
  static_assert(2 * SM::P2 * SM::MBS >= KM * LDC, "Cholesky rows fit in the mailboxes");
  float* Fr = &sm.mb[0][0];  // row i at Fr[i * LDC + c]; LDC = 8 mod 32: a warp's loads hit 32 banks
  const int ct = lane / CPW, cc = warp * CPW + lane % CPW;  // share of the sum, column
  const bool pivsel = signpiv || diagpiv;
  // the key of column c for step i: the largest unscaled Schur diagonal d_c^2 (1 + s_cc) in the
  // sign group of step i (sign pivoting, Algorithm 3.3) or among all remaining columns (diagonal
  // pivoting, HFC), as the value's bits above the low 6 (order-preserving for v >= 0) and 63 - c,
  // so that one warp max-reduction yields the largest value, ties to the smaller index
  auto in_group = [&](int i, int c) { return c < k && (!signpiv || ((i < npos) ? (c < npos) : (c >= npos))); };
  auto key_of = [&](float d2, float s, int c) {
    const float v = fmaxf(d2 * (1.0f + s), 0.0f);
    return (__float_as_uint(v) & 0xFFFFFFC0u) | (unsigned)(63 - c);
  };
  for (int e = tid; e < KM * LDC; e += NT) Fr[e] = 0.0f;
  if (tid < KM) {
    const float s0 = (tid < k) ? sm.S[tid * LDS + tid] : 0.0f;
    sm.dg[0][tid] = s0;
    sm.dg[1][tid] = s0;
    sm.pkey[0][tid] = in_group(0, tid) ? key_of(sm.dd[tid] * sm.dd[tid], s0, tid) : 0u;
  }
  const bool colk = cc < k;
  const float ddc2 = colk ? sm.dd[cc] * sm.dd[cc] : 0.0f;
  bool pivd = !colk;  // this thread's column pivoted already (or absent)
  const float* fcol = Fr + ct * LDC + cc;
  const float* frow = Fr + ct * LDC;
  __syncthreads();
  for (int i = 0; i < k; ++i) {
    // independent of the pivot
    const int b = i & 1;
    const float dgc = sm.dg[b][cc];
    float fc[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) fc[u] = fcol[TPC * u * LDC];
    int p = i;
    if (pivsel) {
      const unsigned key = __reduce_max_sync(0xffffffffu, max(sm.pkey[b][lane], sm.pkey[b][lane + 32 < KM ? lane + 32 : lane]));
      p = 63 - (int)(key & 63u);
    }
    // dependent on the pivot
    const float sii = sm.dg[b][p];
    const float scp = sm.S[max(p, cc) * LDS + min(p, cc)];
    float fp[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) fp[u] = frow[TPC * u * LDC + p];
    const float piv1 = 1.0f + sii;
    // The scaled Schur pivot is 1 / (A~^-1)_pp >= 1 / kappa(A~).  Below 64 eps_32 the column is
    // in the span of the previous ones at the precision of this factorization: the block goes
    // to the FP64 pivot kernel (which tells an ill-conditioned block from a singular one).
    if (!(piv1 > 3.8146973e-6f)) {
      if (tid == 0) sm.bad = 1;
      break;  // uniform: every thread read the same pivot
    }
    pivd = pivd || (p == cc);
    const float rinv = rsqrtf(piv1);  // 1 / r
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
    for (int u = 0; u < NU; u += 4) {
      a0 = fmaf(fp[u], fc[u], a0);
      a1 = fmaf(fp[u + 1], fc[u + 1], a1);
      a2 = fmaf(fp[u + 2], fc[u + 2], a2);
      a3 = fmaf(fp[u + 3], fc[u + 3], a3);
    }
    float dot = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = CPW; o < 32; o <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    // row i of R~ - I (by column index), the Schur diagonal and the next step's key
    const float v = (scp - dot) * rinv;
    const float dn = fmaf(-v, v, dgc);
    const unsigned nk = (!pivd && in_group(i + 1, cc)) ? key_of(ddc2, dn, cc) : 0u;
    if (ct == 0) {
      if (!pivd) {
        Fr[i * LDC + cc] = v;
        sm.dg[b ^ 1][cc] = dn;
      }
      sm.pkey[b ^ 1][cc] = nk;
    } else if (ct == 1 && cc == 0) {
      const float r = piv1 * rinv;
      Fr[i * LDC + p] = __fdividef(sii, 1.0f + r);  // r - 1 without cancellation
      sm.perm[i] = p;
    }
    __syncthreads();
  }
  __syncthreads();
  if (sm.bad) {  // handed over to the FP64 pivot kernel, which decides on rank deficiency
    if (tid == 0) {
      a.skip[pair] = 2;
      atomicOr(err, JAC_DEVERR_HANDOVER);
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = clock64() - t_stats;
      st.cyc[2] = st.cyc[3] = 0;
      stats[pair] = st;
    }
    return 2;
  }
  // R = Dp + F in pivot order: F[c][r] = (R~ - I)[r][c] d_c, r <= c; then d and the signs in
  // pivot order, and the logical order of the inner sweep
  for (int e = tid; e < k * k; e += NT) {
    const int r = e % k, c = e / k;
    if (r <= c) {
      const int pc = sm.perm[c];
      sm.F[c * LDF + r] = Fr[r * LDC + pc] * sm.dd[pc];
    }
  }
  float d_new = 0.0f;
  int j_new = 0;
  if (tid < k) {
    d_new = sm.dd[sm.perm[tid]];
    j_new = sm.jloc[sm.perm[tid]];
  }
  __syncthreads();
  // block-oriented steps after the first of a sweep rotate only the cross pairs (one column of
  // block p, one of block q): block p's columns become the residents of the ring, block q's the
  // travelers, each in pivot order
  const bool cross_only = pp.oriented && s > 0;
  if (tid < SM::P2) {
    sm.pres[tid] = -1;
    sm.ptrav[tid] = -1;
  }
  __syncthreads();
  if (tid < k) {
    sm.dd[tid] = d_new;
    sm.jphys[tid] = j_new;
    if (diagpiv) {
      // diagonal pivoting mixes the signs: the output order puts the pivot-order columns back
      // on positions of their own sign (positives, then negatives, each in pivot order), so
      // that V_P^* J_P V_P = J_P in the block's local order (the reordering of HFC)
      const bool pos = j_new > 0;
      int rank = 0;
      for (int c = 0; c < tid; ++c) rank += ((sm.jloc[sm.perm[c]] > 0) == pos) ? 1 : 0;
      sm.lpos[pos ? rank : npos + rank] = tid;
    } else {
      sm.lpos[tid] = (signpiv && tid >= npos) ? (k - 1 - (tid - npos)) : tid;
    }
    if (cross_only) {
      const bool in_p = sm.perm[tid] < wp;
      int rank = 0;
      for (int c = 0; c < tid; ++c) rank += ((sm.perm[c] < wp) == in_p) ? 1 : 0;
      if (in_p) sm.pres[rank] = tid;
      else sm.ptrav[rank] = tid;
    }
  }
  __syncthreads();
  const long long t_chol = clock64();

  // ---- 3. inner one-sided Jacobi (FP32, shifted representation) -----------------------------
  // inner threshold: at most half the outer one (so that a pair flagged in FP64 is rotated in
  // FP32), at least the FP32 noise level of the shifted dot products
  const float tol_in = fmaxf(0.5f * tolf, 64.0f * 5.9604645e-8f * mx);
  // The columns live in registers: pair slot q (LPP lanes of a warp) holds a resident and a
  // traveler column, R rows per lane (row l R + u in lane l).  An inner sweep is a recursive
  // cross ordering of the KM positions: at group size g (KM/2, KM/4, ..., 1 slots) the
  // travelers of each group go round its ring of g slots, so every resident meets every
  // traveler of the group in g steps; then each group splits in two, its residents pairing among
  // themselves in the first half and its travelers in the second.  Every pair of positions
  // meets once in KM - 1 steps, and between steps each slot passes exactly one column to one
  // other slot through a shared-memory mailbox: one block barrier per step.  Positions >= k are
  // empty.  The logical order of Algorithm 3.3 (reversed J = -1 part) gives the initial
  // placement: position p is the resident of slot p (p < KM/2) or the traveler of slot p - KM/2.
  constexpr int R = KM / LPP, GP = 32 / LPP, P2 = SM::P2, MBS = SM::MBS;
  const int grp = lane / LPP, l = lane % LPP, slot = warp * GP + grp, lane0 = grp * LPP;
  int ci = cross_only ? sm.pres[slot] : ((slot < k) ? sm.lpos[slot] : -1);
  int cj = cross_only ? sm.ptrav[slot] : ((slot + P2 < k) ? sm.lpos[slot + P2] : -1);
  // block-oriented: one inner sweep; after the first step of an outer sweep only the ring of
  // its first level (every column of block p meets every column of block q once)
  const int g_last = cross_only ? P2 : 1;
  const int max_inner = pp.oriented ? 1 : JAC_INNER_MAX_SWEEPS;
  float fi[R], fj[R], wi[R], wj[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    fi[u] = (ci >= 0) ? sm.F[ci * LDF + l * R + u] : 0.0f;
    fj[u] = (cj >= 0) ? sm.F[cj * LDF + l * R + u] : 0.0f;
    wi[u] = 0.0f;
    wj[u] = 0.0f;
  }
  int total_rot = 0, inner = 0, buf = 0;
  for (inner = 0; inner < max_inner; ++inner) {
    // c = ||r||^2 - s^2 = 2 s F_cc + ||f||^2 of both columns, recomputed every inner sweep and
    // tracked through the rotations
    float cni, cnj;
    {
      float qi = 0.0f, qj = 0.0f;
#pragma unroll
      for (int u = 0; u < R; ++u) {
        qi = fmaf(fi[u], fi[u], qi);
        qj = fmaf(fj[u], fj[u], qj);
      }
      qi = group_sum<LPP>(qi);
      qj = group_sum<LPP>(qj);
      const float di = col_entry<R>(fi, ci >= 0 ? ci : 0, lane0);
      const float dj = col_entry<R>(fj, cj >= 0 ? cj : 0, lane0);
      cni = (ci >= 0) ? 2.0f * sm.dd[ci] * di + qi : 0.0f;
      cnj = (cj >= 0) ? 2.0f * sm.dd[cj] * dj + qj : 0.0f;
    }
    int my_rot = 0;       // per slot (uniform over its lanes)
    float my_max = 0.0f;  // largest scaled |a_ij| rotated
    for (int g = P2; g >= g_last; g >>= 1) {
      const int base = slot & ~(g - 1), pos = slot - base;
      for (int st_ = 0; st_ < g; ++st_) {
        // ---- rotate the pair (ci, cj) of this slot
        const bool act = (ci >= 0) && (cj >= 0);
        const int ii = act ? ci : 0, jj = act ? cj : 0;
        // what does not depend on the dot product first
        const float si = sm.dd[ii], sj = sm.dd[jj];
        const bool trig = sm.jphys[ii] == sm.jphys[jj];
        const float aii = fmaf(si, si, cni), ajj = fmaf(sj, sj, cnj);
        const float rs = rsqrtf(aii) * rsqrtf(ajj);
        // a_ij = (d_i e_i + f_i) . (d_j e_j + f_j) = s_i F_ij + s_j F_ji + f_i . f_j in one group
        // reduction: the cross terms enter the partial sums of the lanes that hold rows i and j
        // (predicated FMAs; fetching F_ij and F_ji from the owner lanes first costs a dependent
        // select chain and a shuffle per entry, ~11% of the step)
        float sij = 0.0f, xc = 0.0f;
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int row = l * R + u;
          sij = fmaf(fi[u], fj[u], sij);
          if (row == ii) xc = fmaf(si, fj[u], xc);
          if (row == jj) xc = fmaf(sj, fi[u], xc);
        }
        const float aij_all = group_sum<LPP>(sij + xc);
        if (act) {
          const float aij = aij_all;
          const float beta = fabsf(aij);
          const float scaled = beta * rs;
          if (scaled > tol_in) {
            ++my_rot;
            my_max = fmaxf(my_max, scaled);
            const float e = (aij < 0.0f) ? -1.0f : 1.0f;
            // One branch-free path for both kinds (sg = +1 trigonometric, -1 hyperbolic), so
            // that the slots of a warp never split on the sign pattern:
            //  trigonometric, Eq. (2.1): cot(2 phi) = (a_jj - a_ii) / (2 |a_ij|), i.e.
            //    t = sign(x) 2|a_ij| / (|x| + sqrt(x^2 + 4|a_ij|^2)),  x = a_jj - a_ii;
            //  hyperbolic: coth(2 phi) = -(a_ii + a_jj) / (2 |a_ij|), i.e.
            //    t = -2|a_ij| / (x + sqrt((x - 2|a_ij|)(x + 2|a_ij|))),  x = a_ii + a_jj,
            //    with the |tanh| < 1 guard of Sec. 3.2;
            // both evaluated after an exact power-of-two scaling of x and 2|a_ij| into [1, 4).
            // The square roots are x rsqrt(x): the angle needs FP32 accuracy only, the
            // rotation built from it is orthogonal (J-orthogonal) whatever t is.
            const float sg = trig ? 1.0f : -1.0f;
            const float x = trig ? (sj - si) * (sj + si) + (cnj - cni) : aii + ajj;
            const float mxv = fmaxf(fabsf(x), 2.0f * beta);
            const float sc = __int_as_float(0x7f000000 - (__float_as_int(mxv) & 0x7f800000));
            const float nu = x * sc, b2 = 2.0f * beta * sc;
            const float rr = trig ? fmaf(nu, nu, b2 * b2) : (nu - b2) * (nu + b2);
            const bool ok = rr > 0.0f;
            const float root = ok ? rr * rsqrtf(rr) : 0.0f;
            const float tm = __fdividef(b2, fabsf(nu) + root);
            float t = trig ? copysignf(tm, x) : (ok ? -tm : -1.0f);
            if (!trig && (!(fabsf(t) < 1.0f) || !((1.0f - t) * (1.0f + t) > 0.0f))) t = copysignf(0.9f, t);
            const float c = rsqrtf(fmaf(sg * t, t, 1.0f));  // cos or cosh
            const float s_ = t * c;                          // sin or sinh
            const float q11 = c, q12 = e * s_, q21 = -sg * e * s_;
            const float cm1 = -sg * __fdividef(s_ * s_, 1.0f + c);  // c - 1 without cancellation
            // a_ii' = a_ii - t |a_ij|, a_jj' = a_jj + t |a_ij| (trigonometric); both move by
            // t |a_ij| (hyperbolic: the J-trace is invariant)
            const float dci = -sg * t * beta, dcj = t * beta;
            // F <- F Q + Dp (Q - I), Wd <- Wd Q + (Q - I): the Dp (Q - I) / (Q - I) terms touch
            // rows i and j only
#pragma unroll
            for (int u = 0; u < R; ++u) {
              const int row = l * R + u;
              const float a_i = fi[u], a_j = fj[u], b_i = wi[u], b_j = wj[u];
              float nfi = fmaf(q11, a_i, q21 * a_j), nfj = fmaf(q11, a_j, q12 * a_i);
              float nwi = fmaf(q11, b_i, q21 * b_j), nwj = fmaf(q11, b_j, q12 * b_i);
              if (row == ii) {
                nfi += si * cm1;
                nfj += si * q12;
                nwi += cm1;
                nwj += q12;
              }
              if (row == jj) {
                nfi += sj * q21;
                nfj += sj * cm1;
                nwi += q21;
                nwj += cm1;
              }
              fi[u] = nfi;
              fj[u] = nfj;
              wi[u] = nwi;
              wj[u] = nwj;
            }
            cni += dci;
            cnj += dcj;
          }
        }
        // ---- pass one column on: the traveler round the ring, or at the end of the group's
        // ring its split (first half: traveler to slot + g/2, which sends back its resident)
        if (st_ < g - 1) {
          // ring step (uniform over the block): the traveler goes to the next slot of the group.
          // Row l * R + u of a column sits at u * LPP + l of its mailbox slot: the 8 lanes of a
          // slot write 32 consecutive bytes per u, and the 4 slots of a warp land on distinct
          // banks (lane-contiguous rows l * R + u put lanes l and l + 4 on the same banks)
          const int dst = base + ((pos + 1) & (g - 1));
          float* box = sm.mb[buf] + dst * MBS + l;
#pragma unroll
          for (int u = 0; u < R; ++u) {
            box[u * LPP] = fj[u];
            box[KM + u * LPP] = wj[u];
          }
          if (l == 0) {
            sm.mphys[buf][dst] = cj;
            sm.mcn[buf][dst] = cnj;
          }
          __syncthreads();
          const float* in = sm.mb[buf] + slot * MBS + l;
#pragma unroll
          for (int u = 0; u < R; ++u) {
            fj[u] = in[u * LPP];
            wj[u] = in[KM + u * LPP];
          }
          cj = sm.mphys[buf][slot];
          cnj = sm.mcn[buf][slot];
          buf ^= 1;
        } else if (g > g_last) {
          // end of the group's ring: its split (first half: traveler to slot + g/2, which sends
          // back its resident)
          const bool give_res = pos >= g / 2;
          const int dst = pos < g / 2 ? slot + g / 2 : slot - g / 2;
          float* box = sm.mb[buf] + dst * MBS + l;
#pragma unroll
          for (int u = 0; u < R; ++u) {
            box[u * LPP] = give_res ? fi[u] : fj[u];
            box[KM + u * LPP] = give_res ? wi[u] : wj[u];
          }
          if (l == 0) {
            sm.mphys[buf][dst] = give_res ? ci : cj;
            sm.mcn[buf][dst] = give_res ? cni : cnj;
          }
          __syncthreads();
          const float* in = sm.mb[buf] + slot * MBS + l;
          const int cin = sm.mphys[buf][slot];
          const float cnin = sm.mcn[buf][slot];
          if (give_res) {
#pragma unroll
            for (int u = 0; u < R; ++u) {
              fi[u] = in[u * LPP];
              wi[u] = in[KM + u * LPP];
            }
            ci = cin;
            cni = cnin;
          } else {
#pragma unroll
            for (int u = 0; u < R; ++u) {
              fj[u] = in[u * LPP];
              wj[u] = in[KM + u * LPP];
            }
            cj = cin;
            cnj = cnin;
          }
          buf ^= 1;
        }
      }
    }
    // sweep totals: one count per slot (its lane 0)
    int cnt = (l == 0) ? my_rot : 0;
    cnt = warp_sum_i(cnt);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_max = fmaxf(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
    if (lane == 0) {
      sm.red_i[warp][1] = cnt;
      sm.red_f[warp][2] = my_max;
    }
    __syncthreads();
    int tot = 0;
    float dmax = 0.0f;
    for (int w = 0; w < NW; ++w) {
      tot += sm.red_i[w][1];
      dmax = fmaxf(dmax, sm.red_f[w][2]);
    }
    __syncthreads();
    total_rot += tot;
    // done when nothing was rotated, or when every rotated pair was already so small that the
    // next sweep (quadratic convergence: off-diagonals ~ k delta^2) would find nothing above tol_in
    if (tot == 0 || (float)k * dmax * dmax <= tol_in) break;
  }
  if (!pp.oriented && inner >= JAC_INNER_MAX_SWEEPS && tid == 0) atomicOr(err, JAC_DEVERR_INNER_LIMIT);
  // W columns back to shared memory, physical coordinates
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (ci >= 0) sm.W[ci * LDF + l * R + u] = wi[u];
    if (cj >= 0) sm.W[cj * LDF + l * R + u] = wj[u];
  }
  __syncthreads();
  const long long t_inner = clock64();

  // ---- 4. V = I + Wd (physical coordinates), J-orthogonalized in FP64 if requested ----------
  float wm = 0.0f;
  for (int e = tid; e < KP * KP; e += NT) {
    const int r = e % KP, c = e / KP;
    const float w = (r < k && c < k) ? sm.W[c * LDF + r] : 0.0f;
    const bool diag = (r == c && r < k);
    const double v = oz_f2d(w);  // integer conversion: FP64 instructions are scarce on GB300
    Vs[c * LDV + r] = diag ? v + 1.0 : v;
    sm.Vf[c * LDS + r] = diag ? w + 1.0f : w;
    wm = fmaxf(wm, fabsf(w));
  }
  int ns = 0;
  bool ns_ok = true;
  if (pp.ns_mode) {
    ns_ok = false;
    wm = block_max_f<KM, LPP>(wm, sm, 3);  // includes the barrier after the V build
    const bool small_w = wm <= 9.5367431640625e-7f;  // 2^-20
    for (int it = 0; it < 3; ++it) {
      // residual M = V^T J V - J, J = diag(jphys) on rows and columns
      float mloc = 0.0f;
      if (it == 0 && small_w) {
        // V = I + Wd: M = Wd^T J + J Wd + Wd^T J Wd.  The linear part is exact in FP32 when it
        // cancels (Sterbenz) and rounds relative to itself otherwise; the quadratic part is at
        // most k 2^-40 and carries FP32 relative error.  Stored as fp32(J M) directly.
        for (int e = tid; e < KP * KP; e += NT) {
          const int x = e % KP, j = e / KP;
          float mv = 0.0f;
          if (x < k && j < k) {
            const float jx = (float)sm.jphys[x], jj = (float)sm.jphys[j];
            float quad = 0.0f;
            for (int r = 0; r < k; ++r) quad = fmaf(sm.W[x * LDF + r] * (float)sm.jphys[r], sm.W[j * LDF + r], quad);
            mv = (sm.W[x * LDF + j] * jj + jx * sm.W[j * LDF + x]) + quad;
          }
          mloc = fmaxf(mloc, fabsf(mv));
          sm.S[j * LDS + x] = (x < k) ? (float)sm.jphys[x] * mv : 0.0f;  // (J M)[x][j]
        }
      } else if (pp.oz) {
        mloc = oz_residual<KM, LPP>(sm, Vs, k, KP);
      } else {
        // FP64 mma, upper tiles (8 tj + 7 >= 16 ti) and the mirror of the strict lower part
        const int g = lane >> 2, t = lane & 3;
        const int ntj = KP / 8, ntiles = (KP / 16) * ntj;
        for (int tile = warp; tile < ntiles; tile += NW) {
          const int ti = tile / ntj, tj = tile % ntj;
          if (8 * tj + 7 < 16 * ti) continue;
          double c4[4] = {0.0, 0.0, 0.0, 0.0};
          for (int kq = 0; kq < KP; kq += 16) {
            double av[8], bv[4];
#pragma unroll
            for (int u = 0; u < 8; ++u) av[u] = Vs[(16 * ti + g + 8 * (u & 1)) * LDV + kq + 4 * t + (u >> 1)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = kq + 4 * t + u;
              const double v = Vs[(8 * tj + g) * LDV + r];
              bv[u] = (r < k && sm.jphys[r] < 0) ? -v : v;
            }
            dmma16816(c4, av, bv);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = 16 * ti + g + 8 * (u >> 1), j = 8 * tj + 2 * t + (u & 1);
            if (j < i) continue;  // written once, from the tile holding (j, i) ... (i, j), j >= i
            double v = c4[u];
            if (i == j && i < k) v -= (sm.jphys[i] < 0) ? -1.0 : 1.0;
            sm.M[j * LDV + i] = v;
            sm.M[i * LDV + j] = v;
          }
        }
        __syncthreads();
        for (int e = tid; e < KP * KP; e += NT) {
          const int x = e % KP, j = e / KP;
          const double mv = sm.M[j * LDV + x];
          mloc = fmaxf(mloc, (float)fabs(mv));
          sm.S[j * LDS + x] = (x < k) ? (float)((sm.jphys[x] < 0) ? -mv : mv) : 0.0f;
        }
      }
      const float mm = block_max_f<KM, LPP>(mloc, sm, 0);
      if (mm <= 4.0e-16f) {
        ns_ok = true;
        break;
      }
      // V <- V - V (J M) / 2: the correction is O(|M|), formed in FP32 from the FP32 copy of V;
      // each thread a 4 x CB block (rows rg + RG i, columns cg + CGN c) of the product, so a
      // shared-memory load feeds 4 or CB FMAs; the FP32 copy follows V in FP32
      {
        constexpr int RG = KM / 4, CGN = NT / RG, CB = KM / CGN;
        static_assert(RG * CGN == NT && CGN * CB == KM, "correction blocking");
        const int rg = tid % RG, cg = tid / RG;
        float sum[4][CB];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < CB; ++c) sum[i][c] = 0.0f;
        for (int x = 0; x < k; ++x) {
          float vf[4], sv[CB];
#pragma unroll
          for (int i = 0; i < 4; ++i) vf[i] = sm.Vf[x * LDS + rg + RG * i];
#pragma unroll
          for (int c = 0; c < CB; ++c) sv[c] = sm.S[(cg + CGN * c) * LDS + x];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < CB; ++c) sum[i][c] = fmaf(vf[i], sv[c], sum[i][c]);
        }
        __syncthreads();  // every read of Vf done
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            const int r = rg + RG * i, j = cg + CGN * c;
            if (r < KP && j < KP) {
              Vs[j * LDV + r] -= oz_f2d(0.5f * sum[i][c]);
              sm.Vf[j * LDS + r] -= 0.5f * sum[i][c];
            }
          }
      }
      ++ns;
      __syncthreads();
      // predicted residual after this step: quadratic term + FP32 rounding of the correction
      if (mm * mm + 1.0e-6f * mm <= 2.0e-16f) {
        ns_ok = true;
        break;
      }
    }
  } else {
    __syncthreads();
  }
  const long long t_ns = clock64();
  if (!ns_ok) {  // V is not J-unitary to FP64 accuracy after the step budget: FP64 pivot kernel
    if (tid == 0) {
      a.skip[pair] = 2;
      atomicOr(err, JAC_DEVERR_HANDOVER);
      st.rotations = total_rot;
      st.inner_sweeps = (inner < max_inner) ? inner + 1 : max_inner;
      st.ns_steps = ns;
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = t_chol - t_stats;
      st.cyc[2] = t_inner - t_chol;
      st.cyc[3] = t_ns - t_inner;
      stats[pair] = st;
    }
    return 2;
  }
  // V_P = P V Pi: V_P[perm[r]][l] = V[r][lpos[l]]
  if constexpr (!FUSED) {
    double* out = a.vp + (size_t)pair * a.apld * a.apld;
    for (int e = tid; e < KP * KP; e += NT) {
      const int r = e % KP, l = e / KP;
      double v = 0.0;
      int row = r;
      if (r < k && l < k) {
        v = Vs[sm.lpos[l] * LDV + r];
        row = sm.perm[r];
      }
      out[l * a.apld + row] = v;
    }
  }
  if (tid == 0) {
    a.skip[pair] = FUSED ? 3 : 0;  // 3: updated by the fused step kernel itself
    st.rotations = total_rot;
    st.inner_sweeps = (inner < max_inner) ? inner + 1 : max_inner;
    st.ns_steps = ns;
    st.cyc[0] = t_stats - t_start;
    st.cyc[1] = t_chol - t_stats;
    st.cyc[2] = t_inner - t_chol;
    st.cyc[3] = t_ns - t_inner;
    stats[pair] = st;
  }
  return 0;
}

// KM = 32: four CTAs per SM (shared memory allows four; the register cap keeps them resident, no
// spills), which the batched solves of many small pivots need; KM = 64: one CTA per SM
template <int KM, int LPP>
__global__ void __launch_bounds__((KM / 2) * LPP, KM == 32 ? 4 : 1)
    k_pivot(const JacProb* __restrict__ probs, int s, PivotParams pp) {
  extern __shared__ __align__(16) unsigned char pv_raw[];
  PivotSmem<KM, LPP>& sm = *reinterpret_cast<PivotSmem<KM, LPP>*>(pv_raw);
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s]) return;
  if (a.cached && a.cached[pair]) return;  // skip set, statistics kept (pair_cache.cu)
  pivot_block<KM, LPP, false>(sm, a, s, pair, pp);
}

// ---- the fused step kernel ---------------------------------------------------------------------
// One step of the FP32 sweeps for one pair in one CTA: the Gram block, the pivot and the block
// update, with X_P = [G_p G_q] read from global memory once and written once.  The m rows of X_P
// stay in shared memory from the Gram to the update, in the pivot's digit-product region (the
// FP32 sweeps never form the FP64 J-orthogonality residual); the rows of V go through the column
// mailboxes in chunks of 64.  Used when every problem of the launch has m <= FusedLayout::MF.
template <int KM, int LPP>
struct FusedLayout {
  using SM = PivotSmem<KM, LPP>;
  static constexpr int LDX = KM + 4;  // staged rows of X_P (floats; 16-byte aligned rows)
  static constexpr int LDB = KM + 4;  // V_P in FP32, row c = input column
  static constexpr int REGION = (int)((sizeof(SM::M) > sizeof(SM::D) ? sizeof(SM::M) : sizeof(SM::D)) / 4);
  static constexpr int MF = ((REGION - KM * LDB) / LDX) / 32 * 32;  // largest m
  static_assert(MF >= 32, "staging region");
  static_assert(2 * SM::P2 * SM::MBS >= 64 * LDX, "a 64-row chunk of V fits in the mailboxes");
};

template <int KM, int LPP>
__global__ void __launch_bounds__((KM / 2) * LPP, KM == 32 ? 3 : 1)  // KM = 32: no spills at 3 per SM
    k_step_fused(const JacProb* __restrict__ probs, int s, PivotParams pp) {
  using SM = PivotSmem<KM, LPP>;
  using FL = FusedLayout<KM, LPP>;
  constexpr int NT = SM::NT, LDS = SM::LDS, LDV = SM::LDV, LDX = FL::LDX, LDB = FL::LDB, MF = FL::MF;
  constexpr int CT = KM / 4;  // 4-column groups
  static_assert(NT % CT == 0 && NT / CT == 16, "16 row groups");
  extern __shared__ __align__(16) unsigned char pv_raw[];
  SM& sm = *reinterpret_cast<SM*>(pv_raw);
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s]) return;
  if (a.cached && a.cached[pair]) return;  // skip set, statistics kept (pair_cache.cu)
  const int tid = threadIdx.x, tx = tid % CT, ty = tid / CT;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq, m = a.mp;
  // the driver launches this kernel for the FP32 sweeps (no FP64 residual: the staging region is
  // free) within these bounds; anything else is reported, never trapped
  if (k > KM || m > MF || pp.ns_mode) {
    if (tid == 0) {
      atomicOr(a.pflags, JAC_DEVERR_INNER_LIMIT);
      a.skip[pair] = 1;
    }
    return;
  }
  auto pcol = [&](int c) { return c < wp ? op + c : oq + (c - wp); };
  float* Xs = reinterpret_cast<float*>(&sm.M[0]);  // [r][c], m rows
  float* Bs = Xs + MF * LDX;                       // [c][j]
  float* Vst = &sm.mb[0][0];                       // 64-row chunk of V, [r][c]

  // ---- 0. X_P into shared memory; A_P = X_P^T X_P in FP32 (FP64 storage for the pivot)
  {
    constexpr int NB = 16;  // loads in flight per thread
    for (int e0 = 0; e0 < k * m; e0 += NT * NB) {
      float v[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int e = e0 + u * NT + tid;  // consecutive threads: consecutive rows of a column
        v[u] = (e < k * m) ? __ldg(a.G32 + (size_t)pcol(e / m) * a.mp + e % m) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int e = e0 + u * NT + tid;
        if (e < k * m) Xs[(e % m) * LDX + e / m] = v[u];
      }
    }
  }
  __syncthreads();
  {
    // thread (ty, tx): rows RPT ty .. RPT ty + RPT - 1 and columns 4 tx .. 4 tx + 3 of A_P; the
    // entries (i, j) and (j, i) take the same products in the same order (exactly symmetric)
    constexpr int RPT = KM / 16;
    float acc[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    for (int r = 0; r < m; ++r) {
      const float* xr = Xs + r * LDX;
      const float4 xj = *reinterpret_cast<const float4*>(xr + 4 * tx);
      const float vj[4] = {xj.x, xj.y, xj.z, xj.w};
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const float xi = xr[RPT * ty + u];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xi, vj[v], acc[u][v]);
      }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = RPT * ty + u, j = 4 * tx + v;
        if (i < k && j < k) sm.V[j * LDV + i] = oz_f2d(acc[u][v]);
      }
  }
  // (pivot_block's first barrier publishes A_P)

  // ---- 1.-4. the pivot
  const int pr = pivot_block<KM, LPP, true>(sm, a, s, pair, pp);  // uniform
  if (pr == 2) {
    // handed over: the FP64 pivot kernel reads A_P from the Gram output, as after the Gram kernel
    double* A = a.Ap + (size_t)pair * a.apld * a.apld;
    for (int e = tid; e < k * k; e += NT) A[(e / k) * a.apld + e % k] = sm.V[(e / k) * LDV + e % k];
  }
  if (pr != 0) return;

  // ---- 5. [X_P; V rows] <- [X_P; V rows] V_P in FP32, V_P[perm[r]][l] = V[r][lpos[l]]
  __syncthreads();
  for (int e = tid; e < k * k; e += NT) {
    const int r = e % k, l = e / k;
    Bs[sm.perm[r] * LDB + l] = sm.Vf[sm.lpos[l] * LDS + r];
  }
  __syncthreads();
  // thread (ty, tx): rows 4 ty .. 4 ty + 3 of a 64-row chunk, columns 4 tx .. 4 tx + 3
  auto update_chunk = [&](const float* X, int rows, float* dst, int ld, int r0) {
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    for (int c = 0; c < k; ++c) {
      const float4 b = *reinterpret_cast<const float4*>(Bs + c * LDB + 4 * tx);
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float x = X[(4 * ty + u) * LDX + c];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(x, bv[v], acc[u][v]);
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = 4 * tx + v;
      if (j >= k) continue;
      float* col = dst + (size_t)pcol(j) * ld + r0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * ty + u < rows) col[4 * ty + u] = acc[u][v];
    }
  };
  for (int r0 = 0; r0 < m; r0 += 64) update_chunk(Xs + r0 * LDX, min(64, m - r0), a.G32, a.mp, r0);
  if (a.V32) {
    for (int r0 = 0; r0 < a.np; r0 += 64) {
      const int rows = min(64, a.np - r0);
      constexpr int NV = KM * 64 / NT;
      float v[NV];
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int e = u * NT + tid, c = e / 64, r = e % 64;
        v[u] = (c < k && r < rows) ? a.V32[(size_t)pcol(c) * a.np + r0 + r] : 0.0f;
      }
      __syncthreads();  // the previous chunk's reads of Vst are done
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int e = u * NT + tid;
        Vst[(e % 64) * LDX + e / 64] = v[u];
      }
      __syncthreads();
      update_chunk(Vst, rows, a.V32, a.np, r0);
    }
  }
}

// Lanes per pair slot of each pivot capacity: KM = 64 -> 8 lanes x 8 rows, 256 threads;
// KM = 32 -> 8 lanes x 4 rows, 128 threads.
constexpr int kLpp64 = 8, kLpp32 = 8;
static_assert(sizeof(PivotSmem<64, kLpp64>) <= 232448, "pivot shared memory above the 227 KB per-CTA limit");

int fused_step_max_rows(int km) {
  return km == 32 ? FusedLayout<32, kLpp32>::MF : FusedLayout<64, kLpp64>::MF;
}

size_t pivot_smem_bytes(int km) {
  return km == 32 ? sizeof(PivotSmem<32, kLpp32>) : sizeof(PivotSmem<64, kLpp64>);
}

// Host side of the two instantiations (a kernel template is launched from its own translation unit).
int pivot_set_attributes() {
  bool ok = cudaFuncSetAttribute(k_pivot<32, kLpp32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(PivotSmem<32, kLpp32>)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_pivot<64, kLpp64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PivotSmem<64, kLpp64>)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_step_fused<32, kLpp32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PivotSmem<32, kLpp32>)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_step_fused<64, kLpp64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PivotSmem<64, kLpp64>)) == cudaSuccess;
  return ok ? 0 : 1;
}

// Grid (max_half, nprob): one CTA per pivot block.
void pivot_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                  const PivotParams& pp) {
  if (km == 32)
    k_pivot<32, kLpp32><<<dim3(max_half, nprob), PivotSmem<32, kLpp32>::NT, sizeof(PivotSmem<32, kLpp32>), st>>>(
        probs, s, pp);
  else
    k_pivot<64, kLpp64><<<dim3(max_half, nprob), PivotSmem<64, kLpp64>::NT, sizeof(PivotSmem<64, kLpp64>), st>>>(
        probs, s, pp);
}

// Grid (max_half, nprob): one CTA per pair, the whole FP32 step (fused_step_max_rows bounds m).
void fused_step_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                       const PivotParams& pp) {
  if (km == 32)
    k_step_fused<32, kLpp32><<<dim3(max_half, nprob), PivotSmem<32, kLpp32>::NT, sizeof(PivotSmem<32, kLpp32>),
                               st>>>(probs, s, pp);
  else
    k_step_fused<64, kLpp64><<<dim3(max_half, nprob), PivotSmem<64, kLpp64>::NT, sizeof(PivotSmem<64, kLpp64>),
                               st>>>(probs, s, pp);
}

}  // namespace jac
