// pivot.cu -- one pivot block per CTA: the square factor and the inner one-sided Jacobi.
//
// For the pair (p, q) of a step, with X = [G_p G_q] (m x k) and A_P = X^* X (from the gram
// kernel):
//  1. convergence statistics of A_P: rotate the block iff some |a_ij| > tol sqrt(a_ii a_jj);
//  2. the Cholesky factor P^T A_P P = R^* R (Sec. 3.2), unpivoted (HF) or J_P-sign-pivoted
//     (Algorithm 3.3, HFSC: diagonal pivoting inside the J = +1 part, then inside the Schur
//     complement of the J = -1 part, whose columns are then taken in reverse order);
//  3. the pointwise one-sided Jacobi on the columns of R with respect to J_P (Sec. 2.1, the
//     "one-sided manner" of Sec. 2.2), trigonometric rotations (Eq. (2.1)) for equal signs and
//     hyperbolic ones otherwise, with the tanh = +-1 guard of Sec. 3.2, repeated until an inner
//     sweep rotates nothing (full block algorithm);
//  4. V_P = P W Pi (rows permuted back as Algorithm 3.4 states; Pi = the reversed order of the
//     J = -1 columns of Algorithm 3.3), J_P-unitary to FP64 accuracy when requested.
//
// GB300 placement.  The inner rotations run in FP32 (warp per column pair, up to 32 pairs at
// once).  To keep relative precision when A_P is nearly diagonal, the factor is carried as
//     A_P = D (I + E) D,   R = Dp + F,   W = I + Wd,
// where D = diag(fp32(sqrt(a_ii))) is fixed and only the deviations F, Wd are stored in FP32:
// every rotation Q is applied as F <- F Q + Dp (Q - I) and Wd <- Wd Q + (Q - I), so small
// entries keep their own relative precision and the angles need FP32 only.  The transform that
// is applied to G in FP64 must be J-unitary in FP64; it is corrected by Newton-Schulz,
//     V <- V - V J (V^T J V - J) / 2   (quadratic),
// whose residual M = V^T J V - J is formed in FP32 from the small Wd when max|Wd| <= 2^-20 and
// otherwise on the FP64 mma path (symmetric tiles only); the correction product itself is small
// and is formed in FP32.
#include "jacobi_common.cuh"

namespace jac {

// Pivot capacity KM (largest k = w_p + w_q of the class), KM / 32 rows of a column per lane,
// KM / 2 warps (one column pair each).
template <int KM>
struct PivotSmem {
  static constexpr int LDF = KM;       // F, W column stride (floats)
  static constexpr int LDS = KM + 1;   // Cholesky matrix / FP32 scratch stride (floats)
  static constexpr int LDV = KM + 1;   // FP64 V / M stride
  static constexpr int NW = KM / 2;
  double V[KM * LDV];   // A_P first, then V (physical coordinates), FP64
  double M[KM * LDV];   // FP64 residual
  float S[KM * LDS];    // Cholesky working matrix (upper triangle), later FP32 J M
  float F[KM * LDF];
  float W[KM * LDF];
  float Vf[KM * LDS];   // FP32 copy of V for the correction product
  float cn[KM];         // tracked c_i = ||r_i||^2 - s_i^2 of the inner sweep
  float dd[KM];
  float fid[KM];        // fp32(1 / d_i)
  int perm[KM];
  int lpos[KM];
  int jphys[KM];
  int jloc[KM];
  float red_f[NW][4];
  int red_i[NW][2];
  float4 rotp[NW];      // rotation of pair w in the current inner step: q11, q12, q21, q11-1
  int rflag[NW];
  float sijv[NW];
  double trs[2];
  int piv;
  int bad;
};

// a column slice held by one lane: rows lane*R .. lane*R + R - 1
template <int R>
struct Slice {
  float v[R];
};

template <int R>
__device__ __forceinline__ Slice<R> load_slice(const float* col, int lane) {
  Slice<R> x;
  if (R == 2) {
    const float2 t = reinterpret_cast<const float2*>(col)[lane];
    x.v[0] = t.x;
    x.v[R - 1] = t.y;
  } else {
    x.v[0] = col[lane];
  }
  return x;
}

template <int R>
__device__ __forceinline__ void store_slice(float* col, int lane, const Slice<R>& x) {
  if (R == 2)
    reinterpret_cast<float2*>(col)[lane] = make_float2(x.v[0], x.v[R - 1]);
  else
    col[lane] = x.v[0];
}

template <int KM>
__device__ __forceinline__ float block_max_f(float v, PivotSmem<KM>& sm, int slot) {
  constexpr int NW = KM / 2;
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

template <int KM>
__global__ void __launch_bounds__(KM * 16, 1)
    k_pivot(const JacProb* __restrict__ probs, int s, PivotParams pp) {
  constexpr int NT = KM * 16, NW = KM / 2, R = KM / 32;
  using SM = PivotSmem<KM>;
  constexpr int LDF = SM::LDF, LDS = SM::LDS, LDV = SM::LDV;
  extern __shared__ __align__(16) unsigned char pv_raw[];
  SM& sm = *reinterpret_cast<SM*>(pv_raw);
  const JacProb& a = probs[blockIdx.y];
  unsigned* err = a.pflags;
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s]) return;
  PairStat* stats = a.stats + (size_t)s * a.half;
  const long long t_start = clock64();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
    return;
  }

  // ---- 1. load A_P, scaled matrix E, statistics ----------------------------------------------
  const double* A = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = tid; e < k * k; e += NT) {
    const int i = e % k, j = e / k;
    Vs[j * LDV + i] = A[j * a.apld + i];
  }
  if (tid == 0) sm.bad = 0;
  __syncthreads();
  double tr = 0.0;
  if (tid < k) {
    const int col = tid < wp ? op + tid : oq + (tid - wp);
    sm.jloc[tid] = a.Js[col];
    const double aii = Vs[tid * LDV + tid];
    if (!(aii > 0.0) || !(aii < 1.0e300)) atomicOr(&sm.bad, 1);
    const float d = sqrtf((float)aii);
    const double id = 1.0 / (double)d;
    sm.dd[tid] = d;
    sm.fid[tid] = (float)id;
    sm.perm[tid] = tid;
    // e_ii = a_ii / d_i^2 - 1 in FP64 (cancellation), then rounded once
    sm.S[tid * LDS + tid] = (float)(aii * id * id - 1.0);
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
      stats[pair] = st;
    }
    return;
  }
  // off-diagonal e_ij = a_ij / (d_i d_j) in FP32: it is the scaled off-diagonal entry
  // |a_ij| / sqrt(a_ii a_jj) to FP32 accuracy, so it drives the statistics; only entries within
  // 2^-12 of the threshold are re-decided in FP64.
  const double tol = pp.tol > 0.0 ? pp.tol : fmax((double)a.n, pp.tol_m * sqrt((double)a.mp)) * pp.tol_eps;
  const float tolf = (float)tol;
  float mx = 0.0f, oc = 0.0f, od = 0.0f;
  int cnt = 0;
  for (int e = tid; e < k * k; e += NT) {
    const int i = e % k, j = e / k;
    if (i == j) continue;
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
  const long long t_stats = clock64();
  if (cnt == 0) {
    if (tid == 0) {
      a.skip[pair] = 1;
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = st.cyc[2] = st.cyc[3] = 0;
      stats[pair] = st;
    }
    return;
  }
  __syncthreads();  // red_* and the trace slots are reused below

  // ---- 2. scaled, optionally sign-pivoted Cholesky in FP32 -----------------------------------
  int npos = 0;
  for (int c = 0; c < k; ++c) npos += (sm.jloc[c] > 0) ? 1 : 0;  // J sorted: + block first
  if (tid < k) sm.jphys[tid] = sm.jloc[tid];
  __syncthreads();
  const bool signpiv = (pp.factor == 2);
  // S holds the trailing matrix in its upper triangle: U(a, b) = S[max(a,b) * LDS + min(a,b)]
  const int cx = tid % KM, cy = tid / KM;  // trailing update: column cx, rows i + 1 + cy + 16 u <= cx
  for (int i = 0; i < k; ++i) {
    if (signpiv) {
      // pivot: the largest unscaled Schur diagonal d_j^2 (1 + s_jj) in the sign group of step i
      if (warp == 0) {
        const int hi = (i < npos) ? npos : k;
        float best = -1.0f;
        int bj = i;
        for (int j = i + lane; j < hi; j += 32) {
          const float dj = sm.dd[j];
          const float v = dj * dj * (1.0f + sm.S[j * LDS + j]);
          if (v > best) {
            best = v;
            bj = j;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
          if (ob > best || (ob == best && oj < bj)) {
            best = ob;
            bj = oj;
          }
        }
        if (lane == 0) sm.piv = bj;
      }
      __syncthreads();
      const int pv = sm.piv;
      if (pv != i) {  // uniform
        // symmetric swap of rows/columns i and pv of the trailing matrix (upper storage), of
        // the computed rows of F (columns i and pv), and of the bookkeeping
        for (int tt = tid; tt < k; tt += NT) {
          if (tt > i && tt != pv) {
            const int a1 = tt * LDS + i;
            const int a2 = (tt > pv) ? tt * LDS + pv : pv * LDS + tt;
            const float x = sm.S[a1];
            sm.S[a1] = sm.S[a2];
            sm.S[a2] = x;
          }
          if (tt < i) {
            const float x = sm.F[i * LDF + tt];
            sm.F[i * LDF + tt] = sm.F[pv * LDF + tt];
            sm.F[pv * LDF + tt] = x;
          }
        }
        if (tid == 0) {
          float x = sm.S[i * LDS + i];
          sm.S[i * LDS + i] = sm.S[pv * LDS + pv];
          sm.S[pv * LDS + pv] = x;
          int y = sm.perm[i];
          sm.perm[i] = sm.perm[pv];
          sm.perm[pv] = y;
          float z = sm.dd[i];
          sm.dd[i] = sm.dd[pv];
          sm.dd[pv] = z;
          y = sm.jphys[i];
          sm.jphys[i] = sm.jphys[pv];
          sm.jphys[pv] = y;
        }
        __syncthreads();
      }
    }
    const float sii = sm.S[i * LDS + i];
    const float piv1 = 1.0f + sii;
    // The scaled Schur pivot is 1 / (A~^-1)_ii >= 1 / kappa(A~).  Below 64 eps_32 the column is
    // in the span of the previous ones at the precision of this factorization: the block goes
    // to the FP64 pivot kernel (which tells an ill-conditioned block from a singular one).
    if (!(piv1 > 3.8146973e-6f)) {
      if (tid == 0) sm.bad = 1;
      break;  // uniform: every thread read the same sii
    }
    const float r = sqrtf(piv1), ipiv = 1.0f / piv1;
    // row i of F~ and the trailing update read only row i of S, which this step does not write
    if (cy == 0 && cx > i && cx < k) sm.F[cx * LDF + i] = sm.S[cx * LDS + i] / r;
    if (tid == 0) sm.F[i * LDF + i] = sii / (1.0f + r);
    if (cx > i && cx < k) {
      const float sil = sm.S[cx * LDS + i] * ipiv;
      for (int jj = i + 1 + cy; jj <= cx; jj += NT / KM) sm.S[cx * LDS + jj] -= sil * sm.S[jj * LDS + i];
    }
    __syncthreads();
  }
  __syncthreads();
  if (sm.bad) {  // handed over to the FP64 pivot kernel, which decides on rank deficiency
    if (tid == 0) {
      a.skip[pair] = 2;
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = clock64() - t_stats;
      st.cyc[2] = st.cyc[3] = 0;
      stats[pair] = st;
    }
    return;
  }
  // R = Dp + F: scale the columns of F~ by dd; logical order of the inner sweep
  for (int e = tid; e < k * k; e += NT) {
    const int r = e % k, c = e / k;
    if (r <= c) sm.F[c * LDF + r] *= sm.dd[c];
  }
  if (tid < k) {
    const int l = tid;
    sm.lpos[l] = (signpiv && l >= npos) ? (k - 1 - (l - npos)) : l;
  }
  __syncthreads();
  const long long t_chol = clock64();

  // ---- 3. inner one-sided Jacobi (FP32, shifted representation) -----------------------------
  // inner threshold: at most half the outer one (so that a pair flagged in FP64 is rotated in
  // FP32), at least the FP32 noise level of the shifted dot products
  const float tol_in = fmaxf(0.5f * tolf, 64.0f * 5.9604645e-8f * mx);
  const int kk = k + (k & 1);
  // Each inner step runs in three phases separated by barriers:
  //   A: warp w forms the dot product r_i^T r_j of its pair (shifted: F_i^T F_j);
  //   B: warp 0, lane l, forms the rotation of pair l from a_ii, a_jj, a_ij: the scalar 2x2
  //      work of all pairs shares one instruction stream instead of one per warp;
  //   C: warp w applies its rotation to the columns of F and W.
  int total_rot = 0, inner = 0;
  const int P = kk / 2;
  for (inner = 0; inner < JAC_INNER_MAX_SWEEPS; ++inner) {
    // c_i = 2 s_i F_ii + ||f_i||^2 recomputed at the start of every inner sweep, tracked below
    for (int c = warp; c < k; c += NW) {
      const Slice<R> f = load_slice<R>(sm.F + c * LDF, lane);
      float sq = 0.0f;
#pragma unroll
      for (int u = 0; u < R; ++u) sq = fmaf(f.v[u], f.v[u], sq);
      sq = warp_sum(sq);
      if (lane == 0) sm.cn[c] = 2.0f * sm.dd[c] * sm.F[c * LDF + c] + sq;
    }
    __syncthreads();
    int my_rot = 0;       // warp 0, per lane: rotations of pair `lane` in this sweep
    float my_max = 0.0f;  // largest scaled |a_ij| rotated
    for (int st_ = 0; st_ < kk - 1; ++st_) {
      // ---- A
      int i = 0, j = 0;
      bool act = false;
      Slice<R> fi, fj;
      if (warp < P) {
        int li, lj;
        rr_inner_pair(kk, st_, warp, li, lj);
        act = lj < k;
        if (act) {
          i = sm.lpos[li];
          j = sm.lpos[lj];
          fi = load_slice<R>(sm.F + i * LDF, lane);
          fj = load_slice<R>(sm.F + j * LDF, lane);
          float sij = 0.0f;
#pragma unroll
          for (int u = 0; u < R; ++u) sij = fmaf(fi.v[u], fj.v[u], sij);
          sij = warp_sum(sij);
          if (lane == 0) sm.sijv[warp] = sij;
        }
      }
      __syncthreads();
      // ---- B
      if (warp == 0 && lane < P) {
        int rot = 0;
        float4 rp = make_float4(0.f, 0.f, 0.f, 0.f);
        int li, lj;
        rr_inner_pair(kk, st_, lane, li, lj);
        if (lj < k) {
          const int bi = sm.lpos[li], bj = sm.lpos[lj];
          const float si = sm.dd[bi], sj = sm.dd[bj];
          const float ci = sm.cn[bi], cj = sm.cn[bj];
          const float aij = si * sm.F[bj * LDF + bi] + sj * sm.F[bi * LDF + bj] + sm.sijv[lane];
          const float aii = fmaf(si, si, ci), ajj = fmaf(sj, sj, cj);
          const float beta = fabsf(aij);
          const float scaled = beta * rsqrtf(aii) * rsqrtf(ajj);
          if (scaled > tol_in) {
            rot = 1;
            ++my_rot;
            my_max = fmaxf(my_max, scaled);
            const float e = (aij < 0.0f) ? -1.0f : 1.0f;
            float dci, dcj;
            if (sm.jphys[bi] == sm.jphys[bj]) {
              // trigonometric, Eq. (2.1): cot(2 phi) = (a_jj - a_ii) / (2 |a_ij|), i.e.
              // t = sign(a_jj - a_ii) 2|a_ij| / (|a_jj - a_ii| + sqrt((a_jj - a_ii)^2 + 4|a_ij|^2)),
              // evaluated after an exact power-of-two scaling of both terms into [1, 4)
              const float num = (sj - si) * (sj + si) + (cj - ci);
              const float mxv = fmaxf(fabsf(num), 2.0f * beta);
              const float sc = __int_as_float(0x7f000000 - (__float_as_int(mxv) & 0x7f800000));
              const float nu = num * sc, b2 = 2.0f * beta * sc;
              const float den = fabsf(nu) + sqrtf(fmaf(nu, nu, b2 * b2));
              const float t = copysignf(__fdividef(b2, den), num);
              const float c = rsqrtf(fmaf(t, t, 1.0f));
              const float s_ = t * c;
              rp = make_float4(c, e * s_, -e * s_, -__fdividef(s_ * s_, 1.0f + c));
              dci = -t * beta;  // a_ii' = a_ii - t |a_ij|, a_jj' = a_jj + t |a_ij|
              dcj = t * beta;
            } else {
              // hyperbolic: coth(2 phi) = -(a_ii + a_jj) / (2 |a_ij|), i.e.
              // t = -2|a_ij| / (a_ii + a_jj + sqrt((a_ii + a_jj - 2|a_ij|)(a_ii + a_jj + 2|a_ij|))),
              // with the |tanh| < 1 guard of Sec. 3.2
              const float apd = aii + ajj;
              const float sc = __int_as_float(0x7f000000 - (__float_as_int(apd) & 0x7f800000));
              const float ap = apd * sc, b2 = 2.0f * beta * sc;
              const float r2 = (ap - b2) * (ap + b2);
              float t = (r2 > 0.0f) ? -__fdividef(b2, ap + sqrtf(r2)) : -1.0f;
              if (!(fabsf(t) < 1.0f) || !((1.0f - t) * (1.0f + t) > 0.0f)) t = copysignf(0.9f, t);
              const float ch = rsqrtf((1.0f - t) * (1.0f + t));
              const float sh = t * ch;
              rp = make_float4(ch, e * sh, e * sh, __fdividef(sh * sh, 1.0f + ch));
              dci = t * beta;  // both diagonals move by t |a_ij| (the J-trace is invariant)
              dcj = t * beta;
            }
            sm.cn[bi] = ci + dci;
            sm.cn[bj] = cj + dcj;
          }
        }
        sm.rotp[lane] = rp;
        sm.rflag[lane] = rot;
      }
      __syncthreads();
      // ---- C
      if (act && sm.rflag[warp]) {
        const float4 rp = sm.rotp[warp];
        const float q11 = rp.x, q12 = rp.y, q21 = rp.z, cm1 = rp.w;
        const float si = sm.dd[i], sj = sm.dd[j];
        Slice<R> nfi, nfj;
#pragma unroll
        for (int u = 0; u < R; ++u) {
          nfi.v[u] = fmaf(q11, fi.v[u], q21 * fj.v[u]);
          nfj.v[u] = fmaf(q11, fj.v[u], q12 * fi.v[u]);
        }
        // + Dp (Q - I): column i gets si (q11-1) at row i and sj q21 at row j; column j
        // gets si q12 at row i and sj (q22-1) at row j
        if (lane == i / R) {
          nfi.v[i % R] += si * cm1;
          nfj.v[i % R] += si * q12;
        }
        if (lane == j / R) {
          nfi.v[j % R] += sj * q21;
          nfj.v[j % R] += sj * cm1;
        }
        store_slice<R>(sm.F + i * LDF, lane, nfi);
        store_slice<R>(sm.F + j * LDF, lane, nfj);
        const Slice<R> wi = load_slice<R>(sm.W + i * LDF, lane), wj = load_slice<R>(sm.W + j * LDF, lane);
        Slice<R> nwi, nwj;
#pragma unroll
        for (int u = 0; u < R; ++u) {
          nwi.v[u] = fmaf(q11, wi.v[u], q21 * wj.v[u]);
          nwj.v[u] = fmaf(q11, wj.v[u], q12 * wi.v[u]);
        }
        if (lane == i / R) {
          nwi.v[i % R] += cm1;
          nwj.v[i % R] += q12;
        }
        if (lane == j / R) {
          nwi.v[j % R] += q21;
          nwj.v[j % R] += cm1;
        }
        store_slice<R>(sm.W + i * LDF, lane, nwi);
        store_slice<R>(sm.W + j * LDF, lane, nwj);
      }
      __syncthreads();
    }
    if (warp == 0) {
      const int tot_w = warp_sum_i(my_rot);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) my_max = fmaxf(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
      if (lane == 0) {
        sm.red_i[0][1] = tot_w;
        sm.red_f[0][2] = my_max;
      }
    }
    __syncthreads();
    const int tot = sm.red_i[0][1];
    const float dmax = sm.red_f[0][2];
    __syncthreads();
    total_rot += tot;
    // done when nothing was rotated, or when every rotated pair was already so small that the
    // next sweep (quadratic convergence: off-diagonals ~ k delta^2) would find nothing above tol_in
    if (tot == 0 || (float)k * dmax * dmax <= tol_in) break;
  }
  if (inner >= JAC_INNER_MAX_SWEEPS && tid == 0) atomicOr(err, JAC_DEVERR_INNER_LIMIT);
  const long long t_inner = clock64();

  // ---- 4. V = I + Wd (physical coordinates), J-orthogonalized in FP64 if requested ----------
  float wm = 0.0f;
  for (int e = tid; e < KP * KP; e += NT) {
    const int r = e % KP, c = e / KP;
    const float w = (r < k && c < k) ? sm.W[c * LDF + r] : 0.0f;
    const double v = (double)w + ((r == c && r < k) ? 1.0 : 0.0);
    Vs[c * LDV + r] = v;
    sm.Vf[c * LDS + r] = (float)v;
    wm = fmaxf(wm, fabsf(w));
  }
  int ns = 0;
  bool ns_ok = true;
  if (pp.ns_mode) {
    ns_ok = false;
    wm = block_max_f<KM>(wm, sm, 3);  // includes the barrier after the V build
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
      const float mm = block_max_f<KM>(mloc, sm, 0);
      if (mm <= 4.0e-16f) {
        ns_ok = true;
        break;
      }
      // V <- V - V (J M) / 2: the correction is O(|M|), formed in FP32 from the FP32 copy of V
      for (int e = tid; e < KP * KP; e += NT) {
        const int r = e % KP, j = e / KP;
        float sum = 0.0f;
        for (int x = 0; x < k; ++x) sum = fmaf(sm.Vf[x * LDS + r], sm.S[j * LDS + x], sum);
        Vs[j * LDV + r] -= 0.5 * (double)sum;
      }
      ++ns;
      __syncthreads();
      // predicted residual after this step: quadratic term + FP32 rounding of the correction
      if (mm * mm + 1.0e-6f * mm <= 2.0e-16f) {
        ns_ok = true;
        break;
      }
      for (int e = tid; e < KP * KP; e += NT) {
        const int r = e % KP, c = e / KP;
        sm.Vf[c * LDS + r] = (float)Vs[c * LDV + r];
      }
      __syncthreads();
    }
  } else {
    __syncthreads();
  }
  const long long t_ns = clock64();
  if (!ns_ok) {  // V is not J-unitary to FP64 accuracy after the step budget: FP64 pivot kernel
    if (tid == 0) {
      a.skip[pair] = 2;
      st.rotations = total_rot;
      st.inner_sweeps = inner + 1;
      st.ns_steps = ns;
      st.cyc[0] = t_stats - t_start;
      st.cyc[1] = t_chol - t_stats;
      st.cyc[2] = t_inner - t_chol;
      st.cyc[3] = t_ns - t_inner;
      stats[pair] = st;
    }
    return;
  }
  // V_P = P V Pi: V_P[perm[r]][l] = V[r][lpos[l]]
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
  if (tid == 0) {
    a.skip[pair] = 0;
    st.rotations = total_rot;
    st.inner_sweeps = inner + 1;
    st.ns_steps = ns;
    st.cyc[0] = t_stats - t_start;
    st.cyc[1] = t_chol - t_stats;
    st.cyc[2] = t_inner - t_chol;
    st.cyc[3] = t_ns - t_inner;
    stats[pair] = st;
  }
}

size_t pivot_smem_bytes(int km) { return km == 32 ? sizeof(PivotSmem<32>) : sizeof(PivotSmem<64>); }

// Host side of the two instantiations (a kernel template is launched from its own translation unit).
int pivot_set_attributes() {
  bool ok = cudaFuncSetAttribute(k_pivot<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(PivotSmem<32>)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_pivot<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PivotSmem<64>)) ==
        cudaSuccess;
  return ok ? 0 : 1;
}

// Grid (max_half, nprob): one CTA of km*16 threads per pivot block.
void pivot_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                  const PivotParams& pp) {
  if (km == 32)
    k_pivot<32><<<dim3(max_half, nprob), 32 * 16, sizeof(PivotSmem<32>), st>>>(probs, s, pp);
  else
    k_pivot<64><<<dim3(max_half, nprob), 64 * 16, sizeof(PivotSmem<64>), st>>>(probs, s, pp);
}

}  // namespace jac
