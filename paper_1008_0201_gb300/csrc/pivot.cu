// pivot.cu -- one pivot block per CTA: the square factor and the inner one-sided Jacobi.
//
// For the pair (p, q) of a step, with X = [G_p G_q] (m x k) and A_P = X^* X (from k_gram):
//  1. convergence statistics of A_P: rotate the block iff some |a_ij| > tol sqrt(a_ii a_jj);
//  2. the Cholesky factor P^T A_P P = R^* R (Sec. 3.2), unpivoted (HF) or J_P-sign-pivoted
//     (Algorithm 3.3, HFSC: diagonal pivoting inside the J = +1 part, then inside the Schur
//     complement of the J = -1 part, whose columns are then taken in reverse order);
//  3. the pointwise one-sided Jacobi on the columns of R with respect to J_P (Sec. 2.1, the
//     "one-sided manner" of Sec. 2.2), trigonometric rotations (Eq. (2.1)) for equal signs and
//     hyperbolic ones otherwise, with the tanh = +-1 guard of Sec. 3.2, repeated until an inner
//     sweep rotates nothing (full block algorithm);
//  4. V_P = P W (rows permuted back, Algorithm 3.4), made J_P-unitary to FP64 accuracy.
//
// GB300 placement: the inner rotations run in FP32 (warp per column pair, 32 pairs at once).
// To keep relative precision when A_P is nearly diagonal, the factor is carried as
//     A_P = D (I + E) D,   R = Dp + F,   W = I + Wd,
// where D = diag(fp32(sqrt(a_ii))) is fixed, E is formed in FP64 and rounded once, and only the
// deviations F, Wd are stored in FP32: every rotation is applied as F <- F Q + Dp (Q - I) and
// Wd <- Wd Q + (Q - I), so the small entries keep their own relative precision.  Rotation
// angles therefore only need FP32; the transform applied to G must be J-unitary in FP64, which
// the Newton-Schulz correction V <- V - V J (V^* J V - J) / 2 gives (quadratic; run on the FP64
// mma path until the residual is at rounding level).
#include "jacobi_common.cuh"

namespace jac {

#define PV_KM JAC_KMAX
#define PV_LDF JAC_KMAX        // F, W column stride (floats)
#define PV_LDS (JAC_KMAX + 1)  // Cholesky working matrix stride (floats)
#define PV_LDV (JAC_KMAX + 1)  // FP64 V stride
#define PV_LDM (JAC_KMAX + 1)  // FP64 M / T stride
#define PV_THREADS 1024
#define PV_WARPS 32

struct PivotSmem {
  double V[PV_KM * PV_LDV];   // A_P first (ld PV_LDV), then V_P
  double M[PV_KM * PV_LDM];
  double T[PV_KM * PV_LDM];
  float S[PV_KM * PV_LDS];
  float F[PV_KM * PV_LDF];
  float W[PV_KM * PV_LDF];
  double inva[PV_KM];
  double invd[PV_KM];
  float dd[PV_KM];
  int perm[PV_KM];
  int lpos[PV_KM];
  int jphys[PV_KM];
  int jloc[PV_KM];
  double red_d[PV_WARPS][4];
  int red_i[PV_WARPS];
  int piv;
  int bad;
};

__device__ __forceinline__ void rr_inner_pair(int kk, int s, int w, int& li, int& lj) {
  // circle method on kk (even) positions: position kk-1 fixed
  const int L = kk - 1;
  if (w == 0) {
    li = s;
    lj = kk - 1;
  } else {
    int x = (s + w) % L, y = (s - w + L) % L;
    li = min(x, y);
    lj = max(x, y);
  }
}

// C(i,j) = sum_r A(i,r) B(r,j) for 0 <= i, j < KP on the FP64 mma path, one 16x8 tile per warp
// per iteration.  la/lb read shared memory, sc stores.
template <class LA, class LB, class SC>
__device__ __forceinline__ void cta_dmma(int KP, LA la, LB lb, SC sc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ntj = KP / 8, ntiles = (KP / 16) * ntj;
  for (int tile = warp; tile < ntiles; tile += PV_WARPS) {
    const int ti = tile / ntj, tj = tile % ntj;
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int kk = 0; kk < KP; kk += 16) {
      double av[8], bv[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) av[i] = la(16 * ti + g + 8 * (i & 1), kk + 4 * t + (i >> 1));
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = lb(kk + 4 * t + j, 8 * tj + g);
      dmma16816(c, av, bv);
    }
    sc(16 * ti + g, 8 * tj + 2 * t, c[0]);
    sc(16 * ti + g, 8 * tj + 2 * t + 1, c[1]);
    sc(16 * ti + g + 8, 8 * tj + 2 * t, c[2]);
    sc(16 * ti + g + 8, 8 * tj + 2 * t + 1, c[3]);
  }
}

__global__ void __launch_bounds__(PV_THREADS, 1)
    k_pivot(JacStepArgs a, const int* __restrict__ step_pairs, const int* __restrict__ step_count,
            const double* __restrict__ Ap, PivotParams pp, double* __restrict__ vp, int* __restrict__ skip,
            PairStat* __restrict__ stats, unsigned* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char pv_raw[];
  PivotSmem& sm = *reinterpret_cast<PivotSmem*>(pv_raw);
  const int pair = blockIdx.x;
  if (pair >= *step_count) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p = step_pairs[2 * pair], q = step_pairs[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq, KP = (k + 15) & ~15;
  double* Vs = sm.V;

  // ---- 1. load A_P, statistics -------------------------------------------------------------
  const double* A = Ap + (size_t)pair * JAC_KMAX * JAC_KMAX;
  for (int e = tid; e < k * k; e += PV_THREADS) {
    const int i = e % k, j = e / k;
    Vs[j * PV_LDV + i] = A[j * JAC_KMAX + i];
  }
  if (tid < k) {
    const int col = tid < wp ? op + tid : oq + (tid - wp);
    sm.jloc[tid] = a.Js[col];
  }
  if (tid == 0) sm.bad = 0;
  __syncthreads();
  if (tid < k) {
    const double aii = Vs[tid * PV_LDV + tid];
    if (!(aii > 0.0) || !(aii < 1.0e300)) atomicOr(&sm.bad, 1);
    sm.inva[tid] = 1.0 / aii;
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) {
      atomicOr(err, JAC_DEVERR_NOTPD);
      skip[pair] = 1;
      PairStat st = {};
      stats[pair] = st;
    }
    return;
  }
  const double tol2 = pp.tol * pp.tol;
  double mx = 0.0, oc = 0.0, od = 0.0, tr = 0.0;
  int cnt = 0;
  for (int e = tid; e < k * k; e += PV_THREADS) {
    const int i = e % k, j = e / k;
    if (i < j) {
      const double aij = Vs[j * PV_LDV + i];
      const double a2 = aij * aij;
      const double r2 = a2 * sm.inva[i] * sm.inva[j];
      mx = fmax(mx, r2);
      cnt += (r2 > tol2) ? 1 : 0;
      if ((i < wp) != (j < wp)) oc += a2; else od += a2;
    } else if (i == j) {
      tr += Vs[j * PV_LDV + i];
    }
  }
  mx = warp_max_d(mx);
  oc = warp_sum_d(oc);
  od = warp_sum_d(od);
  tr = warp_sum_d(tr);
  cnt = warp_sum_i(cnt);
  if (lane == 0) {
    sm.red_d[warp][0] = mx;
    sm.red_d[warp][1] = oc;
    sm.red_d[warp][2] = od;
    sm.red_d[warp][3] = tr;
    sm.red_i[warp] = cnt;
  }
  __syncthreads();
  mx = 0.0;
  oc = od = tr = 0.0;
  cnt = 0;
  for (int w = 0; w < PV_WARPS; ++w) {
    mx = fmax(mx, sm.red_d[w][0]);
    oc += sm.red_d[w][1];
    od += sm.red_d[w][2];
    tr += sm.red_d[w][3];
    cnt += sm.red_i[w];
  }
  PairStat st;
  st.max_scaled = sqrt(mx);
  st.off2_cross = oc;
  st.off2_diag = od;
  st.trace = tr;
  st.rotations = 0;
  st.inner_sweeps = 0;
  st.ns_steps = 0;
  st.active = (cnt > 0) ? 1 : 0;
  if (cnt == 0) {
    if (tid == 0) {
      skip[pair] = 1;
      stats[pair] = st;
    }
    return;
  }

  // ---- 2. scaled, optionally sign-pivoted Cholesky in FP32 -----------------------------------
  if (tid < k) {
    const float d = sqrtf((float)Vs[tid * PV_LDV + tid]);
    sm.dd[tid] = d;
    sm.invd[tid] = 1.0 / (double)d;
    sm.perm[tid] = tid;
    sm.jphys[tid] = sm.jloc[tid];
  }
  for (int e = tid; e < PV_KM * PV_LDF; e += PV_THREADS) {
    sm.F[e] = 0.0f;
    sm.W[e] = 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += PV_THREADS) {
    const int i = e % k, j = e / k;
    double v = Vs[j * PV_LDV + i] * sm.invd[i] * sm.invd[j];
    if (i == j) v -= 1.0;
    sm.S[j * PV_LDS + i] = (float)v;
  }
  int npos = 0;
  for (int c = 0; c < k; ++c) npos += (sm.jloc[c] > 0) ? 1 : 0;  // J sorted: + block first
  __syncthreads();
  const bool signpiv = (pp.factor == 2);
  for (int i = 0; i < k; ++i) {
    if (signpiv) {
      if (warp == 0) {
        const int hi = (i < npos) ? npos : k;
        float best = -1.0f;
        int bj = i;
        for (int j = i + lane; j < hi; j += 32) {
          const float dj = sm.dd[j];
          const float v = dj * dj * (1.0f + sm.S[j * PV_LDS + j]);
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
      if (pv != i) {
        // symmetric swap of rows/columns i and pv of the trailing matrix, of the computed rows
        // of F (columns i and pv), and of the bookkeeping
        for (int tt = tid; tt < k; tt += PV_THREADS) {
          if (tt >= i && tt != i && tt != pv) {
            float x = sm.S[i * PV_LDS + tt];
            sm.S[i * PV_LDS + tt] = sm.S[pv * PV_LDS + tt];
            sm.S[pv * PV_LDS + tt] = x;
            x = sm.S[tt * PV_LDS + i];
            sm.S[tt * PV_LDS + i] = sm.S[tt * PV_LDS + pv];
            sm.S[tt * PV_LDS + pv] = x;
          }
          if (tt < i) {
            float x = sm.F[i * PV_LDF + tt];
            sm.F[i * PV_LDF + tt] = sm.F[pv * PV_LDF + tt];
            sm.F[pv * PV_LDF + tt] = x;
          }
        }
        if (tid == 0) {
          float x = sm.S[i * PV_LDS + i];
          sm.S[i * PV_LDS + i] = sm.S[pv * PV_LDS + pv];
          sm.S[pv * PV_LDS + pv] = x;
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
    const float sii = sm.S[i * PV_LDS + i];
    const float piv1 = 1.0f + sii;
    // The scaled Schur pivot is 1 / (A~^-1)_ii >= 1 / kappa(A~).  Below 64 eps_32 the column is
    // in the span of the previous ones at the precision of this factorization: the block (and
    // G) is treated as rank deficient.
    if (!(piv1 > 3.8146973e-6f)) {
      if (tid == 0) sm.bad = 1;
      break;               // uniform: every thread read the same sii
    }
    const float r = sqrtf(piv1);
    for (int j = i + 1 + tid; j < k; j += PV_THREADS) sm.F[j * PV_LDF + i] = sm.S[j * PV_LDS + i] / r;
    if (tid == 0) sm.F[i * PV_LDF + i] = sii / (1.0f + r);
    __syncthreads();
    const int nt = k - i - 1;
    for (int e = tid; e < nt * nt; e += PV_THREADS) {
      const int jj = i + 1 + e % nt, ll = i + 1 + e / nt;
      sm.S[ll * PV_LDS + jj] -= sm.F[jj * PV_LDF + i] * sm.F[ll * PV_LDF + i];
    }
    __syncthreads();
  }
  __syncthreads();
  if (sm.bad) {
    if (tid == 0) {
      atomicOr(err, JAC_DEVERR_NOTPD);
      skip[pair] = 1;
      stats[pair] = st;
    }
    return;
  }
  // R = Dp + F: scale the columns of F~ by dd; logical order of the inner sweep
  for (int e = tid; e < k * k; e += PV_THREADS) {
    const int r = e % k, c = e / k;
    if (r <= c) sm.F[c * PV_LDF + r] *= sm.dd[c];
  }
  if (tid < k) {
    int l = tid;
    sm.lpos[l] = (signpiv && l >= npos) ? (k - 1 - (l - npos)) : l;
  }
  __syncthreads();

  // ---- 3. inner one-sided Jacobi (FP32, shifted representation) -----------------------------
  // inner threshold: at most half the outer one (so that a pair flagged in FP64 is rotated in
  // FP32), at least the FP32 noise level of the shifted dot products
  const float tol_in = fmaxf(0.5f * (float)pp.tol, 64.0f * 5.9604645e-8f * (float)st.max_scaled);
  const int kk = k + (k & 1);
  int total_rot = 0, inner = 0;
  for (inner = 0; inner < JAC_INNER_MAX_SWEEPS; ++inner) {
    int my_rot = 0;
    for (int s = 0; s < kk - 1; ++s) {
      if (warp < kk / 2) {
        int li, lj;
        rr_inner_pair(kk, s, warp, li, lj);
        if (lj < k) {
          const int i = sm.lpos[li], j = sm.lpos[lj];
          float* Fi = sm.F + i * PV_LDF;
          float* Fj = sm.F + j * PV_LDF;
          const float fi0 = Fi[lane], fi1 = Fi[lane + 32], fj0 = Fj[lane], fj1 = Fj[lane + 32];
          float sii = fi0 * fi0 + fi1 * fi1;
          float sjj = fj0 * fj0 + fj1 * fj1;
          float sij = fi0 * fj0 + fi1 * fj1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sii += __shfl_xor_sync(0xffffffffu, sii, o);
            sjj += __shfl_xor_sync(0xffffffffu, sjj, o);
            sij += __shfl_xor_sync(0xffffffffu, sij, o);
          }
          const float si = sm.dd[i], sj = sm.dd[j];
          const float Fii = Fi[i], Fjj = Fj[j], Fji = Fi[j], Fij = Fj[i];
          const float ci = 2.0f * si * Fii + sii, cj = 2.0f * sj * Fjj + sjj;
          const float aij = si * Fij + sj * Fji + sij;
          const float aii = si * si + ci, ajj = sj * sj + cj;
          const float beta = fabsf(aij);
          if (beta > tol_in * sqrtf(aii) * sqrtf(ajj)) {
            ++my_rot;
            const float e = (aij < 0.0f) ? -1.0f : 1.0f;
            float q11, q12, q21, cm1;
            if (sm.jphys[i] == sm.jphys[j]) {
              // trigonometric, Eq. (2.1): cot(2 phi) = (a_jj - a_ii) / (2 |a_ij|)
              const float zeta = ((sj - si) * (sj + si) + (cj - ci)) / (2.0f * beta);
              const float az = fabsf(zeta);
              const float t = (az > 1.0e18f) ? 0.5f / zeta : copysignf(1.0f, zeta) / (az + sqrtf(1.0f + zeta * zeta));
              const float c = 1.0f / sqrtf(1.0f + t * t);
              const float s_ = t * c;
              cm1 = -(s_ * s_) / (1.0f + c);  // c - 1
              q11 = c;
              q12 = e * s_;
              q21 = -e * s_;
            } else {
              // hyperbolic: coth(2 phi) = -(a_ii + a_jj) / (2 |a_ij|); |tanh| < 1 guard (Sec. 3.2)
              const float zeta = -(aii + ajj) / (2.0f * beta);
              const float az = fabsf(zeta);
              float t;
              if (az > 1.0e18f) {
                t = 0.5f / zeta;
              } else {
                const float r2 = (az - 1.0f) * (az + 1.0f);
                t = (r2 > 0.0f) ? copysignf(1.0f, zeta) / (az + sqrtf(r2)) : copysignf(1.0f, zeta);
              }
              if (!(fabsf(t) < 1.0f) || !((1.0f - t) * (1.0f + t) > 0.0f)) t = copysignf(0.9f, t);
              const float ch = 1.0f / sqrtf((1.0f - t) * (1.0f + t));
              const float sh = t * ch;
              cm1 = (sh * sh) / (1.0f + ch);  // ch - 1
              q11 = ch;
              q12 = e * sh;
              q21 = e * sh;
            }
            const float q22 = q11;
            float nfi0 = q11 * fi0 + q21 * fj0, nfi1 = q11 * fi1 + q21 * fj1;
            float nfj0 = q12 * fi0 + q22 * fj0, nfj1 = q12 * fi1 + q22 * fj1;
            // + Dp (Q - I): column i gets si (q11-1) at row i and sj q21 at row j; column j
            // gets si q12 at row i and sj (q22-1) at row j
            if (lane == (i & 31)) {
              if (i < 32) { nfi0 += si * cm1; nfj0 += si * q12; } else { nfi1 += si * cm1; nfj1 += si * q12; }
            }
            if (lane == (j & 31)) {
              if (j < 32) { nfi0 += sj * q21; nfj0 += sj * cm1; } else { nfi1 += sj * q21; nfj1 += sj * cm1; }
            }
            Fi[lane] = nfi0;
            Fi[lane + 32] = nfi1;
            Fj[lane] = nfj0;
            Fj[lane + 32] = nfj1;
            float* Wi = sm.W + i * PV_LDF;
            float* Wj = sm.W + j * PV_LDF;
            const float wi0 = Wi[lane], wi1 = Wi[lane + 32], wj0 = Wj[lane], wj1 = Wj[lane + 32];
            float nwi0 = q11 * wi0 + q21 * wj0, nwi1 = q11 * wi1 + q21 * wj1;
            float nwj0 = q12 * wi0 + q22 * wj0, nwj1 = q12 * wi1 + q22 * wj1;
            if (lane == (i & 31)) {
              if (i < 32) { nwi0 += cm1; nwj0 += q12; } else { nwi1 += cm1; nwj1 += q12; }
            }
            if (lane == (j & 31)) {
              if (j < 32) { nwi0 += q21; nwj0 += cm1; } else { nwi1 += q21; nwj1 += cm1; }
            }
            Wi[lane] = nwi0;
            Wi[lane + 32] = nwi1;
            Wj[lane] = nwj0;
            Wj[lane + 32] = nwj1;
          }
        }
      }
      __syncthreads();
    }
    if (lane == 0) sm.red_i[warp] = my_rot;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < PV_WARPS; ++w) tot += sm.red_i[w];
    __syncthreads();
    total_rot += tot;
    if (tot == 0) break;
  }
  if (inner >= JAC_INNER_MAX_SWEEPS && tid == 0) atomicOr(err, JAC_DEVERR_INNER_LIMIT);

  // ---- 4. V_P = P (I + Wd) Pi in FP64, then J-orthogonalize ---------------------------------
  for (int e = tid; e < KP * KP; e += PV_THREADS) {
    const int r = e % KP, l = e / KP;
    double v = 0.0;
    int row = r;
    if (r < k && l < k) {
      const int c = sm.lpos[l];
      v = (double)sm.W[c * PV_LDF + r] + ((r == c) ? 1.0 : 0.0);
      row = sm.perm[r];
    }
    Vs[l * PV_LDV + row] = v;
  }
  __syncthreads();
  int ns = 0;
  const double ns_thresh = 8.881784197001252e-16;  // 2^-50
  for (int it = 0; it < 4; ++it) {
    // M = V^T J V - J   (J = J_P on rows and on columns: the permutations keep the signs)
    cta_dmma(
        KP, [&](int i, int r) { return Vs[i * PV_LDV + r]; },
        [&](int r, int j) { return (r < k && sm.jloc[r] < 0) ? -Vs[j * PV_LDV + r] : Vs[j * PV_LDV + r]; },
        [&](int i, int j, double v) {
          if (i == j && i < k) v -= (sm.jloc[i] < 0) ? -1.0 : 1.0;
          sm.M[j * PV_LDM + i] = v;
        });
    __syncthreads();
    double mloc = 0.0;
    for (int e = tid; e < KP * KP; e += PV_THREADS) mloc = fmax(mloc, fabs(sm.M[(e / KP) * PV_LDM + e % KP]));
    mloc = warp_max_d(mloc);
    if (lane == 0) sm.red_d[warp][0] = mloc;
    __syncthreads();
    double mm = 0.0;
    for (int w = 0; w < PV_WARPS; ++w) mm = fmax(mm, sm.red_d[w][0]);
    __syncthreads();
    if (mm < ns_thresh) break;
    // T = V (J M)
    cta_dmma(
        KP, [&](int r, int x) { return Vs[x * PV_LDV + r]; },
        [&](int x, int j) { return (x < k && sm.jloc[x] < 0) ? -sm.M[j * PV_LDM + x] : sm.M[j * PV_LDM + x]; },
        [&](int r, int j, double v) { sm.T[j * PV_LDM + r] = v; });
    __syncthreads();
    for (int e = tid; e < KP * KP; e += PV_THREADS) {
      const int r = e % KP, j = e / KP;
      Vs[j * PV_LDV + r] -= 0.5 * sm.T[j * PV_LDM + r];
    }
    __syncthreads();
    ++ns;
  }
  double* out = vp + (size_t)pair * JAC_KMAX * JAC_KMAX;
  for (int e = tid; e < KP * KP; e += PV_THREADS) {
    const int r = e % KP, j = e / KP;
    out[j * JAC_KMAX + r] = Vs[j * PV_LDV + r];
  }
  if (tid == 0) {
    skip[pair] = 0;
    st.rotations = total_rot;
    st.inner_sweeps = inner + 1;
    st.ns_steps = ns;
    stats[pair] = st;
  }
}

size_t pivot_smem_bytes() { return sizeof(PivotSmem); }

}  // namespace jac
