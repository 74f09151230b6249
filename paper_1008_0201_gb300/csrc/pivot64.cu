// pivot64.cu -- the pivot block in FP64 throughout, for the blocks the FP32 pivot kernel hands
// over (skip[pair] == 2): a Cholesky factor whose scaled Schur pivot falls below what FP32
// resolves (an ill-conditioned but full-rank block: kappa(A~) above ~2.6e5), or a transform
// whose J-unitarity Newton-Schulz does not restore to FP64 accuracy in its step budget.
//
// The computation is the one of Sec. 3.2 / Algorithm 3.4 for one block, as the paper runs it:
//  1. the scaled Gram A~ = D^-1 A_P D^-1 (D = diag(sqrt(a_ii))), factored P^T A~ P = R~^T R~ by
//     Cholesky, unpivoted (HF), diagonally pivoted (HFC) or J_P-sign-pivoted (Algorithm 3.3:
//     diagonal pivoting inside the J = +1 part, then inside the Schur complement of the J = -1
//     part), pivoting on the unscaled diagonal d_j^2 s_jj;
//  2. R = R~ D (so R^T R = P^T A_P P) and the pointwise one-sided Jacobi on its columns w.r.t.
//     J_P: trigonometric rotations (Eq. (2.1)) for equal signs, hyperbolic ones otherwise with
//     the |tanh| < 1 guard of Sec. 3.2; the columns of the J = -1 part are taken in reverse
//     order (the Pi of Algorithm 3.3); inner sweeps until none rotates;
//  3. V_P = P W Pi with W the accumulated rotations.
// A Schur pivot at or below 64 eps_64 means the block (so G) is rank deficient: NOTPD.
// One warp per column pair of an inner step; every lane computes its pair's rotation.
#include "jacobi_common.cuh"

namespace jac {

template <int KM>
struct Pivot64Smem {
  static constexpr int LD = KM + 1;
  static constexpr int NW = KM / 2;
  double A[KM * LD];  // scaled Gram, Schur complements in the upper triangle (A[col * LD + row])
  double R[KM * LD];  // R, column-major
  double W[KM * LD];  // accumulated rotations (physical columns)
  double dd[KM];
  int perm[KM];
  int jloc[KM];
  int jphys[KM];
  int lpos[KM];
  int red_i[NW];
  double red_d[NW];
  int piv;
  int bad;
};

template <int KM>
__global__ void __launch_bounds__(KM * 16, 1) k_pivot64(const JacProb* __restrict__ probs, int s, PivotParams pp) {
  constexpr int NT = KM * 16, NW = KM / 2;
  using SM = Pivot64Smem<KM>;
  constexpr int LD = SM::LD;
  extern __shared__ __align__(16) unsigned char p64_raw[];
  SM& sm = *reinterpret_cast<SM*>(p64_raw);
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || a.skip[pair] != 2) return;
  const long long t_start = clock64();
  PairStat* stats = a.stats + (size_t)s * a.half;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq;  // <= KM: the FP32 kernel handed the block over only in that case

  // ---- 1. scaled Gram and its Cholesky factor ------------------------------------------------
  const double* Ag = a.Ap + (size_t)pair * a.apld * a.apld;
  if (tid < k) {
    const int col = tid < wp ? op + tid : oq + (tid - wp);
    sm.jloc[tid] = a.Js[col];
    sm.dd[tid] = sqrt(Ag[tid * a.apld + tid]);  // > 0: checked by the FP32 kernel
    sm.perm[tid] = tid;
  }
  if (tid == 0) sm.bad = 0;
  for (int e = tid; e < KM * LD; e += NT) {
    sm.R[e] = 0.0;
    sm.W[e] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += NT) {
    const int i = e % k, j = e / k;
    if (i <= j) sm.A[j * LD + i] = (i == j) ? 1.0 : Ag[j * a.apld + i] / (sm.dd[i] * sm.dd[j]);
    if (i == j) sm.W[j * LD + i] = 1.0;
  }
  int npos = 0;
  for (int c = 0; c < k; ++c) npos += (sm.jloc[c] > 0) ? 1 : 0;  // J sorted: + part first
  if (tid < k) sm.jphys[tid] = sm.jloc[tid];
  __syncthreads();
  const bool signpiv = (pp.factor == 2), diagpiv = (pp.factor == 1);
  const int cx = tid % KM, cy = tid / KM;
  for (int i = 0; i < k; ++i) {
    if (signpiv || diagpiv) {
      if (warp == 0) {
        const int hi = (signpiv && i < npos) ? npos : k;
        double best = -1.0;
        int bj = i;
        for (int j = i + lane; j < hi; j += 32) {
          const double v = sm.dd[j] * sm.dd[j] * sm.A[j * LD + j];
          if (v > best) {
            best = v;
            bj = j;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
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
      if (pv != i) {  // uniform: symmetric swap of i and pv in the trailing matrix and in R
        for (int tt = tid; tt < k; tt += NT) {
          if (tt > i && tt != pv) {
            const int a1 = tt * LD + i;
            const int a2 = (tt > pv) ? tt * LD + pv : pv * LD + tt;
            const double x = sm.A[a1];
            sm.A[a1] = sm.A[a2];
            sm.A[a2] = x;
          }
          if (tt < i) {
            const double x = sm.R[i * LD + tt];
            sm.R[i * LD + tt] = sm.R[pv * LD + tt];
            sm.R[pv * LD + tt] = x;
          }
        }
        if (tid == 0) {
          double x = sm.A[i * LD + i];
          sm.A[i * LD + i] = sm.A[pv * LD + pv];
          sm.A[pv * LD + pv] = x;
          int y = sm.perm[i];
          sm.perm[i] = sm.perm[pv];
          sm.perm[pv] = y;
          x = sm.dd[i];
          sm.dd[i] = sm.dd[pv];
          sm.dd[pv] = x;
          y = sm.jphys[i];
          sm.jphys[i] = sm.jphys[pv];
          sm.jphys[pv] = y;
        }
        __syncthreads();
      }
    }
    const double piv = sm.A[i * LD + i];
    if (!(piv > 7.105427357601002e-15)) {  // 64 eps_64
      if (tid == 0) sm.bad = 1;
      break;  // uniform
    }
    const double r = sqrt(piv), ipiv = 1.0 / piv;
    if (cy == 0 && cx > i && cx < k) sm.R[cx * LD + i] = sm.A[cx * LD + i] / r;
    if (tid == 0) sm.R[i * LD + i] = r;
    if (cx > i && cx < k) {
      const double sil = sm.A[cx * LD + i] * ipiv;
      for (int jj = i + 1 + cy; jj <= cx; jj += NT / KM) sm.A[cx * LD + jj] -= sil * sm.A[jj * LD + i];
    }
    __syncthreads();
  }
  __syncthreads();
  PairStat st = stats[pair];  // statistics of this block, written by the FP32 kernel
  if (sm.bad) {
    if (tid == 0) {
      atomicOr(a.pflags, JAC_DEVERR_NOTPD);
      a.skip[pair] = 1;
    }
    return;
  }
  // R = R~ D (column c scaled by d_c); logical order of the inner sweep
  for (int e = tid; e < k * k; e += NT) {
    const int rr = e % k, c = e / k;
    if (rr <= c) sm.R[c * LD + rr] *= sm.dd[c];
  }
  if (tid < k) {
    if (diagpiv) {  // positions of the own sign, as in the FP32 kernel (HFC reordering)
      const bool pos = sm.jphys[tid] > 0;
      int rank = 0;
      for (int c = 0; c < tid; ++c) rank += ((sm.jphys[c] > 0) == pos) ? 1 : 0;
      sm.lpos[pos ? rank : npos + rank] = tid;
    } else {
      sm.lpos[tid] = (signpiv && tid >= npos) ? (k - 1 - (tid - npos)) : tid;
    }
  }
  __syncthreads();
  const long long t_chol = clock64();

  // ---- 2. inner one-sided Jacobi in FP64 -----------------------------------------------------
  const double tol = pp.tol > 0.0 ? pp.tol : fmax((double)a.n, pp.tol_m * sqrt((double)a.mp)) * pp.tol_eps;
  // at most half the outer threshold, at least the rounding level of a k-term FP64 dot product;
  // what is left is finished by the FP32 kernel in a later sweep
  const double tol_in = fmax(0.5 * tol, 16.0 * k * 1.1102230246251565e-16);
  const int kk = k + (k & 1);
  const int P = kk / 2;
  int total_rot = 0, inner = 0;
  for (inner = 0; inner < JAC_INNER_MAX_SWEEPS; ++inner) {
    int my_rot = 0;
    double my_max = 0.0;
    for (int st_ = 0; st_ < kk - 1; ++st_) {
      if (warp < P) {
        int li, lj;
        rr_inner_pair(kk, st_, warp, li, lj);
        if (lj < k) {
          const int i = sm.lpos[li], j = sm.lpos[lj];
          double ri[2], rj[2];
          double sii = 0.0, sjj = 0.0, sij = 0.0;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int row = lane + 32 * u;
            ri[u] = (row < k) ? sm.R[i * LD + row] : 0.0;
            rj[u] = (row < k) ? sm.R[j * LD + row] : 0.0;
            sii = fma(ri[u], ri[u], sii);
            sjj = fma(rj[u], rj[u], sjj);
            sij = fma(ri[u], rj[u], sij);
          }
          sii = warp_sum_d(sii);
          sjj = warp_sum_d(sjj);
          sij = warp_sum_d(sij);
          const double beta = fabs(sij);
          const double scaled = beta / sqrt(sii * sjj);
          if (scaled > tol_in) {  // uniform over the warp (same reduced values)
            ++my_rot;
            my_max = fmax(my_max, scaled);
            const double e = (sij < 0.0) ? -1.0 : 1.0;
            double q11, q12, q21;
            if (sm.jphys[i] == sm.jphys[j]) {
              // trigonometric, Eq. (2.1): t = sign(a_jj - a_ii) 2|a_ij| /
              // (|a_jj - a_ii| + sqrt((a_jj - a_ii)^2 + 4|a_ij|^2))
              const double num = sjj - sii;
              const double mxv = fmax(fabs(num), 2.0 * beta);
              const double nu = num / mxv, b2 = 2.0 * beta / mxv;
              const double t = copysign(b2 / (fabs(nu) + sqrt(nu * nu + b2 * b2)), num);
              const double c = 1.0 / sqrt(1.0 + t * t);
              const double sn = t * c;
              q11 = c;
              q12 = e * sn;
              q21 = -e * sn;
            } else {
              // hyperbolic: t = -2|a_ij| / (a_ii + a_jj + sqrt((a_ii + a_jj)^2 - 4|a_ij|^2)),
              // |t| < 1 guarded as in Sec. 3.2
              const double apd = sii + sjj;
              const double ap = 1.0, b2 = 2.0 * beta / apd;
              const double r2 = (ap - b2) * (ap + b2);
              double t = (r2 > 0.0) ? -b2 / (ap + sqrt(r2)) : -1.0;
              if (!(fabs(t) < 1.0) || !((1.0 - t) * (1.0 + t) > 0.0)) t = copysign(0.9, t);
              const double ch = 1.0 / sqrt((1.0 - t) * (1.0 + t));
              const double sh = t * ch;
              q11 = ch;
              q12 = e * sh;
              q21 = e * sh;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int row = lane + 32 * u;
              if (row < k) {
                sm.R[i * LD + row] = fma(q11, ri[u], q21 * rj[u]);
                sm.R[j * LD + row] = fma(q11, rj[u], q12 * ri[u]);
                const double wi = sm.W[i * LD + row], wj = sm.W[j * LD + row];
                sm.W[i * LD + row] = fma(q11, wi, q21 * wj);
                sm.W[j * LD + row] = fma(q11, wj, q12 * wi);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if (lane == 0) {
      sm.red_i[warp] = my_rot;
      sm.red_d[warp] = my_max;
    }
    __syncthreads();
    int tot = 0;
    double dmax = 0.0;
    for (int w = 0; w < NW; ++w) {
      tot += sm.red_i[w];
      dmax = fmax(dmax, sm.red_d[w]);
    }
    __syncthreads();
    total_rot += tot;
    if (tot == 0 || (double)k * dmax * dmax <= tol_in) break;
  }
  if (inner >= JAC_INNER_MAX_SWEEPS && tid == 0) atomicOr(a.pflags, JAC_DEVERR_INNER_LIMIT);
  const long long t_inner = clock64();

  // ---- 3. V_P = P W Pi: V_P[perm[r]][l] = W[r][lpos[l]] ---------------------------------------
  double* out = a.vp + (size_t)pair * a.apld * a.apld;
  for (int e = tid; e < k * k; e += NT) {
    const int rr = e % k, l = e / k;
    out[l * a.apld + sm.perm[rr]] = sm.W[sm.lpos[l] * LD + rr];
  }
  if (tid == 0) {
    a.skip[pair] = 0;
    st.rotations += total_rot;
    st.inner_sweeps += inner + 1;
    st.cyc[1] += t_chol - t_start;
    st.cyc[2] += t_inner - t_chol;
    stats[pair] = st;
  }
}

int pivot64_set_attributes() {
  bool ok = cudaFuncSetAttribute(k_pivot64<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Pivot64Smem<32>)) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_pivot64<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Pivot64Smem<64>)) == cudaSuccess;
  return ok ? 0 : 1;
}

// Same grid as the FP32 pivot kernel; CTAs of blocks not handed over return at once.
void pivot64_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                    const PivotParams& pp) {
  if (km == 32)
    k_pivot64<32><<<dim3(max_half, nprob), 32 * 16, sizeof(Pivot64Smem<32>), st>>>(probs, s, pp);
  else
    k_pivot64<64><<<dim3(max_half, nprob), 64 * 16, sizeof(Pivot64Smem<64>), st>>>(probs, s, pp);
}

}  // namespace jac
