// reduce_finalize.cu -- convergence reduction per sweep, input/output layout kernels.
//
//   k_sweep_reduce: off-norm and rotation counts of a sweep (the convergence test of
//                   Algorithm 3.4, "until convergence"; Sec. 4 calls the criterion natural:
//                   a sweep without rotations ends the iteration).
//   k_colnorm / k_rank / k_scatter: eigenpairs from the converged factor, lambda_k =
//                   j_k ||g_k||^2 and u_k = g_k / ||g_k|| (Sec. 3.2), in ascending lambda.
//   k_gather_in / k_init_v / k_check_finite: internal layout (J sorted to diag(I, -I) as
//                   Algorithms 3.2 and 3.4 assume) and input validation.
#include "jacobi_common.cuh"

namespace jac {

// One CTA, 256 threads.  stats: [nsteps][half]; counts: [nsteps].  Rotated pivots are those
// with rotations > 0.  Each cross-block pair is seen once per sweep; each within-block pair
// and each diagonal entry nb-1 times, hence the weights.
__global__ void k_sweep_reduce(const PairStat* __restrict__ stats, const int* __restrict__ counts, int nsteps,
                               int half, int nb, const unsigned* __restrict__ err, SweepRecord* __restrict__ rec) {
  __shared__ double sm_d[8][3];
  __shared__ long long sm_l[8][8];
  double mx = 0.0, off2 = 0.0, tr = 0.0;
  long long rot = 0, piv = 0, cy[4] = {0, 0, 0, 0}, ns = 0, isw = 0;
  const double wdiag = 1.0 / (double)(nb > 1 ? nb - 1 : 1);
  for (int e = threadIdx.x; e < nsteps * half; e += blockDim.x) {
    const int s = e / half, slot = e % half;
    if (slot >= counts[s]) continue;
    const PairStat st = stats[e];
    mx = fmax(mx, st.max_scaled);
    off2 += 2.0 * st.off2_cross + 2.0 * wdiag * st.off2_diag;
    tr += wdiag * st.trace;
    rot += st.rotations;
    piv += st.active;
    ns += st.ns_steps;
    isw += st.inner_sweeps;
    for (int u = 0; u < 4; ++u) cy[u] += st.cyc[u];
  }
  mx = warp_max_d(mx);
  off2 = warp_sum_d(off2);
  tr = warp_sum_d(tr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rot += __shfl_xor_sync(0xffffffffu, rot, o);
    piv += __shfl_xor_sync(0xffffffffu, piv, o);
    ns += __shfl_xor_sync(0xffffffffu, ns, o);
    isw += __shfl_xor_sync(0xffffffffu, isw, o);
    for (int u = 0; u < 4; ++u) cy[u] += __shfl_xor_sync(0xffffffffu, cy[u], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sm_d[warp][0] = mx;
    sm_d[warp][1] = off2;
    sm_d[warp][2] = tr;
    sm_l[warp][0] = rot;
    sm_l[warp][1] = piv;
    sm_l[warp][2] = ns;
    sm_l[warp][7] = isw;
    for (int u = 0; u < 4; ++u) sm_l[warp][3 + u] = cy[u];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SweepRecord r = {};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      r.max_scaled = fmax(r.max_scaled, sm_d[w][0]);
      r.off2 += sm_d[w][1];
      r.trace += sm_d[w][2];
      r.rotations += sm_l[w][0];
      r.pivots_rotated += sm_l[w][1];
      r.ns_steps += sm_l[w][2];
      r.inner_sweeps += sm_l[w][7];
      for (int u = 0; u < 4; ++u) r.cyc[u] += sm_l[w][3 + u];
    }
    r.err = *err;
    *rec = r;
  }
}

// Gw[r, c] = G[r, perm_in[c]] for r < m, zero rows m..mp-1.  Grid (ceil(mp/256), n).
__global__ void k_gather_in(const double* __restrict__ G, int ldg, int m, int mp, const int* __restrict__ perm_in,
                            double* __restrict__ Gw) {
  const int c = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mp) return;
  const int src = perm_in[c];
  Gw[(size_t)c * mp + r] = (r < m) ? G[(size_t)src * ldg + r] : 0.0;
}

// Vw = Pi (the internal column order): Vw[perm_in[c], c] = 1.  Grid (ceil(np/256), n).
__global__ void k_init_v(int n, int np, const int* __restrict__ perm_in, double* __restrict__ Vw) {
  const int c = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= np) return;
  Vw[(size_t)c * np + r] = (r < n && r == perm_in[c]) ? 1.0 : 0.0;
}

// Sets JAC_DEVERR_NONFINITE if any G entry has an all-ones exponent (NaN / Inf).  Integer test,
// no FP64 instruction.  Grid-stride over the m x n entries.
__global__ void k_check_finite(const double* __restrict__ G, int ldg, int m, int n, unsigned* __restrict__ err) {
  const size_t total = (size_t)m * n;
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t c = e / m, r = e % m;
    const unsigned long long bits = __double_as_longlong(G[c * ldg + r]);
    bad |= ((bits >> 52) & 0x7ffull) == 0x7ffull;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, JAC_DEVERR_NONFINITE);
}

// nrm2[c] = ||Gw[:, c]||^2 (FP64), lam[c] = j_c nrm2[c].  One warp per column.
__global__ void k_colnorm(const double* __restrict__ Gw, int mp, int n, const int8_t* __restrict__ Js,
                          double* __restrict__ nrm2, double* __restrict__ lam) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* g = Gw + (size_t)warp * mp;
  double s = 0.0;
  for (int r = lane; r < mp; r += 32) s += g[r] * g[r];
  s = warp_sum_d(s);
  if (lane == 0) {
    nrm2[warp] = s;
    lam[warp] = (Js[warp] < 0) ? -s : s;
  }
}

// rank[c] = #{l : lam[l] < lam[c] or (lam[l] == lam[c] and l < c)}: ascending order, ties by
// internal index (the stable J sort keeps input order within a sign).
// Keys are the order-preserving unsigned images of the doubles (flip all bits of negatives,
// the sign bit of the rest), so the n^2 comparisons are integer work.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__global__ void k_rank(const double* __restrict__ lam, int n, int* __restrict__ rank) {
  extern __shared__ unsigned long long keys[];
  for (int l = threadIdx.x; l < n; l += blockDim.x) keys[l] = order_key(lam[l]);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const unsigned long long v = keys[c];
  int r = 0;
  for (int l = 0; l < n; ++l) {
    const unsigned long long u = keys[l];
    r += (u < v || (u == v && l < c)) ? 1 : 0;
  }
  rank[c] = r;
}

// Output in ascending order: lambda[rank c] = lam[c]; G[:, rank c] = Gw[:, c];
// U[:, rank c] = Gw[:, c] / ||Gw[:, c]||; V[:, rank c] = Vw[:, c].  Grid n, 128 threads.
__global__ void k_scatter(const double* __restrict__ Gw, int mp, int m, const double* __restrict__ Vw, int np,
                          int n, const double* __restrict__ nrm2, const double* __restrict__ lam,
                          const int* __restrict__ rank, double* __restrict__ lambda, double* __restrict__ G,
                          int ldg, double* __restrict__ U, int ldu, double* __restrict__ V, int ldv) {
  const int c = blockIdx.x;
  const int d = rank[c];
  __shared__ double inv;
  if (threadIdx.x == 0) {
    lambda[d] = lam[c];
    const double nn = nrm2[c];
    inv = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
  }
  __syncthreads();
  const double* g = Gw + (size_t)c * mp;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const double v = g[r];
    G[(size_t)d * ldg + r] = v;
    if (U) U[(size_t)d * ldu + r] = v * inv;
  }
  if (V && Vw) {
    const double* vv = Vw + (size_t)c * np;
    for (int r = threadIdx.x; r < n; r += blockDim.x) V[(size_t)d * ldv + r] = vv[r];
  }
}

}  // namespace jac
