// reduce_finalize.cu -- convergence reduction per sweep, input/output layout kernels.
//
//   k_sweep_reduce: off-norm and rotation counts of a sweep (the convergence test of
//                   Algorithm 3.4, "until convergence"; Sec. 4 calls the criterion natural:
//                   a sweep without rotations ends the iteration).
//   k_colnorm / k_rank / k_scatter: eigenpairs from the converged factor, lambda_k =
//                   j_k ||g_k||^2 and u_k = g_k / ||g_k|| (Sec. 3.2), in ascending lambda.
//   k_gather_in / k_init_v / k_check_finite: internal layout (J sorted to diag(I, -I) as
//                   Algorithms 3.2 and 3.4 assume) and input validation.
// Every kernel takes the problem index from a grid dimension (a single solve is a batch of one).
#include "jacobi_common.cuh"

namespace jac {

// One CTA (256 threads) per problem.  Each cross-block pair is seen once per sweep; each
// within-block pair and each diagonal entry nb-1 times, hence the weights.  With deactivate = 1
// a problem whose sweep rotated no pivot block is marked converged (active = 0); *remaining
// counts the problems still active.
__global__ void k_sweep_reduce(JacProb* __restrict__ probs, JacIO* __restrict__ io, SweepRecord* __restrict__ rec,
                               int deactivate, int* __restrict__ remaining) {
  __shared__ double sm_d[8][3];
  __shared__ long long sm_l[8][9];
  JacProb& a = probs[blockIdx.x];
  if (!a.active) {
    if (threadIdx.x == 0) {
      SweepRecord r = {};
      r.err = *a.pflags;
      rec[blockIdx.x] = r;
    }
    return;
  }
  double mx = 0.0, off2 = 0.0, tr = 0.0;
  long long rot = 0, piv = 0, cy[4] = {0, 0, 0, 0}, ns = 0, isw = 0, ev = 0;
  const double wdiag = 1.0 / (double)(a.nb > 1 ? a.nb - 1 : 1);
  for (int e = threadIdx.x; e < a.nsteps * a.half; e += blockDim.x) {
    const int s = e / a.half, slot = e % a.half;
    if (slot >= a.counts[s]) continue;
    const PairStat st = a.stats[e];
    mx = fmax(mx, st.max_scaled);
    off2 += 2.0 * st.off2_cross + 2.0 * wdiag * st.off2_diag;
    tr += wdiag * st.trace;
    rot += st.rotations;
    piv += st.active;
    ns += st.ns_steps;
    isw += st.inner_sweeps;
    ev += st.evaluated;
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
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
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
    sm_l[warp][8] = ev;
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
      r.evaluated += sm_l[w][8];
      for (int u = 0; u < 4; ++u) r.cyc[u] += sm_l[w][3 + u];
    }
    r.err = *a.pflags;
    rec[blockIdx.x] = r;
    io[blockIdx.x].sweeps += 1;
    io[blockIdx.x].rotations += r.rotations;
    if (r.err & JAC_DEVERR_NOTPD) a.active = 0;
    // converged: nothing rotated, or (from the second sweep on) the sweep's largest scaled
    // off-diagonal delta satisfies delta^2 <= 1e-6 tol (quadratic convergence: the next sweep
    // would rotate nothing)
    if (deactivate && (r.pivots_rotated == 0 ||
                       (io[blockIdx.x].sweeps >= 2 && r.max_scaled * r.max_scaled <= 1e-6 * a.tol)))
      a.active = 0;
    if (remaining && a.active) atomicAdd(remaining, 1);
  }
}

// Internal column order (Algorithms 3.2 / 3.4 take J = diag(I, -I)): perm_in lists the
// columns with j = +1, then those with j = -1, each in input order; Js are the sorted signs.
// An entry other than +-1 sets io.flags bit 1.  One warp per problem (grid nprob, 32 threads).
__global__ void k_sort_signs(const JacProb* __restrict__ probs, JacIO* __restrict__ io, int8_t* __restrict__ Js_all,
                             const long long* __restrict__ js_off) {
  const JacProb& a = probs[blockIdx.x];
  JacIO& o = io[blockIdx.x];
  int8_t* Js = Js_all + js_off[blockIdx.x];
  const int lane = threadIdx.x;
  int npos = 0;
  bool bad = false;
  // positives: prefix counts over 32-wide chunks
  for (int c0 = 0; c0 < a.n; c0 += 32) {
    const int c = c0 + lane;
    int v = 1;
    if (c < a.n && o.J) {
      v = o.J[c];
      bad |= (v != 1 && v != -1);
    }
    const unsigned pos = __ballot_sync(0xffffffffu, c < a.n && v > 0);
    if (c < a.n && v > 0) {
      const int dst = npos + __popc(pos & ((1u << lane) - 1u));
      o.perm_in[dst] = c;
      Js[dst] = 1;
    }
    npos += __popc(pos);
  }
  int nneg = 0;
  for (int c0 = 0; c0 < a.n; c0 += 32) {
    const int c = c0 + lane;
    const int v = (c < a.n && o.J) ? o.J[c] : 1;
    const unsigned neg = __ballot_sync(0xffffffffu, c < a.n && v <= 0);
    if (c < a.n && v <= 0) {
      const int dst = npos + nneg + __popc(neg & ((1u << lane) - 1u));
      o.perm_in[dst] = c;
      Js[dst] = -1;
    }
    nneg += __popc(neg);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) o.flags |= 2;
}

// Problems that failed validation (io.flags) or have a single column take no sweep.  One thread
// per problem.
__global__ void k_apply_flags(JacProb* __restrict__ probs, const JacIO* __restrict__ io, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  if ((io[i].flags & 3) || probs[i].n <= 1) probs[i].active = 0;
}

// The eigenpairs are extracted only from a factor that passed validation and every pivot.
__device__ __forceinline__ bool finalize_skip(const JacProb& a, const JacIO& o) {
  return (o.flags & 3) != 0 || (*a.pflags & (JAC_DEVERR_NOTPD | JAC_DEVERR_NONFINITE)) != 0;
}

// Gw[r, c] = G[r, perm_in[c]] for r < m, zero rows m..mp-1.  Grid (ceil(mp/256), n, nprob).
__global__ void k_gather_in(const JacProb* __restrict__ probs, const JacIO* __restrict__ io) {
  const JacProb& a = probs[blockIdx.z];
  const JacIO& o = io[blockIdx.z];
  const int c = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n || r >= a.mp) return;
  const int src = o.perm_in[c];
  a.Gw[(size_t)c * a.mp + r] = (r < o.m) ? o.G[(size_t)src * o.ldg + r] : 0.0;
}

// Vw = Pi (the internal column order): Vw[perm_in[c], c] = 1; or, with a starting transform,
// Vw = Vinit Pi.  Grid (ceil(np/256), n, nprob).
__global__ void k_init_v(const JacProb* __restrict__ probs, const JacIO* __restrict__ io) {
  const JacProb& a = probs[blockIdx.z];
  const JacIO& o = io[blockIdx.z];
  const int c = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (!a.Vw || c >= a.n || r >= a.np) return;
  double v;
  if (o.Vinit) v = (r < a.n) ? o.Vinit[(size_t)o.perm_in[c] * o.ldvi + r] : 0.0;
  else v = (r < a.n && r == o.perm_in[c]) ? 1.0 : 0.0;
  a.Vw[(size_t)c * a.np + r] = v;
}

// Sets JAC_DEVERR_NONFINITE (and, per problem, io.flags bit 0) if an entry of G has an all-ones
// exponent (NaN / Inf).  Integer test, no FP64 instruction.  Grid (blocks, nprob).
__global__ void k_check_finite(const JacProb* __restrict__ probs, JacIO* __restrict__ io) {
  const JacProb& a = probs[blockIdx.y];
  JacIO& o = io[blockIdx.y];
  const size_t total = (size_t)o.m * a.n;
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t c = e / o.m, r = e % o.m;
    const unsigned long long bits = __double_as_longlong(o.G[c * o.ldg + r]);
    bad |= ((bits >> 52) & 0x7ffull) == 0x7ffull;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
    atomicOr(a.pflags, JAC_DEVERR_NONFINITE);
    atomicOr(&o.flags, 1);
  }
}

// nrm2[c] = ||Gw[:, c]||^2 (FP64), lam[c] = j_c nrm2[c].  One warp per column.
// Grid (ceil(n*32/256), nprob).
__global__ void k_colnorm(const JacProb* __restrict__ probs, const JacIO* __restrict__ io) {
  const JacProb& a = probs[blockIdx.y];
  const JacIO& o = io[blockIdx.y];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= a.n || finalize_skip(a, o)) return;
  const double* g = a.Gw + (size_t)warp * a.mp;
  double s = 0.0;
  for (int r = lane; r < a.mp; r += 32) s += g[r] * g[r];
  s = warp_sum_d(s);
  if (lane == 0) {
    o.nrm2[warp] = s;
    o.lam[warp] = (a.Js[warp] < 0) ? -s : s;
  }
}

// Keys are the order-preserving unsigned images of the doubles (flip all bits of negatives,
// the sign bit of the rest), so the n^2 comparisons are integer work.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// rank[c] = #{l : lam[l] < lam[c] or (lam[l] == lam[c] and l < c)}: ascending order, ties by
// internal index (the stable J sort keeps input order within a sign).
// Grid (ceil(n/256), nprob), dynamic shared memory n keys.
__global__ void k_rank(const JacProb* __restrict__ probs, const JacIO* __restrict__ io) {
  extern __shared__ unsigned long long keys[];
  const JacProb& a = probs[blockIdx.y];
  const JacIO& o = io[blockIdx.y];
  if (finalize_skip(a, o)) return;  // uniform over the CTA
  for (int l = threadIdx.x; l < a.n; l += blockDim.x) keys[l] = order_key(o.lam[l]);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n) return;
  const unsigned long long v = keys[c];
  int r = 0;
  for (int l = 0; l < a.n; ++l) {
    const unsigned long long u = keys[l];
    r += (u < v || (u == v && l < c)) ? 1 : 0;
  }
  o.rank[c] = r;
}

// Output in ascending order: lambda[rank c] = lam[c]; G[:, rank c] = Gw[:, c];
// U[:, rank c] = Gw[:, c] / ||Gw[:, c]||; V[:, rank c] = Vw[:, c].  Grid (n, nprob), 128 threads.
__global__ void k_scatter(const JacProb* __restrict__ probs, const JacIO* __restrict__ io) {
  const JacProb& a = probs[blockIdx.y];
  const JacIO& o = io[blockIdx.y];
  const int c = blockIdx.x;
  if (c >= a.n || finalize_skip(a, o)) return;
  const int d = o.rank[c];
  __shared__ double inv;
  if (threadIdx.x == 0) {
    o.lambda[d] = o.lam[c];
    const double nn = o.nrm2[c];
    inv = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
  }
  __syncthreads();
  const double* g = a.Gw + (size_t)c * a.mp;
  for (int r = threadIdx.x; r < o.m; r += blockDim.x) {
    const double v = g[r];
    o.G[(size_t)d * o.ldg + r] = v;
    if (o.U) o.U[(size_t)d * o.ldu + r] = v * inv;
  }
  if (o.V && a.Vw) {
    const double* vv = a.Vw + (size_t)c * a.np;
    for (int r = threadIdx.x; r < a.n; r += blockDim.x) o.V[(size_t)d * o.ldv + r] = vv[r];
  }
}

}  // namespace jac
