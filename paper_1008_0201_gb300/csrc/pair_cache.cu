// pair_cache.cu -- skipping pairs whose outcome is already known, exactly.
//
// The Gram block A_P of a pair (Eq. (3.4)) depends only on the columns of its two blocks, and every
// step kernel is deterministic.  So when neither block has changed since the pair was last
// evaluated in the same slot of the same step, and it did not rotate then, its Gram block, the
// pivot's decision (no rotation) and its statistics would come out bitwise as before: the step
// kernels return at once for it, and the sweep reduction reads the statistics it left.  Late
// sweeps, where few pairs still rotate, then cost little more than the pairs that do.  Versions
// count the rotations that touched each block; a pair's record holds the versions it saw.
// Off for the per-cycle weight ordering (its slots change from sweep to sweep).
#include "jacobi_common.cuh"

namespace jac {

// Grid (nprob), 256 threads: no pair cached, no record valid, versions 0.
__global__ void k_cache_init(const JacProb* __restrict__ probs) {
  const JacProb& a = probs[blockIdx.x];
  if (!a.cached) return;
  for (int i = threadIdx.x; i < a.half; i += blockDim.x) a.cached[i] = 1;
  for (int i = threadIdx.x; i < a.nsteps * a.half; i += blockDim.x) a.pver[i] = make_int4(-1, -1, -1, -1);
  for (int i = threadIdx.x; i < a.nb; i += blockDim.x) a.bver[i] = 0;
}

// Grid (nprob), 256 threads (one CTA per problem: the record must be complete before the check).
// rec >= 0: record the outcome of step rec (-2: the problem's last step) for the pairs evaluated
// there; chk >= 0: mark the cached pairs of step chk and set their skip flags.
__global__ void k_cache_step(const JacProb* __restrict__ probs, int rec, int chk) {
  const JacProb& a = probs[blockIdx.x];
  if (!a.active || !a.cached) return;
  if (rec == -2) rec = a.nsteps - 1;
  if (rec >= 0 && rec < a.nsteps) {
    const int* sp = a.pairs + (size_t)rec * a.half * 2;
    for (int i = threadIdx.x; i < a.counts[rec]; i += blockDim.x) {
      if (a.cached[i]) continue;  // not evaluated in that step
      const int p = sp[2 * i], q = sp[2 * i + 1];
      const bool rot = a.skip[i] != 1;  // rotated, or handed over without a rotation
      if (rot) {  // the pairs of a step are disjoint: no other thread touches these blocks
        ++a.bver[p];
        ++a.bver[q];
      }
      a.pver[(size_t)rec * a.half + i] = make_int4(p, q, rot ? -1 : a.bver[p], a.bver[q]);
    }
  }
  __syncthreads();
  if (chk < 0) return;
  if (chk >= a.nsteps) {
    for (int i = threadIdx.x; i < a.half; i += blockDim.x) a.cached[i] = 1;
    return;
  }
  const int* sp = a.pairs + (size_t)chk * a.half * 2;
  for (int i = threadIdx.x; i < a.counts[chk]; i += blockDim.x) {
    const int p = sp[2 * i], q = sp[2 * i + 1];
    const int4 e = a.pver[(size_t)chk * a.half + i];
    const int hit = (e.x == p && e.y == q && e.z == a.bver[p] && e.w == a.bver[q]) ? 1 : 0;
    a.cached[i] = hit;
    if (hit) {
      a.skip[i] = 1;
      PairStat& st = a.stats[(size_t)chk * a.half + i];  // the decision stays; the work is not redone
      st.inner_sweeps = 0;
      st.ns_steps = 0;
      st.evaluated = 0;
      for (int u = 0; u < 4; ++u) st.cyc[u] = 0;
    }
  }
}

}  // namespace jac
