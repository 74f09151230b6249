// sched.cu -- device-side parallel block ordering (Sec. 2.4 of the paper).
//
// One "step" is a set of disjoint block pairs (p < q) that are transformed concurrently;
// disjointness is what makes them independent (Sec. 2.4).  A cycle (sweep) visits every
// pair of the nb blocks.  Tables are written as pairs[(s*half + slot)*2 + {0,1}] with the
// pairs of a step sorted by p, and counts[s].
#include "jacobi_common.cuh"

namespace jac {

// Modulus strategy: step k pairs the blocks on the k-th block antidiagonal taken modulo nb,
// {p < q : p + q = k (mod nb)} (Sec. 2.4, Fig. 2-3).  The modified modulus strategy also
// pairs the two blocks left over on even steps.  Round-robin is the circle method (block
// nb-1 fixed): one perfect matching per step, nb-1 steps.
__global__ void k_sched_static(int nb, int ordering, int nsteps, int* pairs, int* counts) {
  const int half = nb / 2;
  const int s = blockIdx.x;
  if (s >= nsteps) return;
  for (int slot = threadIdx.x; slot < half; slot += blockDim.x) {
    pairs[(s * half + slot) * 2] = -1;
    pairs[(s * half + slot) * 2 + 1] = -1;
  }
  __syncthreads();
  if (ordering == 0 || ordering == 1) {
    const int k = s;
    // thread per candidate first index p; its slot is the number of valid p' < p
    for (int p = threadIdx.x; p < nb; p += blockDim.x) {
      int q = ((k - p) % nb + nb) % nb;
      bool valid = p < q;
      bool fixed_pair = false;
      int fq = -1;
      if (!valid && ordering == 1 && ((2 * p - k) % nb + nb) % nb == 0 && (nb % 2 == 0)) {
        // p is a fixed point (2p = k mod nb); the smaller one is paired with the larger
        int p2 = p + nb / 2;
        if (p2 < nb && ((2 * p2 - k) % nb + nb) % nb == 0) {
          fixed_pair = true;
          fq = p2;
        }
      }
      if (!valid && !fixed_pair) continue;
      int slot = 0;
      for (int pp = 0; pp < p; ++pp) {
        int qq = ((k - pp) % nb + nb) % nb;
        bool v = pp < qq;
        if (!v && ordering == 1 && ((2 * pp - k) % nb + nb) % nb == 0) {
          int p2 = pp + nb / 2;
          if (p2 < nb && ((2 * p2 - k) % nb + nb) % nb == 0) v = true;
        }
        slot += v ? 1 : 0;
      }
      pairs[(s * half + slot) * 2] = p;
      pairs[(s * half + slot) * 2 + 1] = valid ? q : fq;
    }
    if (threadIdx.x == 0) {
      int c = 0;
      for (int p = 0; p < nb; ++p) {
        int q = ((k - p) % nb + nb) % nb;
        if (p < q) ++c;
      }
      if (ordering == 1 && (k % 2 == 0) && (nb % 2 == 0)) ++c;
      counts[s] = c;
    }
  } else {
    // round-robin: pair r = 0 is (s, nb-1); r >= 1 is ((s+r) mod L, (s-r) mod L), L = nb-1
    const int L = nb - 1;
    for (int r = threadIdx.x; r < half; r += blockDim.x) {
      int a, b;
      if (r == 0) {
        a = s;
        b = nb - 1;
      } else {
        int x = ((s + r) % L + L) % L, y = ((s - r) % L + L) % L;
        a = min(x, y);
        b = max(x, y);
      }
      int slot = 0;
      for (int rr = 0; rr < half; ++rr) {
        int aa;
        if (rr == 0) {
          aa = s;
        } else {
          int x = ((s + rr) % L + L) % L, y = ((s - rr) % L + L) % L;
          aa = min(x, y);
        }
        slot += (aa < a) ? 1 : 0;
      }
      pairs[(s * half + slot) * 2] = a;
      pairs[(s * half + slot) * 2 + 1] = b;
    }
    if (threadIdx.x == 0) counts[s] = half;
  }
}

// Per-cycle largest-weight ordering: sort all pairs p < q by descending weight w[p*nb+q]
// (ties: enumeration order p, then q), then fill steps greedily in that order with pairs
// disjoint from those already in the step, until every pair is scheduled once.
//
// Ranking: k_sched_rank gives pair x the number of pairs y that precede it, y before x iff
// key(w_y) > key(w_x) or (key(w_y) == key(w_x) and y < x), with key(v) = v except that a NaN
// ranks last (key -inf).  This is a total order on (key, id), so the ranks are a permutation
// of 0..npairs-1 whatever the weights hold.  Grid ceil(npairs / 256) x 256 threads, one pair
// per thread; the weight matrix is staged row by row in shared memory (nb doubles).
__device__ __forceinline__ double rank_key(double v) {
  return (v == v) ? v : -__longlong_as_double(0x7ff0000000000000ll);
}

__global__ void __launch_bounds__(256) k_sched_rank(int nb, const double* __restrict__ w, int* __restrict__ order) {
  extern __shared__ double sh_row[];  // [nb]
  const int npairs = nb * (nb - 1) / 2;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  double kx = 0.0;
  if (x < npairs) {
    int p = 0, rem = x;
    while (rem >= nb - 1 - p) {
      rem -= nb - 1 - p;
      ++p;
    }
    kx = rank_key(w[(size_t)p * nb + p + 1 + rem]);
  }
  int rank = 0, y = 0;
  for (int pp = 0; pp + 1 < nb; ++pp) {
    __syncthreads();
    for (int qq = pp + 1 + threadIdx.x; qq < nb; qq += blockDim.x) sh_row[qq] = rank_key(w[(size_t)pp * nb + qq]);
    __syncthreads();
    if (x < npairs)
      for (int qq = pp + 1; qq < nb; ++qq, ++y) {
        const double ky = sh_row[qq];
        rank += (ky > kx || (ky == kx && y < x)) ? 1 : 0;
      }
  }
  if (x < npairs) order[rank] = x;
}

// Greedy packing of the ranked pairs (one CTA; order[] from k_sched_rank).  order[] is
// caller-provided global scratch of npairs ints (rank -> pair id, entries marked done in
// place); only the busy mask (nb ints) is in dynamic shared memory.
__global__ void k_sched_cycle_weight(int nb, int* order, int* pairs, int* counts, int max_steps, int* nsteps_out) {
  extern __shared__ int sh_sched[];
  const int npairs = nb * (nb - 1) / 2;
  const int half = nb / 2;
  int* busy = sh_sched;  // [nb]
  for (int i = threadIdx.x; i < max_steps * half; i += blockDim.x) {
    pairs[i * 2] = -1;
    pairs[i * 2 + 1] = -1;
  }
  __syncthreads();
  // 2. greedy packing (warp 0); the scan is in rank order, so conflicts inside a chunk of 32
  //    candidates are resolved lane by lane in that order
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int left = npairs, step = 0;
    // done flags: reuse the sign bit of order[] entries
    while (left > 0 && step < max_steps) {
      for (int b = lane; b < nb; b += 32) busy[b] = 0;
      __syncwarp();
      int np = 0;
      for (int base = 0; base < npairs; base += 32) {
        int r = base + lane;
        int x = (r < npairs) ? order[r] : -1;
        bool cand = x >= 0;
        int p = 0, q = 0;
        if (cand) {
          int rem = x;
          while (rem >= nb - 1 - p) {
            rem -= nb - 1 - p;
            ++p;
          }
          q = p + 1 + rem;
          cand = !busy[p] && !busy[q];
        }
        unsigned m = __ballot_sync(0xffffffffu, cand);
        while (m) {
          int first = __ffs(m) - 1;
          int fp = __shfl_sync(0xffffffffu, p, first);
          int fq = __shfl_sync(0xffffffffu, q, first);
          if (lane == first) {
            busy[fp] = 1;
            busy[fq] = 1;
            order[r] = -1 - x;  // mark done
            pairs[(step * half + np) * 2] = fp;
            pairs[(step * half + np) * 2 + 1] = fq;
            cand = false;
          }
          __syncwarp();
          if (cand) cand = !busy[p] && !busy[q];
          ++np;
          m = __ballot_sync(0xffffffffu, cand);
        }
        __syncwarp();
      }
      // the pairs of a step are written in rank order; sort them by p for a canonical table
      if (lane == 0) {
        int* P = pairs + step * half * 2;
        for (int a = 1; a < np; ++a) {
          int ap = P[2 * a], aq = P[2 * a + 1], b = a - 1;
          while (b >= 0 && P[2 * b] > ap) {
            P[2 * (b + 1)] = P[2 * b];
            P[2 * (b + 1) + 1] = P[2 * b + 1];
            --b;
          }
          P[2 * (b + 1)] = ap;
          P[2 * (b + 1) + 1] = aq;
        }
        counts[step] = np;
      }
      left -= np;
      ++step;
      __syncwarp();
    }
    if (lane == 0) *nsteps_out = (left == 0) ? step : -1;
  }
}

// Block weights for the per-cycle ordering, w[p*nb+q] = ||G_p^* G_q||_F^2 / (||G_p||_F^2 ||G_q||_F^2),
// from an FP32 copy of G (the weights only rank the pairs).  One CTA (256 threads) per pair
// p < q; thread (ty = tid / 16, tx = tid % 16) owns a 2 x 2 block of the <= 32 x 32 product.
__global__ void k_block_weights32(const float* __restrict__ G32, int mp, int nb, const int* __restrict__ boff,
                                  double* __restrict__ w) {
  __shared__ float xp[32][33], xq[32][33];
  __shared__ float red[8][3];
  const int npairs = nb * (nb - 1) / 2;
  const int x = blockIdx.x;
  if (x >= npairs) return;
  int p = 0, rem = x;
  while (rem >= nb - 1 - p) {
    rem -= nb - 1 - p;
    ++p;
  }
  const int q = p + 1 + rem;
  const int op = boff[p], wp = boff[p + 1] - op, oq = boff[q], wq = boff[q + 1] - oq;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, np2 = 0.f, nq2 = 0.f;
  for (int r0 = 0; r0 < mp; r0 += 32) {
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += 256) {
      const int r = idx & 31, c = idx >> 5;
      xp[r][c] = (c < wp && r0 + r < mp) ? G32[(size_t)(op + c) * mp + r0 + r] : 0.f;
      xq[r][c] = (c < wq && r0 + r < mp) ? G32[(size_t)(oq + c) * mp + r0 + r] : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < 32; ++r) {
      const float a0 = xp[r][2 * ty], a1 = xp[r][2 * ty + 1], b0 = xq[r][2 * tx], b1 = xq[r][2 * tx + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    if (tid < 32) {
      for (int r = 0; r < 32; ++r) np2 = fmaf(xp[r][tid], xp[r][tid], np2);
    } else if (tid < 64) {
      for (int r = 0; r < 32; ++r) nq2 = fmaf(xq[r][tid - 32], xq[r][tid - 32], nq2);
    }
  }
  float f = acc[0][0] * acc[0][0] + acc[0][1] * acc[0][1] + acc[1][0] * acc[1][0] + acc[1][1] * acc[1][1];
  f = warp_sum(f);
  np2 = warp_sum(np2);
  nq2 = warp_sum(nq2);
  const int warp = tid >> 5, lane = tid & 31;
  if (lane == 0) {
    red[warp][0] = f;
    red[warp][1] = np2;
    red[warp][2] = nq2;
  }
  __syncthreads();
  if (tid == 0) {
    float ff = 0.f;
    for (int u = 0; u < 8; ++u) ff += red[u][0];
    const double den = (double)red[0][1] * (double)red[1][2];
    double wv = (den > 0.0) ? (double)ff / den : 0.0;
    // by Cauchy-Schwarz the weight lies in [0, 1]; FP32 norms that overflowed give inf / inf:
    // such a pair is ranked as the heaviest
    if (!(wv == wv)) wv = 1.0;
    w[p * nb + q] = wv;
  }
}

}  // namespace jac
