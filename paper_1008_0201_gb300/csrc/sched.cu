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
// One CTA.  order[] (npairs ints) and the busy mask live in dynamic shared memory, so
// nb*(nb-1)/2 + nb ints must fit (nb <= 128 here; larger nb use the global scratch variant).
__global__ void k_sched_cycle_weight(int nb, const double* __restrict__ w, int* order_g, int* pairs,
                                     int* counts, int max_steps, int* nsteps_out) {
  extern __shared__ int sh_sched[];
  const int npairs = nb * (nb - 1) / 2;
  const int half = nb / 2;
  int* order = order_g;  // global scratch [npairs]: rank -> pair id
  int* busy = sh_sched;  // [nb]
  __shared__ int s_done_count;
  // pair id x <-> (p, q) in enumeration order
  // 1. rank each pair: number of pairs that come before it in the sorted order
  for (int x = threadIdx.x; x < npairs; x += blockDim.x) {
    // decode x -> (p, q)
    int p = 0, rem = x;
    while (rem >= nb - 1 - p) {
      rem -= nb - 1 - p;
      ++p;
    }
    int q = p + 1 + rem;
    double wx = w[p * nb + q];
    int rank = 0;
    int y = 0;
    for (int pp = 0; pp < nb; ++pp)
      for (int qq = pp + 1; qq < nb; ++qq, ++y) {
        double wy = w[pp * nb + qq];
        rank += (wy > wx || (wy == wx && y < x)) ? 1 : 0;
      }
    order[rank] = x;
  }
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
    if (lane == 0) {
      s_done_count = left;
      *nsteps_out = (left == 0) ? step : -1;
    }
  }
  __syncthreads();
  // restore order[] (not needed by callers, keeps the scratch reusable)
  (void)s_done_count;
}

// Block weights for the per-cycle ordering: w[p*nb+q] = ||G_p^* G_q||_F^2 / (||G_p||_F^2 ||G_q||_F^2)
// One CTA (4 warps) per pair p < q (grid = npairs); FP64 mma over all rows.  Block widths <= 32.
__global__ void k_block_weights(const double* __restrict__ Gw, int mp, int nb, const int* __restrict__ boff,
                                double* __restrict__ w) {
  __shared__ double sX[2][16][33];  // [block][row][col] chunk of 16 rows
  __shared__ double red[4][3];
  const int npairs = nb * (nb - 1) / 2;
  int x = blockIdx.x;
  if (x >= npairs) return;
  int p = 0, rem = x;
  while (rem >= nb - 1 - p) {
    rem -= nb - 1 - p;
    ++p;
  }
  int q = p + 1 + rem;
  const int op = boff[p], wp = boff[p + 1] - op, oq = boff[q], wq = boff[q + 1] - oq;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // warp w computes the 16x8 tile (rows 16*(w>>2)... of the 32x32 product G_p^T G_q:
  // 32x32 = 2 row tiles x 4 col tiles = 8 tiles, 2 per warp
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  double np2 = 0.0, nq2 = 0.0;
  for (int r0 = 0; r0 < mp; r0 += 16) {
    for (int i = threadIdx.x; i < 16 * 32; i += blockDim.x) {
      int r = i & 15, c = i >> 4;
      sX[0][r][c] = (c < wp) ? Gw[(size_t)(op + c) * mp + r0 + r] : 0.0;
      sX[1][r][c] = (c < wq) ? Gw[(size_t)(oq + c) * mp + r0 + r] : 0.0;
    }
    __syncthreads();
    // column norms (threads 0..31 for p, 32..63 for q)
    if (threadIdx.x < 64) {
      int b = threadIdx.x >> 5, c = threadIdx.x & 31;
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < 16; ++r) s += sX[b][r][c] * sX[b][r][c];
      if (b == 0) np2 += s; else nq2 += s;
    }
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
      int tile = warp * 2 + tt;       // 0..7
      int ti = tile >> 2, tj = tile & 3;
      double a[8], bb[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = sX[0][4 * t + (i >> 1)][16 * ti + g + 8 * (i & 1)];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = sX[1][4 * t + j][8 * tj + g];
      dmma16816(acc[tt], a, bb);
    }
    __syncthreads();
  }
  double fro = 0.0;
#pragma unroll
  for (int tt = 0; tt < 2; ++tt)
#pragma unroll
    for (int i = 0; i < 4; ++i) fro += acc[tt][i] * acc[tt][i];
  fro = warp_sum_d(fro);
  if (threadIdx.x < 64) {
    // reduce the column norms of this lane's block
    double v = (threadIdx.x < 32) ? np2 : nq2;
    v = warp_sum_d(v);
    if (lane == 0) red[warp][1] = v;
  }
  if (lane == 0) red[warp][0] = fro;
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = red[0][0] + red[1][0] + red[2][0] + red[3][0];
    double a = red[0][1], b = red[1][1];
    double den = a * b;
    w[p * nb + q] = (den > 0.0) ? f / den : 0.0;
  }
}

}  // namespace jac
