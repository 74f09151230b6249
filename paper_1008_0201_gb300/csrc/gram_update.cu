// gram_update.cu -- the two dense contractions of a parallel step (Sec. 2.3):
//   gram:   A_P = [G_p G_q]^* [G_p G_q]                    (Eq. (3.4))
//   update: [G_p G_q] <- [G_p G_q] V_P,  [V_p V_q] <- [V_p V_q] V_P   (Algorithm 3.4)
// Both run on the FP64 tensor path (mma.sync m16n8k16 f64).  The pairs of a step are disjoint,
// so every CTA owns its columns and the update is in place.  Problems of a batch are indexed by
// grid dimension y (gram, pivot) or z (update).
#include <cooperative_groups.h>

#include "jacobi_common.cuh"

namespace cg = cooperative_groups;

namespace jac {

// smem row stride of a 64-row column slab: 66 doubles = 528 B keeps the 16-byte fragment
// loads of the 8 column groups in a warp on distinct bank quads.
#define GRAM_RS 64
#define GRAM_LDS (GRAM_RS + 2)
#define GRAM_LDC (JAC_KMAX + 1)

__device__ __forceinline__ int pair_col(int c, int wp, int op, int oq) { return c < wp ? op + c : oq + (c - wp); }

// Grid (half * CS, nprob), cluster (CS,1,1): the CS CTAs of a cluster share one pair and split
// its rows; their k x k partial sums are added through distributed shared memory, each CTA
// reducing and storing 1/CS of the entries.  Output Ap[pair] (ld apld, k x k used), symmetric,
// column-major.
__global__ void __launch_bounds__(128) k_gram(const JacProb* __restrict__ probs, int s, int CS) {
  extern __shared__ __align__(16) double gsm[];
  double* Xs = gsm;                                  // [KMAX cols][GRAM_LDS rows]
  double* Cs = gsm + JAC_KMAX * GRAM_LDS;            // [KMAX][GRAM_LDC]
  cg::cluster_group cluster = cg::this_cluster();
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x / CS;
  const int crank = (int)cluster.block_rank();
  // uniform over the cluster: no cluster barrier is pending
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || (a.cached && a.cached[pair])) return;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq, KP = (k + 15) & ~15;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nti = KP / 16, ntj = KP / 8, ntiles = nti * ntj;
  // rows of this CTA
  const int rpc = ((a.mp / CS + 15) & ~15);
  const int r_begin = min(a.mp, crank * rpc), r_end = min(a.mp, r_begin + rpc);

  double acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

  for (int r0 = r_begin; r0 < r_end; r0 += GRAM_RS) {
    const int rs = min(GRAM_RS, r_end - r0);  // multiple of 16
    __syncthreads();
    // load the slab: column c rows r0..r0+rs-1 (zero columns k..KP-1); all of a thread's loads
    // are issued before its stores
    {
      constexpr int NLD = JAC_KMAX * (GRAM_RS / 2) / 128;
      const int tot = KP * (rs / 2);
      double2 v[NLD];
#pragma unroll
      for (int u = 0; u < NLD; ++u) {
        const int idx = threadIdx.x + u * 128, c = idx / (rs / 2), rr = (idx % (rs / 2)) * 2;
        v[u] = (idx < tot && c < k)
                   ? __ldg(reinterpret_cast<const double2*>(a.Gw + (size_t)pair_col(c, wp, op, oq) * a.mp + r0 + rr))
                   : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < NLD; ++u) {
        const int idx = threadIdx.x + u * 128, c = idx / (rs / 2), rr = (idx % (rs / 2)) * 2;
        if (idx < tot) *reinterpret_cast<double2*>(Xs + c * GRAM_LDS + rr) = v[u];
      }
    }
    __syncthreads();
    for (int kk = 0; kk < rs; kk += 16) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int tile = warp + 4 * u;
        if (tile < ntiles) {
          const int ti = tile / ntj, tj = tile % ntj;
          if (8 * tj + 7 < 16 * ti) continue;  // strictly below the diagonal: mirrored later
          double av[8], bv[4];
          const double* xa0 = Xs + (16 * ti + g) * GRAM_LDS + kk + 4 * t;
          const double* xa1 = xa0 + 8 * GRAM_LDS;
          const double* xb = Xs + (8 * tj + g) * GRAM_LDS + kk + 4 * t;
          double2 a0 = *reinterpret_cast<const double2*>(xa0), a1 = *reinterpret_cast<const double2*>(xa0 + 2);
          double2 a2 = *reinterpret_cast<const double2*>(xa1), a3 = *reinterpret_cast<const double2*>(xa1 + 2);
          double2 b0 = *reinterpret_cast<const double2*>(xb), b1 = *reinterpret_cast<const double2*>(xb + 2);
          // a[i]: row g + 8*(i&1), k = 4t + (i>>1)
          av[0] = a0.x; av[2] = a0.y; av[4] = a1.x; av[6] = a1.y;
          av[1] = a2.x; av[3] = a2.y; av[5] = a3.x; av[7] = a3.y;
          bv[0] = b0.x; bv[1] = b0.y; bv[2] = b1.x; bv[3] = b1.y;
          dmma16816(acc[u], av, bv);
        }
      }
    }
  }
  // partial -> own shared memory (upper tiles and their mirror)
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int tile = warp + 4 * u;
    if (tile < ntiles) {
      const int ti = tile / ntj, tj = tile % ntj;
      if (8 * tj + 7 < 16 * ti) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = 16 * ti + g + 8 * (v >> 1), c = 8 * tj + 2 * t + (v & 1);
        // each entry written once: (r, c) with c >= r and its mirror; (r, c) with c < r of a
        // tile crossing the diagonal comes from the tile holding (c, r)
        if (c >= r) {
          Cs[r * GRAM_LDC + c] = acc[u][v];
          Cs[c * GRAM_LDC + r] = acc[u][v];
        }
      }
    }
  }
  cluster.sync();
  // reduce entries e in [crank*KP*KP/CS, ...) over the CS partials, fixed order
  const int tot = k * k;
  const int per = (tot + CS - 1) / CS;
  const int e0 = crank * per, e1 = min(tot, e0 + per);
  double* out = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int i = e % k, j = e / k;
    double part[16];  // all remote loads issued before the (fixed-order) sum
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) part[rk] = (rk < CS) ? cluster.map_shared_rank(Cs, rk)[i * GRAM_LDC + j] : 0.0;
    double sum = 0.0;
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) sum += part[rk];
    out[j * a.apld + i] = sum;
  }
  cluster.sync();  // keep every partial alive until all remote reads are done
}

// Grid (half, nslab, nprob); slab y covers 64 rows of Gw (y < gslabs) or of Vw.  128 threads.
// Y = X V_P with X the slab (64 x k), V_P (k x k) from the pivot kernel; written in place.
#define UPD_RS 64
#define UPD_LD (JAC_KMAX + 2)
__global__ void __launch_bounds__(128) k_update(const JacProb* __restrict__ probs, int s, int gslabs) {
  extern __shared__ __align__(16) double usm[];
  double* Bs = usm;                       // V_P: [col j][UPD_LD] (k index contiguous)
  double* Xs = usm + JAC_KMAX * UPD_LD;   // X slab row-major: [row][UPD_LD]
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
    r0 = blockIdx.y * UPD_RS;
    rs = min(UPD_RS, a.mp - r0);
  } else {
    if (!a.Vw) return;
    base = a.Vw;
    ld = a.np;
    r0 = (blockIdx.y - gslabs) * UPD_RS;
    rs = min(UPD_RS, a.np - r0);
  }
  if (rs <= 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const double* V = a.vp + (size_t)pair * a.apld * a.apld;
  for (int idx = threadIdx.x; idx < KP * KP; idx += blockDim.x) {
    const int c = idx % KP, j = idx / KP;  // V_P[c][j], column-major source
    Bs[j * UPD_LD + c] = (c < k && j < k) ? V[j * a.apld + c] : 0.0;
  }
  for (int idx = threadIdx.x; idx < KP * rs; idx += blockDim.x) {
    const int r = idx % rs, c = idx / rs;
    Xs[r * UPD_LD + c] = (c < k) ? base[(size_t)pair_col(c, wp, op, oq) * ld + r0 + r] : 0.0;
  }
  __syncthreads();
  const int nti = rs / 16, ntj = KP / 8, ntiles = nti * ntj;
  double acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int kk = 0; kk < KP; kk += 16) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int tile = warp + 4 * u;
      if (tile < ntiles) {
        const int ti = tile / ntj, tj = tile % ntj;
        const double* xa0 = Xs + (16 * ti + g) * UPD_LD + kk + 4 * t;
        const double* xa1 = xa0 + 8 * UPD_LD;
        const double* xb = Bs + (8 * tj + g) * UPD_LD + kk + 4 * t;
        double2 a0 = *reinterpret_cast<const double2*>(xa0), a1 = *reinterpret_cast<const double2*>(xa0 + 2);
        double2 a2 = *reinterpret_cast<const double2*>(xa1), a3 = *reinterpret_cast<const double2*>(xa1 + 2);
        double2 b0 = *reinterpret_cast<const double2*>(xb), b1 = *reinterpret_cast<const double2*>(xb + 2);
        double av[8], bv[4];
        av[0] = a0.x; av[2] = a0.y; av[4] = a1.x; av[6] = a1.y;
        av[1] = a2.x; av[3] = a2.y; av[5] = a3.x; av[7] = a3.y;
        bv[0] = b0.x; bv[1] = b0.y; bv[2] = b1.x; bv[3] = b1.y;
        dmma16816(acc[u], av, bv);
      }
    }
  }
  __syncthreads();  // all reads of Xs done: reuse it for the result
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int tile = warp + 4 * u;
    if (tile < ntiles) {
      const int ti = tile / ntj, tj = tile % ntj;
      const int r = 16 * ti + g, c = 8 * tj + 2 * t;
      *reinterpret_cast<double2*>(Xs + r * UPD_LD + c) = make_double2(acc[u][0], acc[u][1]);
      *reinterpret_cast<double2*>(Xs + (r + 8) * UPD_LD + c) = make_double2(acc[u][2], acc[u][3]);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * rs; idx += blockDim.x) {
    const int r = idx % rs, c = idx / rs;
    base[(size_t)pair_col(c, wp, op, oq) * ld + r0 + r] = Xs[r * UPD_LD + c];
  }
}

}  // namespace jac
