// dense.cu -- contractions of the mixed-precision phases (Sec. 4, last paragraphs: the outer
// Jacobi iteration is self-correcting, so early sweeps may use a less accurate inner solution as
// long as the transforms finally applied to G are (J-)unitary to working precision).
//
//   Phase 1 (FP32 copy): k_gram32 / k_update32 are the gram and update of a step on an FP32
//     copy of G and an FP32 accumulator of V; no J-orthogonalization per pivot.
//   Phase 2 (transfer): the accumulated V is made J-unitary in FP64 by Newton-Schulz,
//     M = V^T J_r V - J_c (k_gemm64, symmetric tiles), V <- V - V (J_c M) / 2 (the correction
//     is small: k_gemm32 in FP32), then G = G_in V (k_gemm64).
//   Phase 3 continues with the FP64 step kernels.
#include <cooperative_groups.h>

#include "jacobi_common.cuh"

namespace cg = cooperative_groups;

namespace jac {

__device__ __forceinline__ int pcol(int c, int wp, int op, int oq) { return c < wp ? op + c : oq + (c - wp); }

// ----------------------------------------------------------------------------- FP32 gram
// Grid (half * CS, nprob), cluster (CS,1,1), 128 threads.  Thread (ty = tid / 8, tx = tid % 8) owns
// rows 4ty..4ty+3 and columns 8tx..8tx+7 of the 64 x 64 partial.  Partials are added through
// distributed shared memory and written to Ap (FP64 storage, FP32 accuracy).
#define G32_RS 32
__global__ void __launch_bounds__(128) k_gram32(const JacProb* __restrict__ probs, int s, int CS) {
  __shared__ __align__(16) float Xs[G32_RS][JAC_KMAX];
  __shared__ float Cs[JAC_KMAX][JAC_KMAX + 1];
  cg::cluster_group cluster = cg::this_cluster();
  const JacProb& a = probs[blockIdx.y];
  const int pair = blockIdx.x / CS;
  const int crank = (int)cluster.block_rank();
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || (a.cached && a.cached[pair])) return;  // uniform
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq;
  const float* G32 = a.G32;
  const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
  const int rpc = ((a.mp / CS + 15) & ~15);
  const int r_begin = min(a.mp, crank * rpc), r_end = min(a.mp, r_begin + rpc);
  float acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.0f;
  for (int r0 = r_begin; r0 < r_end; r0 += G32_RS) {
    const int rs = min(G32_RS, r_end - r0);
    __syncthreads();
    {  // loads first, then stores: one global latency per slab
      constexpr int NLD = JAC_KMAX * G32_RS / 128;
      float v[NLD];
#pragma unroll
      for (int u = 0; u < NLD; ++u) {
        const int idx = tid + u * 128, c = idx / G32_RS, r = idx % G32_RS;
        v[u] = (c < k && r < rs) ? __ldg(G32 + (size_t)pcol(c, wp, op, oq) * a.mp + r0 + r) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < NLD; ++u) {
        const int idx = tid + u * 128;
        Xs[idx % G32_RS][idx / G32_RS] = v[u];
      }
    }
    __syncthreads();
    for (int r = 0; r < rs; ++r) {
      const float4 xi = *reinterpret_cast<const float4*>(&Xs[r][4 * ty]);
      const float4 xj0 = *reinterpret_cast<const float4*>(&Xs[r][8 * tx]);
      const float4 xj1 = *reinterpret_cast<const float4*>(&Xs[r][8 * tx + 4]);
      const float vi[4] = {xi.x, xi.y, xi.z, xi.w};
      const float vj[8] = {xj0.x, xj0.y, xj0.z, xj0.w, xj1.x, xj1.y, xj1.z, xj1.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(vi[u], vj[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) Cs[4 * ty + u][8 * tx + v] = acc[u][v];
  cluster.sync();
  const int tot = k * k, per = (tot + CS - 1) / CS;
  const int e0 = crank * per, e1 = min(tot, e0 + per);
  double* out = a.Ap + (size_t)pair * a.apld * a.apld;
  for (int e = e0 + tid; e < e1; e += 128) {
    const int i = e % k, j = e / k;
    float part[16];  // all remote loads issued before the (fixed-order) sum
#pragma unroll
    for (int rk = 0; rk < 16; ++rk)
      part[rk] = (rk < CS) ? cluster.map_shared_rank(&Cs[0][0], rk)[i * (JAC_KMAX + 1) + j] : 0.0f;
    float sum = 0.0f;
#pragma unroll
    for (int rk = 0; rk < 16; ++rk) sum += part[rk];
    out[j * a.apld + i] = (double)sum;
  }
  cluster.sync();
}

// ----------------------------------------------------------------------------- FP32 update
// Grid (half, nslab, nprob), 256 threads; slab = 64 rows of G32 (y < gslabs) or V32.  Y = X V_P
// in FP32 with V_P read from the FP64 pivot output.  Thread (ty = tid / 16, tx = tid % 16) owns
// rows 4ty..+3 and columns 4tx..+3.
__global__ void __launch_bounds__(256) k_update32(const JacProb* __restrict__ probs, int s, int gslabs) {
  __shared__ __align__(16) float Bs[JAC_KMAX][JAC_KMAX + 4];  // V_P[c][j] row-major in c
  __shared__ __align__(16) float Xs[64][JAC_KMAX + 4];        // X[r][c]
  const JacProb& a = probs[blockIdx.z];
  const int pair = blockIdx.x;
  if (!a.active || s >= a.nsteps || pair >= a.counts[s] || a.skip[pair]) return;
  const int* sp = a.pairs + (size_t)s * a.half * 2;
  const int p = sp[2 * pair], q = sp[2 * pair + 1];
  const int op = a.boff[p], wp = a.boff[p + 1] - op, oq = a.boff[q], wq = a.boff[q + 1] - oq;
  const int k = wp + wq;
  float* base;
  int ld, r0, rs;
  if ((int)blockIdx.y < gslabs) {
    base = a.G32;
    ld = a.mp;
    r0 = blockIdx.y * 64;
    rs = min(64, a.mp - r0);
  } else {
    if (!a.V32) return;
    base = a.V32;
    ld = a.np;
    r0 = (blockIdx.y - gslabs) * 64;
    rs = min(64, a.np - r0);
  }
  if (rs <= 0) return;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const double* V = a.vp + (size_t)pair * a.apld * a.apld;
  {  // all loads of the thread first, then the stores: one global latency, not one per element
    constexpr int NB = JAC_KMAX * JAC_KMAX / 256, NX = JAC_KMAX * 64 / 256;
    float vb[NB], vx[NX];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = tid + u * 256, c = idx % JAC_KMAX, j = idx / JAC_KMAX;
      vb[u] = (c < k && j < k) ? (float)__ldg(V + j * a.apld + c) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int idx = tid + u * 256, r = idx % 64, c = idx / 64;
      vx[u] = (c < k && r < rs) ? base[(size_t)pcol(c, wp, op, oq) * ld + r0 + r] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = tid + u * 256;
      Bs[idx % JAC_KMAX][idx / JAC_KMAX] = vb[u];
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int idx = tid + u * 256;
      Xs[idx % 64][idx / 64] = vx[u];
    }
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
  for (int c = 0; c < k; ++c) {
    const float4 b = *reinterpret_cast<const float4*>(&Bs[c][4 * tx]);
    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float x = Xs[4 * ty + u][c];
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(x, bv[v], acc[u][v]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Xs[4 * ty + u][4 * tx + v] = acc[u][v];
  __syncthreads();
  for (int idx = tid; idx < k * rs; idx += 256) {
    const int r = idx % rs, c = idx / rs;
    base[(size_t)pcol(c, wp, op, oq) * ld + r0 + r] = Xs[r][c];
  }
}

// ----------------------------------------------------------------------------- FP64 GEMM
// C = op(A) * diag(sb) * op(B) - diag(dsub)  (FP64 mma m16n8k16), column-major, C is Mr x Nc;
// blockIdx.z selects a batch member at element strides sa, sbb, sc.
//   transB = 1: op(B)[r][j] = B[r * ldb + j]; else B[j * ldb + r].
//   transA = 1: op(A)[i][r] = A[i * lda + r]  (A stored K x Mr: C = A^T B)
//   transA = 0: op(A)[i][r] = A[r * lda + i]  (A stored Mr x K)
//   sb: optional +-1 per r (row signs of B); dsub: optional, subtracted on the diagonal.
//   sym = 1: only tiles with tile_j >= tile_i are computed, and only entries j >= i are stored,
//            each mirrored (C exactly symmetric; Mr == Nc).
// Grid (ceil(Mr/32), ceil(Nc/32)); 128 threads; K chunk 32.
#define DG_T 32
#define DG_LD (DG_T + 2)
__global__ void __launch_bounds__(128) k_gemm64(int Mr, int Nc, int K, const double* __restrict__ A, int lda,
                                               int transA, const double* __restrict__ B, int ldb,
                                               const int8_t* __restrict__ sb, const int8_t* __restrict__ dsub,
                                               double* __restrict__ C, int ldc, int sym, int transB, long long sa,
                                               long long sbb, long long sc) {
  __shared__ __align__(16) double As[DG_T * DG_LD];  // [i][r]
  __shared__ __align__(16) double Bs[DG_T * DG_LD];  // [j][r]
  A += (size_t)blockIdx.z * sa;
  B += (size_t)blockIdx.z * sbb;
  C += (size_t)blockIdx.z * sc;
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (sym && bj < bi) return;
  const int i0 = bi * DG_T, j0 = bj * DG_T;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int wi = (warp & 1) * 16, wj = (warp >> 1) * 16;
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int k0 = 0; k0 < K; k0 += DG_T) {
    __syncthreads();
    for (int idx = tid; idx < DG_T * DG_T; idx += 128) {
      int i, r;
      double va = 0.0;
      if (transA) {
        r = idx % DG_T;
        i = idx / DG_T;
        if (i0 + i < Mr && k0 + r < K) va = A[(size_t)(i0 + i) * lda + k0 + r];
      } else {
        i = idx % DG_T;
        r = idx / DG_T;
        if (i0 + i < Mr && k0 + r < K) va = A[(size_t)(k0 + r) * lda + i0 + i];
      }
      As[i * DG_LD + r] = va;
      int rb, jb;
      double vb = 0.0;
      if (transB) {  // op(B)[r][j] = B[r * ldb + j]
        jb = idx % DG_T;
        rb = idx / DG_T;
        if (j0 + jb < Nc && k0 + rb < K) vb = B[(size_t)(k0 + rb) * ldb + j0 + jb];
      } else {
        rb = idx % DG_T;
        jb = idx / DG_T;
        if (j0 + jb < Nc && k0 + rb < K) vb = B[(size_t)(j0 + jb) * ldb + k0 + rb];
      }
      if (sb && k0 + rb < K && sb[k0 + rb] < 0) vb = -vb;
      Bs[jb * DG_LD + rb] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < DG_T; kq += 16) {
      const double* xa0 = As + (wi + g) * DG_LD + kq + 4 * t;
      const double* xa1 = xa0 + 8 * DG_LD;
      double2 a0 = *reinterpret_cast<const double2*>(xa0), a1 = *reinterpret_cast<const double2*>(xa0 + 2);
      double2 a2 = *reinterpret_cast<const double2*>(xa1), a3 = *reinterpret_cast<const double2*>(xa1 + 2);
      double av[8] = {a0.x, a2.x, a0.y, a2.y, a1.x, a3.x, a1.y, a3.y};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double* xb = Bs + (wj + 8 * h + g) * DG_LD + kq + 4 * t;
        double2 b0 = *reinterpret_cast<const double2*>(xb), b1 = *reinterpret_cast<const double2*>(xb + 2);
        double bv[4] = {b0.x, b0.y, b1.x, b1.y};
        dmma16816(acc[h], av, bv);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + wi + g + 8 * (u >> 1), j = j0 + wj + 8 * h + 2 * t + (u & 1);
      if (i < Mr && j < Nc && (!sym || j >= i)) {
        double v = acc[h][u];
        if (dsub && i == j) v -= (dsub[i] < 0) ? -1.0 : 1.0;
        C[(size_t)j * ldc + i] = v;
        if (sym && j > i) C[(size_t)i * ldc + j] = v;  // exactly symmetric: (j, i) is never computed
      }
    }
}

// ----------------------------------------------------------------------------- FP32 GEMM
// T = Af (Mr x K) * Bf (K x Nc), FP32, column-major; then V[i][j] -= 0.5 * T[i][j] in FP64.
// Grid (ceil(Mr/64), ceil(Nc/64)), 256 threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_ns_correct(int Mr, int Nc, int K, const float* __restrict__ Af, int lda,
                                                   const float* __restrict__ Bf, int ldb, double* __restrict__ V,
                                                   int ldv) {
  __shared__ float As[16][64 + 4];  // [r][i]
  __shared__ float Bs[16][64 + 4];  // [r][j]
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    __syncthreads();
    for (int idx = tid; idx < 16 * 64; idx += 256) {
      const int i = idx % 64, r = idx / 64;
      As[r][i] = (i0 + i < Mr && k0 + r < K) ? Af[(size_t)(k0 + r) * lda + i0 + i] : 0.0f;
      const int rb = idx % 16, jb = idx / 16;
      Bs[rb][jb] = (j0 + jb < Nc && k0 + rb < K) ? Bf[(size_t)(j0 + jb) * ldb + k0 + rb] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float4 x = *reinterpret_cast<const float4*>(&As[r][4 * ty]);
      const float4 y = *reinterpret_cast<const float4*>(&Bs[r][4 * tx]);
      const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + 4 * ty + u, j = j0 + 4 * tx + v;
      if (i < Mr && j < Nc) V[(size_t)j * ldv + i] -= 0.5 * (double)acc[u][v];
    }
}

// ----------------------------------------------------------------------------- helpers
// dst (FP32, rows x cols, ld_d) = src (FP64, ld_s), optionally row-signed: dst[i][j] = s_i src[i][j]
__global__ void k_cvt64to32(int rows, int cols, const double* __restrict__ src, int lds, float* __restrict__ dst,
                            int ldd, const int8_t* __restrict__ rsign) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    float v = (float)src[(size_t)j * lds + i];
    if (rsign && rsign[i] < 0) v = -v;
    dst[(size_t)j * ldd + i] = v;
  }
}

// dst (FP64) = src (FP32)
__global__ void k_cvt32to64(int rows, int cols, const float* __restrict__ src, int lds, double* __restrict__ dst,
                            int ldd) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[(size_t)j * ldd + i] = (double)src[(size_t)j * lds + i];
  }
}

// max |M| over an n x n FP64 matrix into *out (as the bits of a non-negative double, atomicMax)
__global__ void k_absmax64(int n, const double* __restrict__ M, int ldm, unsigned long long* __restrict__ out) {
  double mloc = 0.0;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    mloc = fmax(mloc, fabs(M[(size_t)j * ldm + i]));
  }
  mloc = warp_max_d(mloc);
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mloc));
}

// FP32 copies <-> FP64 working arrays of every problem (same layouts: Gw/G32 ld mp, Vw/V32 ld np).
// to64 = 0: G32 = Gw, V32 = Vw (rounded); to64 = 1: Gw = G32, Vw = V32.  Grid (blocks, nprob).
__global__ void k_lowp_copy(const JacProb* __restrict__ probs, int to64) {
  const JacProb& a = probs[blockIdx.y];
  if (!a.G32) return;
  const size_t ng = (size_t)a.mp * a.n;
  const size_t nv = (a.V32 && a.Vw) ? (size_t)a.np * a.n : 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ng + nv; e += (size_t)gridDim.x * blockDim.x) {
    if (e < ng) {
      if (to64) a.Gw[e] = (double)a.G32[e];
      else a.G32[e] = (float)a.Gw[e];
    } else {
      const size_t f = e - ng;
      if (to64) a.Vw[f] = (double)a.V32[f];
      else a.V32[f] = (float)a.Vw[f];
    }
  }
}

}  // namespace jac
