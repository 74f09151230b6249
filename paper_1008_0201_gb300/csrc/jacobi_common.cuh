// jacobi_common.cuh -- shared device helpers and internal types of the GB300 Jacobi library.
//
// Arithmetic placement on GB300 (measured on the target: FP64 FFMA ~1.0 TFLOP/s, mma.sync
// m16n8k16 f64 ~1.0 TFLOP/s, FP16 mma.sync ~600 TFLOP/s, FP32 FFMA ~74 TFLOP/s, FP64 sqrt/div
// ~650 cycles latency):
//   - every FP64 contraction (pivot Gram block, block update, J-orthogonality residual of V_P)
//     is an FP64-accurate sum of exact FP16 tensor-core digit products (ozaki.cuh), or, when
//     selected, runs on the FP64 tensor path, mma.sync.m16n8k16.f64;
//   - the 2x2 rotation angles are computed in FP32 on a shifted representation that keeps
//     relative precision near convergence; FP64 enters them only through A_P.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define JAC_KMAX 64          // largest pivot block order k = w_p + w_q handled (w <= 32)
#define JAC_WMAX 32          // largest block width
#define JAC_INNER_MAX_SWEEPS 40

// device error flags (OR-ed into a global word; never trapped)
#define JAC_DEVERR_NOTPD 1u
#define JAC_DEVERR_INNER_LIMIT 2u
#define JAC_DEVERR_NONFINITE 4u
#define JAC_DEVERR_HANDOVER 8u  // a pivot block went to the FP64 pivot kernel (not an error)
#define JAC_DEVERR_TIMEOUT 16u  // a bounded wait on a TMA load or tensor-core MMA gave up

namespace jac {

// D = A(16x16) * B(16x8) + C, f64.  Fragment layout (checked on the target against a CPU
// product): lane = 4g + t; A element (row g + 8*(i&1), k = 4t + (i>>1)) in a[i]; B element
// (k = 4t + j, col g) in b[j]; C/D element (row g + 8*(i>>1), col 2t + (i&1)) in c[i].
// Any permutation of k applied to both A and B gives the same product; this one makes the
// four k-values of a thread contiguous.
__device__ __forceinline__ void dmma16816(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
        "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Inner step s of the circle (round-robin) ordering on kk (even) positions, position kk-1 fixed:
// the pair (li < lj) of slot w.
__device__ __forceinline__ void rr_inner_pair(int kk, int s, int w, int& li, int& lj) {
  const int L = kk - 1;
  if (w == 0) {
    li = s;
    lj = kk - 1;
  } else {
    int x = s + w, y = s - w;
    if (x >= L) x -= L;
    if (y < 0) y += L;
    li = min(x, y);
    lj = max(x, y);
  }
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace jac

// ------------------------------------------------------------------ internal problem view
// One problem of a batch (a single solve is a batch of one).  Internal layout: Gw is (mp x n)
// column-major, ld = mp = m rounded up to 16 with zero rows; columns are sorted so that
// J = diag(I_npos, -I).  Vw is (np x n), np = n rounded up to 16, rows in input order.  Block b
// spans columns [boff[b], boff[b+1]).  The step kernels take an array of these and a step index
// s, and index the problem by a grid dimension; a problem with active = 0 is skipped.
struct JacProb {
  double* Gw;        // FP64 factor
  double* Vw;        // FP64 V (NULL if not accumulated)
  float* G32;        // FP32 copies used by the FP32 sweeps (NULL otherwise)
  float* V32;
  int mp, np, n, nb, half, nsteps;
  const int* boff;   // [nb+1]
  const int8_t* Js;  // [n] internal (sorted) signs
  const int* pairs;  // [nsteps][half][2]
  const int* counts; // [nsteps]
  double* Ap;        // [half][apld * apld] Gram blocks
  double* vp;        // [half][apld * apld] pivot transforms V_P
  int apld;          // leading dimension of a pivot block (the pivot capacity of its class)
  int active;        // 0: converged or failed, every kernel skips the problem
  double tol;        // rotation threshold of the problem (batched convergence test)
  int* skip;         // [half]
  struct PairStat* stats;  // [nsteps][half]
  unsigned* pflags;  // JAC_DEVERR_* bits of this problem
  // Pair cache (NULL: off).  A pair whose two blocks have not changed since it was last
  // evaluated in the same (step, slot), and which did not rotate then, would give bitwise the
  // same Gram block, decision and statistics: its step kernels return at once.
  int* cached;       // [half] 1: the pair of this slot is cached in the current step
  int4* pver;        // [nsteps][half] (p, q, version of p, version of q) at the last evaluation;
                     // version of p = -1 if the pair rotated
  int* bver;         // [nb] block versions, bumped when a pair containing the block rotates
};

// User-side buffers of one problem and its finalize scratch.
struct JacIO {
  double* G;           // user factor (device), m x n, read at set-up and overwritten at the end
  int ldg, m;
  const int8_t* J;     // user signs (device), NULL for J = I
  int* perm_in;        // [n] internal column c holds input column perm_in[c]
  double* lambda;      // [n]
  double* U;           // may be NULL
  int ldu;
  double* V;           // may be NULL
  int ldv;
  const double* Vinit; // NULL: V starts as I; else V starts as this n x n matrix (ld ldvi)
  int ldvi;
  double* nrm2;        // [n] scratch
  double* lam;         // [n] scratch
  int* rank;           // [n] scratch
  int flags;           // bit 0: non-finite input, bit 1: invalid sign entry
  int sweeps;          // sweeps run while active
  long long rotations;
};

struct PairStat;
struct PivotParams {
  double tol;        // outer rotation threshold; <= 0: max(n, tol_m sqrt(mp)) tol_eps for a problem
  double tol_eps;    // of order n with mp (padded) rows: the FP32 Gram resolves no less than ~eps sqrt(m)
  double tol_m;
  int factor;        // 0 unpivoted, 2 sign-pivoted
  int ns_mode;       // 1: make V_P J-unitary in FP64 (Newton-Schulz); 0: leave the FP32 transform
  int oriented;      // 1: block-oriented inner sweep (one sweep; cross block only after step 0)
  int oz;            // FP64 Gram / update / V_P residual from exact FP16 digit products (ozaki.cuh)
};

// per (step, pair) record written by the pivot kernel, reduced per sweep
struct PairStat {
  double max_scaled;  // max |a_ij|/sqrt(a_ii a_jj) over the pivot block
  double off2_cross;  // sum over the cross block A_pq of |a_ij|^2 (one triangle)
  double off2_diag;   // sum over the strictly upper parts of A_pp and A_qq of |a_ij|^2
  double trace;       // sum of a_ii over the pivot block
  int rotations;      // inner rotations applied (0: the pair was already diagonal)
  int inner_sweeps;
  int ns_steps;
  int active;         // 1 iff some |a_ij| > tol sqrt(a_ii a_jj): the FP64 convergence test
  int evaluated;      // 1: the pivot ran for this pair in this sweep; 0: cached (pair_cache.cu)
  long long cyc[4];   // SM clocks of the pivot phases: stats, Cholesky, inner sweeps, J-orth.
};

struct SweepRecord {
  double max_scaled;
  double off2;
  double trace;
  long long rotations;
  long long pivots_rotated;
  long long cyc[4];
  long long ns_steps;
  long long inner_sweeps;
  long long evaluated;  // pairs whose Gram block and pivot ran (not cached)
  unsigned int err;
  int pad;
};
