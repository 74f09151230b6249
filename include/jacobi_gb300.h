/*
 * jacobi_gb300.h -- C ABI of the GB300 (sm_103a) block one-sided Jacobi library.
 *
 * The library computes the eigendecomposition of a Hermitian matrix given by a factor,
 *     H = G J G^*,   G: m x n,   J = diag(j_1..j_n), j_k in {+1, -1},
 * by the parallel one-sided block Jacobi method of Singer, Singer, Novakovic, Uscumlic and
 * Dunjko, "Novel Modifications of Parallel Jacobi Algorithms":
 *   - J = I: the one-sided trigonometric algorithm (Sec. 2.1, Sec. 3.1; H positive definite),
 *   - J != I: the one-sided hyperbolic algorithm, i.e. the hyperbolic SVD G = U Sigma V^{-1}
 *     with V^* J V = J (Sec. 1, Eq. (1.3); Sec. 3.2, Algorithm 3.4).
 * G is right-multiplied by J-unitary block transforms V_P (Sec. 2.3) over disjoint pairs of
 * column blocks chosen by a parallel ordering (Sec. 2.4) until its columns are orthogonal.
 * Then lambda_k = j_k ||g_k||^2 and u_k = g_k / ||g_k|| (Sec. 3.2).
 *
 * Conventions common to every entry point:
 *   - Matrices are column-major with a leading dimension (ld >= rows).  Real data is IEEE
 *     double; complex data (dtype JAC_C128) is interleaved (re, im) double pairs and leading
 *     dimensions count complex elements.
 *   - Array arguments (G, J, lambda, U, V, ...) are DEVICE pointers on the current CUDA
 *     device, owned by the caller.  opts and info are HOST pointers.
 *   - All work is ordered on `stream` (NULL = the legacy default stream).  Each call returns
 *     after the solve has finished: the sweep loop reads one small convergence record back
 *     per sweep.  Internal scratch is taken from the stream-ordered allocator
 *     (cudaMallocAsync) and returned before the call returns.
 *   - Errors are reported by the return value and never by abort or trap.  A negative value
 *     -k means argument k (1-based) is invalid; nothing has been written then.  Positive
 *     values are the jac_status codes below; outputs are then unspecified except for info.
 *   - Outputs are returned in ascending lambda order; ties keep the input column order.
 */
#ifndef JACOBI_GB300_H
#define JACOBI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the runtime's stream handle); NULL selects the legacy default stream. */
typedef struct CUstream_st* jac_stream_t;

/* Return codes (>= 0).  -k: argument k invalid. */
enum jac_status {
  JAC_OK = 0,
  JAC_ENOTCONV = 1,   /* max_sweeps reached with rotations still applied in the last sweep */
  JAC_ENOTPD = 2,     /* a pivot block G_P^* G_P was not positive definite in its Cholesky
                         factorization: G lacks full column rank (Sec. 3.2 requires it) */
  JAC_ENONFINITE = 3, /* G holds a NaN or Inf */
  JAC_ECUDA = 4,      /* a CUDA runtime call failed */
  JAC_ENOMEM = 5,     /* device scratch could not be allocated */
  JAC_EINTERNAL = 6   /* a bounded device loop hit its limit (reported, never trapped) */
};

/* Element type of G, U, V. */
enum jac_dtype { JAC_R64 = 0, JAC_C128 = 1 };

/* Parallel block ordering (Sec. 2.4). */
enum jac_ordering {
  JAC_ORDER_MODULUS = 0,      /* step k pairs the blocks {p<q: p+q = k mod nb}, nb steps */
  JAC_ORDER_MODULUS_MOD = 1,  /* modulus, plus the two left-over blocks on even steps */
  JAC_ORDER_ROUND_ROBIN = 2,  /* circle method: nb-1 perfect matchings */
  JAC_ORDER_CYCLE_WEIGHT = 3  /* per cycle: pairs by descending ||G_p^* G_q||_F^2 /
                                 (||G_p||_F^2 ||G_q||_F^2), greedily packed into steps;
                                 every pair once per cycle.  At most JAC_CYCLE_WEIGHT_MAX_NB
                                 blocks: a solve whose partition has more blocks is rejected
                                 as an invalid opts argument */
};

/* Largest block count of the per-cycle weight ordering (its greedy packing scans every
 * remaining pair once per step, O(nb^3) work in one CTA per cycle). */
#define JAC_CYCLE_WEIGHT_MAX_NB 512

/* Pivot block processing (Sec. 2.2). */
enum jac_block_mode {
  JAC_BLOCK_FULL = 0,     /* diagonalize each pivot block (full block: HF / HFSC, Sec. 2.2) */
  JAC_BLOCK_ORIENTED = 1  /* block-oriented (HB / HBSC, Sec. 2.2 and Algorithm 3.4): the first
                             step of a sweep annihilates every off-diagonal element of its pivot
                             blocks once, the other steps only the elements of the cross block
                             A_pq, once */
};

/* Factorization of the pivot block A_P = G_P^* G_P (Sec. 3.2). */
enum jac_factor {
  JAC_FACTOR_CHOL = 0,         /* unpivoted Cholesky (HF) */
  JAC_FACTOR_CHOL_DIAGPIV = 1, /* Cholesky with diagonal pivoting over the whole block (HFC, Sec. 3.2);
                                  J_P follows the pivot order */
  JAC_FACTOR_CHOL_SIGNPIV = 2  /* J_P-sign-pivoted Cholesky, Algorithm 3.3 (HFSC) */
};

/* Arithmetic of the sweeps (FP64 and FP32 return FP64-accurate results). */
enum jac_precision {
  JAC_PREC_FP64 = 0, /* every sweep: Gram, update and J-orthogonalization of V_P FP64-accurate
                        (products per opts->f64_products) */
  JAC_PREC_FP32 = 1, /* sweeps on an FP32 copy of G with FP32 Gram/update products until the scaled
                        off-norm reaches what FP32 resolves, then V is made J-unitary in FP64,
                        G = G_in V, and FP64 sweeps polish to tol (the outer iteration is
                        self-correcting, Sec. 4).  jacobi_hsvd / jacobi_eig_pd only. */
  JAC_PREC_FP32_ONLY = 2 /* every sweep on the FP32 copy, no FP64 polish: results accurate to
                            FP32 (eps = 2^-24); tol <= 0 selects max(n, 8 sqrt(m)) * 2^-24, the
                            smallest scaled off-diagonal an FP32 Gram of m rows resolves */
};

/* Arithmetic of the FP64 Gram, update and V_P J-orthogonality products (FP64 sweeps). */
enum jac_f64_products {
  JAC_F64_MMA = 0,    /* FP64 tensor-core mma (m16n8k16 f64) */
  JAC_F64_SPLIT16 = 1,/* exact FP16 tensor-core products of 7-bit digit slices of each operand,
                         8 slices, recombined once to FP64 (error-free splitting after Ozaki et
                         al.): each product term exact to 2^-53 of its operand group bounds.  The
                         update runs on the tcgen05 tensor cores (accumulators in tensor memory,
                         integer rounding to FP64), the Gram block on the warp-level FP16 mma */
  JAC_F64_SPLIT16_TC = 2 /* as JAC_F64_SPLIT16 with the Gram block on tcgen05 as well (same
                            results to FP64 accuracy; slower on GB300 today: its 128-row digit
                            groups leave the tensor-memory read-out latency exposed) */
};

typedef struct {
  int block_w;     /* target block-column width w; nb = max(2, 2*ceil(n/(2w))) blocks whose
                      widths differ by at most one (Sec. 3).  1 <= w <= 32 in this version. */
  int ordering;    /* enum jac_ordering */
  int block_mode;  /* enum jac_block_mode */
  int factor;      /* enum jac_factor */
  int precision;   /* enum jac_precision */
  int max_sweeps;  /* >= 1 */
  int want_v;      /* 1: accumulate and return V (n x n); 0: V is not touched */
  double tol;      /* rotate a pair (i,j) iff |a_ij| > tol sqrt(a_ii a_jj); <= 0 selects n*2^-53 */
  int f64_products;/* enum jac_f64_products */
  int fused_step;  /* 1: the FP32 sweeps of small problems run Gram, pivot and update of a pair in
                      one kernel (X_P read from and written to HBM once per step; m <= 96 rows for
                      pivot blocks of k <= 32 columns, m <= 192 for k <= 64); 0: three kernels per
                      step.  Same arithmetic either way (FP32 Gram and update products). */
} jac_opts;

typedef struct {
  int sweeps;              /* sweeps run (the last one applied no rotation when converged) */
  int converged;           /* 1 iff a sweep ended with no rotation */
  int status;              /* same as the return value */
  int steps_per_sweep;     /* parallel steps in the last sweep */
  long long rotations;     /* inner 2x2 rotations applied, all sweeps */
  long long pivots_rotated;/* pivot blocks transformed, all sweeps */
  double max_scaled_off;   /* last sweep: max |a_ij| / sqrt(a_ii a_jj) over all pairs seen */
  double off_rel;          /* last sweep: off_F(G^* G) / ||G||_F^2 estimated from the pivots */
  long long launches;      /* kernels launched by this call */
  int lowp_sweeps;         /* sweeps of the FP32 phase (JAC_PREC_FP32) */
  int global_ns_steps;     /* Newton-Schulz steps applied to the accumulated V after that phase */
  long long pivot_ns_steps;/* Newton-Schulz steps applied to pivot transforms V_P */
  long long pivot_cycles[4]; /* SM clocks summed over pivots: statistics, Cholesky, inner sweeps,
                                J-orthogonalization */
  double sweep_max_scaled[64]; /* per sweep (first 64): max |a_ij| / sqrt(a_ii a_jj) seen */
  long long inner_sweeps;  /* inner sweeps summed over the transformed pivot blocks */
  double sweep_ms[64];     /* per sweep (first 64): host wall time from its first launch to its
                              completion, the precision switch included (single solves) */
  long long pivots_rotated_lowp; /* of pivots_rotated: those of the FP32 sweeps */
  long long pairs_evaluated;     /* pivot pairs whose Gram block and pivot ran, all sweeps (pairs
                                    whose two blocks were unchanged since a non-rotating
                                    evaluation are skipped: their outcome is already known) */
  long long pairs_evaluated_lowp;/* of pairs_evaluated: those of the FP32 sweeps */
} jac_info;

/* Fills *opts with the defaults: w = 32, round-robin, full block, sign-pivoted Cholesky,
 * FP64, max_sweeps = 50, want_v = 1, tol = n*2^-53 (tol <= 0), FP64 products JAC_F64_SPLIT16,
 * fused FP32 steps on. */
void jacobi_default_opts(jac_opts* opts);

/* Short text for a return code. */
const char* jacobi_status_string(int status);

/* Library version, major*10000 + minor*100 + patch.  The minor number changes with the layout of
 * jac_opts / jac_info (0.3: jac_opts.f64_products; 0.4: jac_info.pivots_rotated_lowp;
 * 0.5: jac_opts.fused_step). */
#define JAC_VERSION 500
int jacobi_version(void);

/*
 * jacobi_hsvd -- hyperbolic (or, for J = I, trigonometric) one-sided block Jacobi on G.
 * Sec. 3.2, Algorithm 3.4 (full block; Cholesky per opts->factor, Algorithm 3.3).
 *
 *  1 m, 2 n        G is m x n, m >= n >= 1 (full column rank required when J != I).
 *  3 dtype         JAC_R64 or JAC_C128 (G, U, V interleaved (re, im) doubles, leading
 *                  dimensions in complex elements; n <= 10000).  A complex problem is solved
 *                  as the real one of twice the order, G_r = [X -Y; Y X] for G = X + iY and
 *                  J_r = diag(J, J), whose spectrum is that of H twice; the complex results are
 *                  read off every other column (JAC_EINTERNAL if the two copies of an eigenvalue
 *                  differ by more than 1e-6 relative).  opts->tol bounds the complex scaled
 *                  off-diagonal entries: the real sweep rotates above tol / sqrt(2), as the real
 *                  and imaginary parts of a complex entry are two real Gram entries.
 *  4 G, 5 ldg      device, in/out.  On return G = G_in V: the unnormalized U Sigma, columns in
 *                  output order.
 *  6 J             device int8[n], entries +1 / -1, any order (sorted internally to
 *                  diag(I, -I) as Sec. 3 assumes; the output order undoes it).
 *  7 opts          host; NULL selects jacobi_default_opts.
 *  8 lambda        device double[n]: lambda_k = j_k ||g_k||^2, ascending.
 *  9 U, 10 ldu     device m x n or NULL: normalized columns g_k/||g_k|| (must not alias G).
 * 11 V, 12 ldv     device n x n or NULL (required iff opts->want_v): the J-unitary
 *                  V with G_out = G_in V, V^* J V = J_out (J_out: signs in output order).
 * 13 info          host, may be NULL.
 * 14 stream        CUDA stream.
 */
int jacobi_hsvd(int m, int n, int dtype, void* G, int ldg, const int8_t* J, const jac_opts* opts,
                double* lambda, void* U, int ldu, void* V, int ldv, jac_info* info,
                jac_stream_t stream);

/*
 * jacobi_eig_pd -- positive definite H = G G^*: jacobi_hsvd with J = I, so only trigonometric
 * rotations (Eq. (2.1)) are used.  Arguments as jacobi_hsvd without J (positions shift by one:
 * 1 m, 2 n, 3 dtype, 4 G, 5 ldg, 6 opts, 7 lambda, 8 U, 9 ldu, 10 V, 11 ldv, 12 info,
 * 13 stream).
 */
int jacobi_eig_pd(int m, int n, int dtype, void* G, int ldg, const jac_opts* opts, double* lambda,
                  void* U, int ldu, void* V, int ldv, jac_info* info, jac_stream_t stream);

/*
 * jacobi_eig_batched -- many independent problems of uneven order in one call: the same sweep
 * (Algorithm 3.4, Sec. 3.2) of every problem runs in the same kernel launches, each problem taking
 * its pivot pairs from the grid, and a problem leaves the launches when one of its sweeps rotates
 * nothing.  Problem b is jacobi_hsvd(m[b], n[b], dtype, G[b], ldg[b], J[b], opts, lambda[b],
 * U[b], ldu[b], V[b], ldv[b], &info[b]) except that opts->block_w is ignored: the block width
 * is chosen per size class (one pivot block of the whole problem for n <= 64, blocks of 32
 * columns above).  Batches above 32768 problems run as consecutive chunks of that size.
 *  1 batch         >= 0 problems (0: nothing is done).
 *  2 m, 3 n        host int[batch]; 1 <= n[b] <= m[b], n[b] <= 20000.
 *  4 dtype         JAC_R64.
 *  5 G, 6 ldg      host arrays of device pointers / leading dimensions, as jacobi_hsvd.
 *  7 J             host array of device int8 pointers; NULL (the array) means J = I for every
 *                  problem, a NULL entry J = I for that problem.  Entries other than +-1 fail
 *                  that problem with info[b].status = -7.
 *  8 opts          host, as jacobi_hsvd; ordering JAC_ORDER_CYCLE_WEIGHT and precision
 *                  JAC_PREC_FP32 are rejected (-8); JAC_PREC_FP32_ONLY is the FP32 variant.
 *  9 lambda        host array of device double pointers, lambda[b] of n[b] entries.
 * 10 U, 11 ldu     host arrays or NULL; a NULL entry skips U for that problem; U[b] != G[b].
 * 12 V, 13 ldv     host arrays, required iff opts->want_v.
 * 14 info          host jac_info[batch] or NULL: per problem sweeps, converged, status,
 *                  rotations, steps_per_sweep; info[0].launches counts the launches of the call.
 * 15 stream        CUDA stream.
 * Returns a negative argument position, a call-wide error (JAC_ECUDA, JAC_ENOMEM), or else the
 * first non-zero per-problem status in input order (0 when every problem converged).  Failing
 * problems do not stop the others; a problem that fails validation or a pivot leaves its G and
 * outputs unwritten.  Blocks the host until the batch is done.
 */
int jacobi_eig_batched(int batch, const int* m, const int* n, int dtype, void* const* G,
                       const int* ldg, const int8_t* const* J, const jac_opts* opts,
                       double* const* lambda, void* const* U, const int* ldu, void* const* V,
                       const int* ldv, jac_info* info, jac_stream_t stream);

/*
 * jacobi_eig_backward -- adjoint of the eigendecomposition returned by jacobi_hsvd /
 * jacobi_eig_pd / jacobi_eig_batched for square problems (m = n).  The paper computes the
 * forward map only; this is the standard adjoint of the symmetric eigendecomposition
 * H = G J G^T = U diag(lambda) U^T (U orthonormal, Sec. 3.2: u_k = g_k/||g_k||):
 *     H_bar = U sym(diag(lambda_bar) + F o (U^T U_bar)) U^T,  sym(X) = (X + X^T)/2,
 *     F_ij = 1/(lambda_j - lambda_i) for i != j, F_ii = 0, and F_ij = 0 where
 *     |lambda_i - lambda_j| <= deg_tol max_k |lambda_k| (exact only for losses invariant inside
 *     a degenerate eigenspace);
 * and, through the factor, G_bar = (H_bar + H_bar^T) G J = 2 H_bar G J.
 * A batch of problems of one order n at fixed element strides; all arrays device, column-major.
 * The n x n products are FP64-accurate sums of exact FP16 digit products (each term exact to
 * ~2^-53 of its own row and column scale).
 *  1 batch          0 <= batch <= 65535
 *  2 n              order, 1 <= n <= 20000
 *  3 lambda, 4 s_lam            eigenvalues (as returned, ascending), problem b at lambda + b s_lam
 *  5 U, 6 ldu, 7 s_u            orthonormal eigenvectors, n x n
 *  8 lambda_bar, 9 s_lbar       dL/dlambda, or NULL (zero)
 * 10 U_bar, 11 ldub, 12 s_ubar  dL/dU, or NULL (zero)
 * 13 deg_tol        >= 0 (1e-12 is a sensible default)
 * 14 H_bar, 15 ldh, 16 s_h      output dL/dH, n x n, exactly symmetric
 * 17 G, 18 ldg, 19 s_g          the input factor (G_in, not the overwritten one), or NULL
 * 20 J, 21 s_j                  int8 signs of G's columns, or NULL (J = I)
 * 22 G_bar, 23 ldgb, 24 s_gb    output dL/dG, or NULL (then G may be NULL)
 * 25 stream
 * Returns 0, a negative argument position, JAC_ENOMEM or JAC_ECUDA.  Asynchronous on stream
 * (its n x n x batch scratch comes from cudaMallocAsync on that stream).
 */
int jacobi_eig_backward(int batch, int n, const double* lambda, long long s_lam, const double* U,
                        int ldu, long long s_u, const double* lambda_bar, long long s_lbar,
                        const double* U_bar, int ldub, long long s_ubar, double deg_tol,
                        double* H_bar, int ldh, long long s_h, const double* G, int ldg,
                        long long s_g, const int8_t* J, long long s_j, double* G_bar, int ldgb,
                        long long s_gb, jac_stream_t stream);

/*
 * jacobi_autotune_batched -- measures, on the current device, which block width makes
 * jacobi_eig_batched fastest for each size class of orders 8..128 (no counterpart in the paper;
 * Sec. 3 leaves the block width free).  It solves one synthetic batch of `count` problems drawn
 * like the batched workload (orders spread evenly over 8..128, so that every class shares the
 * launches as in a real batch; Gaussian entries; round(0.3 n) signs -1 at random positions) and
 * goes through the classes (8-16, 17-32, 33-48, 49-64, 65-96, 97-128) in turn: a candidate rule
 * replaces a class's current rule only when the whole batch, timed as the best of two runs, is
 * at least 3% faster with it.  The candidates are one pivot block for the whole problem (rule 0,
 * n <= 64; the default up to 64) and fixed widths 8, 16 or 32 (32: the default above 64).
 * jacobi_eig_batched uses the chosen rules on this device from then on.
 *  1 count       problems of the tuning batch, 1..4096; 0 restores the default widths on this device
 *  2 precision   JAC_PREC_FP64 or JAC_PREC_FP32_ONLY (the arithmetic to tune for)
 *  3 rules       host int[129] or NULL: the rule chosen for each order n (-1 outside 8..128)
 *  4 stream
 * Returns 0, a negative argument position, JAC_ENOMEM or JAC_ECUDA (the defaults then stay).
 * Blocks the host; allocates its inputs with cudaMallocAsync.
 */
int jacobi_autotune_batched(int count, int precision, int* rules, jac_stream_t stream);

/*
 * jacobi_sched_pairs -- the device scheduler on its own (Sec. 2.4), for inspection and tests.
 * Writes the block pairs of every step of one cycle for nb blocks (nb even, 2 <= nb <= 4096;
 * nb <= JAC_CYCLE_WEIGHT_MAX_NB for the weight ordering, else -1).
 *  1 nb
 *  2 ordering      enum jac_ordering
 *  3 weights       device double[nb*nb] (row p, column q, q > p used) for
 *                  JAC_ORDER_CYCLE_WEIGHT, else ignored (may be NULL).  Pairs are ranked by
 *                  descending weight, ties (and equal weights) in enumeration order (p, then
 *                  q); a NaN weight ranks after every other value, so any weights give a
 *                  schedule that covers every pair exactly once.
 *  4 pairs         device int[max_steps * (nb/2) * 2]: pairs[(s*(nb/2) + slot)*2 + {0,1}],
 *                  p < q; unused slots are set to -1
 *  5 counts        device int[max_steps]: pairs in step s
 *  6 max_steps     capacity of pairs/counts in steps (nb for the modulus orderings, nb-1 for
 *                  round-robin, nb*(nb-1)/2 always suffices for the weight ordering)
 *  7 nsteps        host int*: number of steps written
 *  8 stream
 */
int jacobi_sched_pairs(int nb, int ordering, const double* weights, int* pairs, int* counts,
                       int max_steps, int* nsteps, jac_stream_t stream);

/* Largest block count accepted by jacobi_sched_pairs_noalloc. */
#define JAC_NOALLOC_MAX_NB 256

/*
 * jacobi_sched_pairs_noalloc -- jacobi_sched_pairs for callers that cannot allocate device
 * memory (no counterpart in the paper).  Same arguments, outputs and return codes as
 * jacobi_sched_pairs, but it calls no cudaMalloc / cudaMallocAsync / cudaFree and no allocating
 * library routine: the scratch of the per-cycle weight ordering (the ranked pair list and the
 * step count) is a fixed array of about 128 KiB inside the library, which every device that
 * loads the library holds until the process exits.  Meant for callers whose device memory is
 * owned by an external pool, that run under a fixed memory budget, or that must not take the
 * allocator's locks or its implicit synchronization.
 *  - nb above JAC_NOALLOC_MAX_NB (256) is rejected with -1 before any work is queued.
 *  - The first call on a device resolves the array's device address (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents (the step count is
 *    cleared at the start of every call): calls that overlap on the GPU, on different streams
 *    or from different host threads, race on it and must be serialized by the caller.
 */
int jacobi_sched_pairs_noalloc(int nb, int ordering, const double* weights, int* pairs, int* counts,
                               int max_steps, int* nsteps, jac_stream_t stream);

/* Kernels that the timing hooks below can bracket: the Gram and update of the FP64(-accurate)
 * sweeps, the pivot kernel (FP32 and FP64 pivots of a step together), the Gram and update of the
 * FP32 sweeps (tensor cores), and the fused FP32 step: Gram, pivot and update of a pair in one
 * CTA, used in the FP32 sweeps when every problem of the launch has at most 96 rows of G (rows
 * padded to 16; pivot blocks of k <= 32 columns) or 192 (k <= 64); the FP64 pivot of a block it
 * hands over is counted with it. */
enum jac_kernel {
  JAC_KERNEL_GRAM = 0,
  JAC_KERNEL_PIVOT = 1,
  JAC_KERNEL_UPDATE = 2,
  JAC_KERNEL_GRAM_LOWP = 3,
  JAC_KERNEL_UPDATE_LOWP = 4,
  JAC_KERNEL_STEP_FUSED = 5,
  JAC_KERNEL_COUNT = 6
};

/*
 * Kernel timing for measurement tools (no counterpart in the paper).  jacobi_profile_begin(mask)
 * resets the totals and, until jacobi_profile_end(), brackets every launch of each kernel whose
 * bit (1 << jac_kernel) is set in mask with a pair of CUDA events on the solve's stream; the
 * elapsed times are added up when each solve finishes.  jacobi_profile_read returns the total
 * milliseconds and the number of launches of one kernel.  Host-only state, one process-wide
 * profile; returns 0 or -k for a bad argument k.
 */
int jacobi_profile_begin(int mask);
int jacobi_profile_read(int kernel, double* total_ms, long long* launches);
int jacobi_profile_end(void);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI_GB300_H */
