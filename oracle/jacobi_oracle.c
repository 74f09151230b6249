/*
 * jacobi_oracle.c -- CPU oracle for the one-sided trigonometric / hyperbolic Jacobi method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its Python
 * binding) may link, load or call this file.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Singer et al., "Novel Modifications of Parallel Jacobi Algorithms"):
 *
 *   Given G (m x n, column-major, real or complex) and a signature J = diag(j_k), j_k = +-1,
 *   the pointwise one-sided Jacobi method of Sec. 2.1 right-multiplies G by 2x2 rotations
 *   until the columns of G are mutually orthogonal.  For a pivot pair (i, j) it forms
 *   A_P = [g_i g_j]^* [g_i g_j] (Sec. 2.1, hyperbolic step 1; for J = I this is the
 *   trigonometric algorithm applied to the factor), and
 *     - if j_i == j_j: a trigonometric rotation, Eq. (2.1),
 *     - else:          a hyperbolic rotation (cosh / sinh, Sec. 2.1),
 *   chosen so that Q_P^* A_P Q_P is diagonal, then [g_i g_j] <- [g_i g_j] Q_P (step 3).
 *   The transforms are accumulated in V (V^* J V = J).  At convergence the eigenvalues of
 *   H = G J G^* are lambda_k = j_k ||g_k||^2 and the eigenvectors are g_k / ||g_k||
 *   (Sec. 1, the hyperbolic SVD G = U Sigma V^{-1}; Sec. 3.2, "normalizing the columns").
 *
 *   The pivot order is the row-cyclic one, (0,1),(0,2),...,(0,n-1),(1,2),...: the inner
 *   strategy for which the paper's convergence argument holds (Sec. 2.4).
 *
 * Readings where the paper is silent:
 *   - Rotation formulas.  The paper cites them but does not print them.  Writing
 *     b = a_ij = g_i^* g_j = |b| e^{i alpha}:
 *       trig:  zeta = (a_jj - a_ii) / (2|b|),  t = tan(phi) = sign(zeta)/(|zeta| + sqrt(1+zeta^2)),
 *              c = 1/sqrt(1+t^2), s = t c,
 *              g_i' = c g_i - e^{-i alpha} s g_j,   g_j' = e^{i alpha} s g_i + c g_j.
 *       hyp:   zeta = -(a_ii + a_jj) / (2|b|),  t = tanh(phi) = sign(zeta)/(|zeta| + sqrt(zeta^2-1)),
 *              if |t| >= 1 (possible only in rounding) t = 0.9 sign(t)  (Sec. 3.2),
 *              ch = 1/sqrt(1-t^2), sh = t ch,
 *              g_i' = ch g_i + e^{-i alpha} sh g_j, g_j' = e^{i alpha} sh g_i + ch g_j.
 *     These are Q_P of Eq. (2.1) and of the hyperbolic rotation of Sec. 2.1 with the phase
 *     placement printed there.
 *   - Stopping criterion.  The paper calls it "natural" (Sec. 4).  A pair is rotated iff
 *     |a_ij| > tol * sqrt(a_ii a_jj); the sweep loop stops after a sweep with no rotation.
 *
 * Parity pins (tests/test_oracle_*.py): Example 1 of Sec. 3.1 (eigenvalues -1, 1, 1, 3),
 * closed-form 2x2 eigenvalues, prescribed spectra Q diag(sigma) W, exact characteristic
 * polynomial roots for n <= 6, SVD for J = I, and the invariants V^* J V = J, G0 V = G,
 * G^* G diagonal.  The block orderings (modulus, modified modulus, round-robin, per-cycle
 * weight) are pinned by exhaustive enumeration.  The eigendecomposition adjoint
 * (oracle_eig_backward, no counterpart in the paper) is pinned by the Hellmann-Feynman
 * eigenvalue derivatives, the closed form on diagonal H and central finite differences of a
 * loss on eigenvalues and eigenvectors with LAPACK as the forward map.  The three
 * wide-precision checks (oracle_check_*) are pinned by hand-worked closed forms with nonzero
 * answers and by exact rational evaluations of their definitions on integer and
 * Gaussian-integer matrices (tests/test_oracle_checkers.py).
 *
 * Precision: IEEE double throughout the method; the check routines accumulate in long double
 * (80-bit on x86-64, binary128 on aarch64).  Compile with -ffp-contract=off so that results
 * do not depend on FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_NOTCONV 1
#define ORACLE_EINVAL (-1)

/* A planted mistake, for the mutation tests that show the pins can fail.  0 = none.
 * 1: trig rotation applied with the wrong sign of s.
 * 2: hyperbolic pairs rotated with the trigonometric formula.
 * 3: complex phase not conjugated in g_i'.
 * 4: eigenvalue sign j_k dropped.
 * 5: V accumulation skipped on the second column of each pair.
 * 6: adjoint formed with (U_bar^T U) in place of (U^T U_bar).
 * 7: off-norm check counts each off-diagonal pair once (the factor 2 of a_ij, a_ji dropped).
 * 8: off-norm check drops the imaginary part of a complex g_i^* g_j.
 * 9: J-unitarity check signs the rows of V with J_col instead of J_row.
 * 10: J-unitarity check leaves out the off-diagonal entries of V^* J V - J.
 * 11: factor residual check multiplies by V^T instead of V.
 * 12: factor residual check normalizes by ||G||_F instead of ||G0||_F.                    */
static int g_mutation = 0;
void oracle_set_mutation(int k) { g_mutation = k; }
int oracle_get_mutation(void) { return g_mutation; }

/* ---------------------------------------------------------------- rotations (2x2) */

/* Parameters of the rotation that diagonalizes [[a, b],[conj(b), d]] with |b| = beta > 0.
 * hyperbolic = 0: returns c, s of Eq. (2.1).  hyperbolic = 1: returns ch, sh.
 * t_out receives tan(phi) or tanh(phi).                                                   */
void oracle_rotation_params(double a, double d, double beta, int hyperbolic,
                            double* cs_out, double* sn_out, double* t_out) {
  double t;
  if (!hyperbolic) {
    double zeta = (d - a) / (2.0 * beta);
    double az = fabs(zeta);
    double sg = (zeta < 0.0) ? -1.0 : 1.0; /* sign(0) = +1 */
    if (az > 1.0e150)
      t = 1.0 / (2.0 * zeta); /* zeta^2 would overflow; t = 1/(2 zeta) to first order */
    else
      t = sg / (az + sqrt(1.0 + zeta * zeta));
    double c = 1.0 / sqrt(1.0 + t * t);
    *cs_out = c;
    *sn_out = t * c;
  } else {
    double zeta = -(a + d) / (2.0 * beta);
    double az = fabs(zeta);
    double sg = (zeta < 0.0) ? -1.0 : 1.0;
    if (az > 1.0e150)
      t = 1.0 / (2.0 * zeta);
    else
      t = sg / (az + sqrt(zeta * zeta - 1.0));
    if (!(fabs(t) < 1.0) || !(1.0 - t * t > 0.0)) t = (t < 0.0 ? -0.9 : 0.9); /* Sec. 3.2 guard */
    double ch = 1.0 / sqrt(1.0 - t * t);
    *cs_out = ch;
    *sn_out = t * ch;
  }
  if (t_out) *t_out = t;
}

/* ---------------------------------------------------------------- pointwise sweep */

static double dot_re(int m, const double* x, const double* y) {
  double s = 0.0;
  for (int r = 0; r < m; ++r) s += x[r] * y[r];
  return s;
}

/* complex vectors are stored interleaved (re, im); returns x^* y in (*re, *im) */
static void dot_cx(int m, const double* x, const double* y, double* re, double* im) {
  double sr = 0.0, si = 0.0;
  for (int r = 0; r < m; ++r) {
    double xr = x[2 * r], xi = x[2 * r + 1], yr = y[2 * r], yi = y[2 * r + 1];
    sr += xr * yr + xi * yi;
    si += xr * yi - xi * yr;
  }
  *re = sr;
  *im = si;
}

/* Apply [x y] <- [x y] Q with Q = [[q11, q12],[q21, q22]] where, writing e = er + i ei,
 *   trig: q11 = c, q12 = e s, q21 = -conj(e) s, q22 = c
 *   hyp:  q11 = ch, q12 = e sh, q21 = conj(e) sh, q22 = ch                               */
static void rotate_re(int m, double* x, double* y, double cs, double sn, double e, int hyperbolic,
                      int skip_second) {
  for (int r = 0; r < m; ++r) {
    double xv = x[r], yv = y[r];
    double nx, ny;
    if (!hyperbolic) {
      double s_eff = (g_mutation == 1) ? -sn : sn;
      nx = cs * xv - e * s_eff * yv;
      ny = e * s_eff * xv + cs * yv;
    } else {
      nx = cs * xv + e * sn * yv;
      ny = e * sn * xv + cs * yv;
    }
    x[r] = nx;
    if (!skip_second) y[r] = ny;
  }
}

static void rotate_cx(int m, double* x, double* y, double cs, double sn, double er, double ei,
                      int hyperbolic, int skip_second) {
  /* conj(e) = er - i ei */
  double cer = er, cei = (g_mutation == 3) ? ei : -ei;
  for (int r = 0; r < m; ++r) {
    double xr = x[2 * r], xi = x[2 * r + 1], yr = y[2 * r], yi = y[2 * r + 1];
    /* conj(e) * y and e * x */
    double cyr = cer * yr - cei * yi, cyi = cer * yi + cei * yr;
    double exr = er * xr - ei * xi, exi = er * xi + ei * xr;
    double nxr, nxi, nyr, nyi;
    if (!hyperbolic) {
      double s_eff = (g_mutation == 1) ? -sn : sn;
      nxr = cs * xr - s_eff * cyr;
      nxi = cs * xi - s_eff * cyi;
      nyr = s_eff * exr + cs * yr;
      nyi = s_eff * exi + cs * yi;
    } else {
      nxr = cs * xr + sn * cyr;
      nxi = cs * xi + sn * cyi;
      nyr = sn * exr + cs * yr;
      nyi = sn * exi + cs * yi;
    }
    x[2 * r] = nxr;
    x[2 * r + 1] = nxi;
    if (!skip_second) {
      y[2 * r] = nyr;
      y[2 * r + 1] = nyi;
    }
  }
}

/*
 * Sequential row-cyclic one-sided Jacobi (Sec. 2.1) on G (m x n, column-major, ld = ldg).
 * cplx = 1: complex, interleaved (re, im) doubles, ldg counted in complex elements.
 * J: n signs (+1 / -1).  V (n x n, ld = ldv), may be NULL; when given it is set to I first.
 * Returns ORACLE_OK on convergence, ORACLE_NOTCONV after max_sweeps sweeps with rotations.
 */
int oracle_hsvd(int m, int n, int cplx, double* G, int ldg, const int8_t* J, double tol,
                int max_sweeps, double* V, int ldv, int* sweeps_out, long long* rotations_out) {
  if (m < 0 || n < 0 || ldg < (m > 1 ? m : 1) || (V && ldv < (n > 1 ? n : 1))) return ORACLE_EINVAL;
  const int es = cplx ? 2 : 1; /* doubles per element */
  if (V) {
    for (int c = 0; c < n; ++c)
      for (int r = 0; r < n; ++r) {
        V[((size_t)c * ldv + r) * es] = (r == c) ? 1.0 : 0.0;
        if (cplx) V[((size_t)c * ldv + r) * es + 1] = 0.0;
      }
  }
  long long total = 0;
  int sweep = 0, status = ORACLE_NOTCONV;
  if (n < 2) status = ORACLE_OK;
  while (status != ORACLE_OK && sweep < max_sweeps) {
    long long rot = 0;
    for (int i = 0; i < n - 1; ++i) {
      for (int j = i + 1; j < n; ++j) {
        double* gi = G + (size_t)i * ldg * es;
        double* gj = G + (size_t)j * ldg * es;
        double a, d, br, bi = 0.0;
        if (!cplx) {
          a = dot_re(m, gi, gi);
          d = dot_re(m, gj, gj);
          br = dot_re(m, gi, gj);
        } else {
          double tmp;
          dot_cx(m, gi, gi, &a, &tmp);
          dot_cx(m, gj, gj, &d, &tmp);
          dot_cx(m, gi, gj, &br, &bi);
        }
        double beta = cplx ? hypot(br, bi) : fabs(br);
        if (!(beta > tol * sqrt(a * d))) continue;
        int hyp = (J[i] != J[j]);
        if (g_mutation == 2) hyp = 0;
        double cs, sn;
        oracle_rotation_params(a, d, beta, hyp, &cs, &sn, NULL);
        if (!cplx) {
          double e = (br < 0.0) ? -1.0 : 1.0;
          rotate_re(m, gi, gj, cs, sn, e, hyp, 0);
          if (V)
            rotate_re(n, V + (size_t)i * ldv, V + (size_t)j * ldv, cs, sn, e, hyp, g_mutation == 5);
        } else {
          double er = br / beta, ei = bi / beta;
          rotate_cx(m, gi, gj, cs, sn, er, ei, hyp, 0);
          if (V)
            rotate_cx(n, V + (size_t)i * ldv * 2, V + (size_t)j * ldv * 2, cs, sn, er, ei, hyp,
                      g_mutation == 5);
        }
        ++rot;
      }
    }
    ++sweep;
    total += rot;
    if (rot == 0) status = ORACLE_OK;
  }
  if (sweeps_out) *sweeps_out = sweep;
  if (rotations_out) *rotations_out = total;
  return status;
}

/*
 * Eigenpairs from the converged factor (Sec. 1 and Sec. 3.2): lambda_k = j_k ||g_k||^2,
 * u_k = g_k / ||g_k||, returned in ascending lambda order (ties: lower column index first).
 * perm[k] = original column of the k-th output.  U (m x n, ld = ldu) may be NULL.
 */
void oracle_eigenpairs(int m, int n, int cplx, const double* G, int ldg, const int8_t* J,
                       double* lambda, double* U, int ldu, int* perm) {
  const int es = cplx ? 2 : 1;
  double* nrm2 = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* lam = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  int* idx = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) {
    const double* g = G + (size_t)k * ldg * es;
    double s = 0.0;
    for (int r = 0; r < m * es; ++r) s += g[r] * g[r];
    nrm2[k] = s;
    lam[k] = (g_mutation == 4) ? s : (J[k] < 0 ? -s : s);
    idx[k] = k;
  }
  /* stable insertion sort by lambda (n is small enough for the tests that use it; the
     bench sample calls it once) */
  for (int a = 1; a < n; ++a) {
    int v = idx[a];
    int b = a - 1;
    while (b >= 0 && lam[idx[b]] > lam[v]) {
      idx[b + 1] = idx[b];
      --b;
    }
    idx[b + 1] = v;
  }
  for (int k = 0; k < n; ++k) {
    int src = idx[k];
    lambda[k] = lam[src];
    if (perm) perm[k] = src;
    if (U) {
      double inv = (nrm2[src] > 0.0) ? 1.0 / sqrt(nrm2[src]) : 0.0;
      const double* g = G + (size_t)src * ldg * es;
      double* u = U + (size_t)k * ldu * es;
      for (int r = 0; r < m * es; ++r) u[r] = g[r] * inv;
    }
  }
  free(nrm2);
  free(lam);
  free(idx);
}

/* ---------------------------------------------------------------- block orderings */

/*
 * Modulus strategy (Sec. 2.4, Fig. 2-3): in step k (0 <= k < nb) the block pairs are the
 * {p < q} with p + q = k (mod nb), i.e. the k-th block antidiagonal taken modulo nb.  For
 * even nb and even k the two indices with 2p = k (mod nb) are left unpaired; the modified
 * modulus strategy (modified = 1) pairs those two as well.  Pairs are written as (p, q),
 * p < q, in increasing p.  Returns the number of pairs.
 */
int oracle_pairs_modulus(int nb, int k, int modified, int* pairs) {
  int np = 0;
  for (int p = 0; p < nb; ++p) {
    int q = ((k - p) % nb + nb) % nb;
    if (p < q) {
      pairs[2 * np] = p;
      pairs[2 * np + 1] = q;
      ++np;
    }
  }
  if (modified) {
    int fix[2], nf = 0;
    for (int p = 0; p < nb; ++p)
      if (((2 * p - k) % nb + nb) % nb == 0) fix[nf++] = p;
    if (nf == 2) {
      /* insert keeping increasing p */
      int p = fix[0], q = fix[1], pos = np;
      while (pos > 0 && pairs[2 * (pos - 1)] > p) {
        pairs[2 * pos] = pairs[2 * (pos - 1)];
        pairs[2 * pos + 1] = pairs[2 * (pos - 1) + 1];
        --pos;
      }
      pairs[2 * pos] = p;
      pairs[2 * pos + 1] = q;
      ++np;
    }
  }
  return np;
}

/*
 * Round-robin (circle) ordering for even nb: nb - 1 steps, each a perfect matching.  Index
 * nb - 1 is fixed; in step s it meets s, and (s + r) mod (nb-1) meets (s - r) mod (nb-1) for
 * r = 1 .. nb/2 - 1.  Pairs are written as (min, max) sorted by the first index.
 */
int oracle_pairs_round_robin(int nb, int s, int* pairs) {
  int np = 0, L = nb - 1;
  int tmp[2 * 4096];
  if (nb < 2 || nb > 4096) return 0;
  tmp[0] = s < nb - 1 ? s : nb - 1;
  tmp[1] = nb - 1;
  np = 1;
  for (int r = 1; r < nb / 2; ++r) {
    int a = ((s + r) % L + L) % L, b = ((s - r) % L + L) % L;
    tmp[2 * np] = a < b ? a : b;
    tmp[2 * np + 1] = a < b ? b : a;
    ++np;
  }
  /* sort by first index */
  for (int x = 1; x < np; ++x) {
    int p = tmp[2 * x], q = tmp[2 * x + 1], y = x - 1;
    while (y >= 0 && tmp[2 * y] > p) {
      tmp[2 * (y + 1)] = tmp[2 * y];
      tmp[2 * (y + 1) + 1] = tmp[2 * y + 1];
      --y;
    }
    tmp[2 * (y + 1)] = p;
    tmp[2 * (y + 1) + 1] = q;
  }
  memcpy(pairs, tmp, sizeof(int) * 2 * np);
  return np;
}

/*
 * Per-cycle largest-weight ordering (a build extension of the paper's per-cycle pivoting,
 * Sec. 3.2 / Sec. 4): given the weights w[p*nb + q] (p < q) of all block pairs for this
 * cycle, sort the pairs by descending weight (ties: smaller p, then smaller q), then fill
 * steps greedily: each step scans the not-yet-scheduled pairs in that order and takes every
 * pair disjoint from those already taken in the step.  Every pair is scheduled exactly once
 * per cycle.  Writes pairs[step][slot][2] with slot stride nb/2, counts[step]; returns the
 * number of steps.
 */
int oracle_pairs_cycle_weight(int nb, const double* w, int* pairs, int* counts) {
  int npairs = nb * (nb - 1) / 2;
  int* order = (int*)malloc(sizeof(int) * 2 * (npairs > 0 ? npairs : 1));
  double* wt = (double*)malloc(sizeof(double) * (npairs > 0 ? npairs : 1));
  char* done = (char*)calloc(npairs > 0 ? npairs : 1, 1);
  char* busy = (char*)malloc(nb > 0 ? nb : 1);
  int c = 0;
  for (int p = 0; p < nb; ++p)
    for (int q = p + 1; q < nb; ++q) {
      order[2 * c] = p;
      order[2 * c + 1] = q;
      wt[c] = w[p * nb + q];
      ++c;
    }
  /* stable insertion sort by descending weight; the enumeration order gives the ties */
  for (int x = 1; x < npairs; ++x) {
    int p = order[2 * x], q = order[2 * x + 1];
    double v = wt[x];
    int y = x - 1;
    while (y >= 0 && wt[y] < v) {
      order[2 * (y + 1)] = order[2 * y];
      order[2 * (y + 1) + 1] = order[2 * y + 1];
      wt[y + 1] = wt[y];
      --y;
    }
    order[2 * (y + 1)] = p;
    order[2 * (y + 1) + 1] = q;
    wt[y + 1] = v;
  }
  int half = nb / 2, steps = 0, left = npairs;
  while (left > 0) {
    memset(busy, 0, nb);
    int np = 0;
    for (int x = 0; x < npairs; ++x) {
      if (done[x]) continue;
      int p = order[2 * x], q = order[2 * x + 1];
      if (busy[p] || busy[q]) continue;
      busy[p] = busy[q] = 1;
      done[x] = 1;
      pairs[(steps * half + np) * 2] = p;
      pairs[(steps * half + np) * 2 + 1] = q;
      ++np;
      --left;
    }
    counts[steps] = np;
    ++steps;
  }
  free(order);
  free(wt);
  free(done);
  free(busy);
  return steps;
}

/* Block partition (Sec. 3: widths within a pivot block differ by at most one).  nb blocks
 * over n columns as evenly as possible; the first n mod nb blocks are one wider.
 * Writes off[nb + 1].                                                                      */
void oracle_block_offsets(int n, int nb, int* off) {
  int base = n / nb, rem = n % nb, o = 0;
  for (int b = 0; b < nb; ++b) {
    off[b] = o;
    o += base + (b < rem ? 1 : 0);
  }
  off[nb] = o;
}

/* ---------------------------------------------------------------- wide-precision checks */

typedef long double wide;

/* off_F(G^* G) / ||G||_F^2 and max_{i != j} |a_ij| / sqrt(a_ii a_jj) of the final factor. */
void oracle_check_offdiag(int m, int n, int cplx, const double* G, int ldg, double* off_rel,
                          double* max_scaled) {
  const int es = cplx ? 2 : 1;
  wide* dg = (wide*)malloc(sizeof(wide) * (n > 0 ? n : 1));
  wide tr = 0, off2 = 0, mx = 0;
  for (int i = 0; i < n; ++i) {
    const double* gi = G + (size_t)i * ldg * es;
    wide s = 0;
    for (int r = 0; r < m * es; ++r) s += (wide)gi[r] * gi[r];
    dg[i] = s;
    tr += s;
  }
  for (int i = 0; i < n; ++i) {
    const double* gi = G + (size_t)i * ldg * es;
    for (int j = i + 1; j < n; ++j) {
      const double* gj = G + (size_t)j * ldg * es;
      wide sr = 0, si = 0;
      if (!cplx) {
        for (int r = 0; r < m; ++r) sr += (wide)gi[r] * gj[r];
      } else {
        for (int r = 0; r < m; ++r) {
          wide xr = gi[2 * r], xi = gi[2 * r + 1], yr = gj[2 * r], yi = gj[2 * r + 1];
          sr += xr * yr + xi * yi;
          si += xr * yi - xi * yr;
        }
      }
      if (g_mutation == 8) si = 0;
      wide b2 = sr * sr + si * si;
      off2 += (g_mutation == 7) ? b2 : 2 * b2;
      wide den = dg[i] * dg[j];
      if (den > 0) {
        wide sc = b2 / den;
        if (sc > mx) mx = sc;
      }
    }
  }
  *off_rel = (tr > 0) ? (double)(sqrtl(off2) / tr) : 0.0;
  *max_scaled = (double)sqrtl(mx);
  free(dg);
}

/* || V^* J_row V - J_col ||_F.  J_row signs the rows of V (the input columns of G), J_col the
 * columns (the output order); for V in the input order both are J.                          */
double oracle_check_vjv(int n, int cplx, const double* V, int ldv, const int8_t* J,
                        const int8_t* Jc) {
  const int es = cplx ? 2 : 1;
  wide acc = 0;
  for (int i = 0; i < n; ++i) {
    const double* vi = V + (size_t)i * ldv * es;
    for (int j = i; j < n; ++j) {
      const double* vj = V + (size_t)j * ldv * es;
      wide sr = 0, si = 0;
      for (int r = 0; r < n; ++r) {
        wide jr = (((g_mutation == 9) ? Jc[r] : J[r]) < 0) ? -1.0L : 1.0L;
        if (!cplx) {
          sr += jr * vi[r] * vj[r];
        } else {
          wide xr = vi[2 * r], xi = vi[2 * r + 1], yr = vj[2 * r], yi = vj[2 * r + 1];
          sr += jr * (xr * yr + xi * yi);
          si += jr * (xr * yi - xi * yr);
        }
      }
      if (i == j) sr -= (Jc[i] < 0) ? -1.0L : 1.0L;
      wide e2 = sr * sr + si * si;
      if (g_mutation == 10 && i != j) e2 = 0;
      acc += (i == j) ? e2 : 2 * e2;
    }
  }
  return (double)sqrtl(acc);
}

/* || G0 V - G ||_F / || G0 ||_F   (G0, G: m x n; V: n x n) */
double oracle_check_factor_residual(int m, int n, int cplx, const double* G0, int ldg0,
                                    const double* V, int ldv, const double* G, int ldg) {
  const int es = cplx ? 2 : 1;
  wide num = 0, den = 0;
  for (int c = 0; c < n; ++c) {
    for (int r = 0; r < m; ++r) {
      wide sr = 0, si = 0;
      for (int k = 0; k < n; ++k) {
        const size_t vk = (g_mutation == 11) ? (size_t)k * ldv + c : (size_t)c * ldv + k;
        if (!cplx) {
          sr += (wide)G0[(size_t)k * ldg0 + r] * V[vk];
        } else {
          wide ar = G0[((size_t)k * ldg0 + r) * 2], ai = G0[((size_t)k * ldg0 + r) * 2 + 1];
          wide br = V[vk * 2], bi = V[vk * 2 + 1];
          sr += ar * br - ai * bi;
          si += ar * bi + ai * br;
        }
      }
      if (!cplx) {
        wide d = sr - G[(size_t)c * ldg + r];
        num += d * d;
      } else {
        wide dr = sr - G[((size_t)c * ldg + r) * 2], di = si - G[((size_t)c * ldg + r) * 2 + 1];
        num += dr * dr + di * di;
      }
    }
  }
  for (int c = 0; c < n; ++c)
    for (int r = 0; r < m * es; ++r) {
      wide v = (g_mutation == 12) ? G[(size_t)c * ldg * es + r] : G0[(size_t)c * ldg0 * es + r];
      den += v * v;
    }
  return (den > 0) ? (double)sqrtl(num / den) : 0.0;
}

/*
 * Reference gradient of L(H) for the symmetric eigendecomposition H = U diag(lambda) U^T
 * (real), given lambda_bar (n) and U_bar (n x n):
 *   H_bar = sym( U ( diag(lambda_bar) + F o (U^T U_bar) ) U^T ),  F_ij = 1/(lambda_j - lambda_i)
 * for i != j and |lambda_i - lambda_j| > mask * max|lambda|, else 0; sym(X) = (X + X^T)/2.
 * Standard adjoint of the eigendecomposition; the paper has no backward pass.  Accumulated
 * in long double.  U, Ubar, Hbar: column-major, ld = n.
 */
void oracle_eig_backward(int n, const double* lambda, const double* U, const double* lambda_bar,
                         const double* U_bar, double mask, double* H_bar) {
  wide* X = (wide*)malloc(sizeof(wide) * (size_t)n * n);
  wide* Y = (wide*)malloc(sizeof(wide) * (size_t)n * n);
  double lmax = 0.0;
  for (int i = 0; i < n; ++i)
    if (fabs(lambda[i]) > lmax) lmax = fabs(lambda[i]);
  /* X = diag(lambda_bar) + F o (U^T U_bar) */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      wide v = 0;
      if (i == j) {
        v = lambda_bar ? lambda_bar[i] : 0.0;
      } else if (U_bar) {
        wide gap = (wide)lambda[j] - (wide)lambda[i];
        if (fabsl(gap) > (wide)mask * lmax) {
          wide s = 0;
          for (int r = 0; r < n; ++r)
            s += (g_mutation == 6) ? (wide)U_bar[(size_t)i * n + r] * U[(size_t)j * n + r]
                                   : (wide)U[(size_t)i * n + r] * U_bar[(size_t)j * n + r];
          v = s / gap;
        }
      }
      X[(size_t)j * n + i] = v;
    }
  /* Y = U X */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      wide s = 0;
      for (int k = 0; k < n; ++k) s += (wide)U[(size_t)k * n + i] * X[(size_t)j * n + k];
      Y[(size_t)j * n + i] = s;
    }
  /* Z = Y U^T, H_bar = (Z + Z^T)/2 */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= j; ++i) {
      wide zij = 0, zji = 0;
      for (int k = 0; k < n; ++k) {
        zij += Y[(size_t)k * n + i] * U[(size_t)k * n + j];
        zji += Y[(size_t)k * n + j] * U[(size_t)k * n + i];
      }
      double h = (double)((zij + zji) / 2);
      H_bar[(size_t)j * n + i] = h;
      H_bar[(size_t)i * n + j] = h;
    }
  free(X);
  free(Y);
}
