// complex.cu -- complex Hermitian problems (dtype JAC_C128) through the real path.
//
// For G = X + iY (m x n) the real factor
//     G_r = [ X  -Y ]        (2m x 2n),   J_r = diag(J, J),
//           [ Y   X ]
// has H_r = G_r J_r G_r^T = [Re H  -Im H; Im H  Re H], whose eigenvalues are those of
// H = G J G^* (Sec. 1), each twice, and whose eigenvector pairs are [x; y] and [-y; x] for an
// eigenvector x + iy of H.  The one-sided sweep on G_r therefore ends with pairs of equal column
// norms, and any column [x; y] of a pair gives the complex column x + iy of G_out = G_in V:
//     G_r [a; b] = [X a - Y b; Y a + X b] = realified G (a + ib).
// These kernels build G_r, J_r and map the real result back: column 2i of the ascending real
// result is the complex column i (the two copies of an eigenvalue are adjacent).
//
// The real sweep does not keep the pair structure exactly: at convergence the two columns of a
// pair span the complex line of an eigenvector only to within tol / (relative gap), so the
// columns x + iy read off are mutually orthogonal in their real parts to tol but in their
// imaginary parts only to that eigenspace accuracy.  The complex path therefore rebuilds the
// exact pair structure from column 2i of every pair (k_restructure) and sweeps once more in
// FP64: the second pass starts with off-diagonals of that size and converges quadratically.
// It ends only on a sweep that rotates nothing: the complex columns read off after a rotating
// sweep would carry that sweep's structure error.
#include "jacobi_common.cuh"

namespace jac {

// G_r[:, c] = [Re g_c; Im g_c], G_r[:, n + c] = [-Im g_c; Re g_c]; J_r = (J, J) (J NULL: +1).
// Grid-stride over m n.
__global__ void k_realify(int m, int n, const double2* __restrict__ G, int ldg, const int8_t* __restrict__ J,
                          double* __restrict__ Gr, int8_t* __restrict__ Jr) {
  const size_t total = (size_t)m * n, ld = 2 * (size_t)m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    const double2 z = G[(size_t)c * ldg + r];
    Gr[c * ld + r] = z.x;
    Gr[c * ld + m + r] = z.y;
    Gr[(n + c) * ld + r] = -z.y;
    Gr[(n + c) * ld + m + r] = z.x;
    if (r == 0) {
      const int8_t j = J ? J[c] : (int8_t)1;
      Jr[c] = j;
      Jr[n + c] = j;
    }
  }
}

// Output column i from real column 2i: G[:, i] = x + iy, U[:, i] = G[:, i] / sqrt|lambda_i|,
// V[:, i] = a + ib, lambda_i = lambda_r[2i].  Flags *bad when the two copies of an eigenvalue
// differ by more than 1e-6 relative (pairing not resolved).  Grid (blocks, n), 128 threads.
__global__ void k_complexify(int m, int n, const double* __restrict__ Gr, const double* __restrict__ lam_r,
                             const double* __restrict__ Vr, double2* __restrict__ G, int ldg,
                             double* __restrict__ lambda, double2* __restrict__ U, int ldu, double2* __restrict__ V,
                             int ldv, unsigned* __restrict__ bad) {
  const int i = blockIdx.y, src = 2 * i;
  const double l0 = lam_r[src], l1 = lam_r[src + 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    lambda[i] = l0;
    if (!(fabs(l0 - l1) <= 1e-6 * fmax(fabs(l0), fabs(l1)))) atomicOr(bad, 1u);
  }
  const double inv = (l0 != 0.0) ? 1.0 / sqrt(fabs(l0)) : 0.0;
  const size_t ld = 2 * (size_t)m;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const double x = Gr[src * ld + r], y = Gr[src * ld + m + r];
    G[(size_t)i * ldg + r] = make_double2(x, y);
    if (U) U[(size_t)i * ldu + r] = make_double2(x * inv, y * inv);
  }
  if (V) {
    const size_t lv = 2 * (size_t)n;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
      V[(size_t)i * ldv + r] = make_double2(Vr[src * lv + r], Vr[src * lv + n + r]);
  }
}

// Rebuild exact pairs from the first column of each pair of an ascending real result:
// out[:, i] = in[:, 2i] = [x; y], out[:, n + i] = [-y; x] (rows 2h: x in rows 0..h-1); with lam,
// also the signs of the rebuilt columns, Jout[i] = Jout[n + i] = sign(lam[2i]) (lambda = j ||g||^2).
// Grid-stride over h n.
__global__ void k_restructure(int h, int n, const double* __restrict__ in, double* __restrict__ out,
                              const double* __restrict__ lam, int8_t* __restrict__ Jout) {
  const size_t total = (size_t)h * n, ld = 2 * (size_t)h;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % h), i = (int)(e / h);
    const double x = in[(size_t)(2 * i) * ld + r], y = in[(size_t)(2 * i) * ld + h + r];
    out[(size_t)i * ld + r] = x;
    out[(size_t)i * ld + h + r] = y;
    out[(size_t)(n + i) * ld + r] = -y;
    out[(size_t)(n + i) * ld + h + r] = x;
    if (lam && r == 0) {
      const int8_t j = (lam[2 * i] < 0.0) ? (int8_t)-1 : (int8_t)1;
      Jout[i] = j;
      Jout[n + i] = j;
    }
  }
}

}  // namespace jac
