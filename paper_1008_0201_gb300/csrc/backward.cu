// backward.cu -- adjoint of the eigendecomposition the sweep produces (no counterpart in the
// paper, which computes the forward map only).
//
// The forward result of a square problem is H = G J G^T = U diag(lambda) U^T with orthonormal U
// (u_k = g_k / ||g_k||, lambda_k = j_k ||g_k||^2, Sec. 3.2), so a loss L(lambda, U) pulls back
// through the symmetric eigendecomposition:
//     H_bar = U sym(diag(lambda_bar) + F o (U^T U_bar)) U^T,   sym(X) = (X + X^T) / 2,
//     F_ij = 1 / (lambda_j - lambda_i) (i != j),  F_ii = 0,
// with F_ij set to 0 where |lambda_i - lambda_j| <= deg_tol max_k |lambda_k| (degenerate pairs:
// exact only for losses invariant inside a degenerate eigenspace).  Through the factor,
// H = G J G^T gives G_bar = (H_bar + H_bar^T) G J = 2 H_bar G J (J-adjusted for J != I).
// The n x n products run as FP64-accurate sums of exact FP16 tensor-core digit products
// (k_gemm_oz, ozaki.cu), the elementwise middle step and the column signs in the kernels below.
#include <algorithm>
#include <cstring>

#include "jacobi_common.cuh"
#include "jacobi_gb300.h"

namespace jac {
int oz_gemm_launch(int Mr, int Nc, int K, const double* A, int lda, int transA, const double* B, int ldb,
                   const int8_t* sb, const int8_t* dsub, double* C, int ldc, int sym, int transB, long long sa,
                   long long sbb, long long sc, int batch, cudaStream_t st);

// In place on M = U^T U_bar (n x n, ld n, problem blockIdx.y at stride sM):
//   M_ii <- lambda_bar_i,   M_ij, M_ji <- (M_ij - M_ji) / (2 (lambda_j - lambda_i))  (0 if degenerate)
// which is sym(diag(lambda_bar) + F o M).  Each unordered pair is owned by the thread of (i < j).
// Grid (blocks, batch), 256 threads.
__global__ void k_bwd_mid(int n, double* __restrict__ M, long long sM, const double* __restrict__ lam,
                          long long sl, const double* __restrict__ lbar, long long slb, int have_ubar,
                          double deg_tol) {
  __shared__ double red[8];
  const int b = blockIdx.y;
  M += (size_t)b * sM;
  lam += (size_t)b * sl;
  if (lbar) lbar += (size_t)b * slb;
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(lam[i]));
  mx = warp_max_d(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  const double thr = deg_tol * mx;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) continue;
    if (i == j) {
      M[(size_t)i * n + i] = lbar ? lbar[i] : 0.0;
      continue;
    }
    double v = 0.0;
    if (have_ubar) {
      const double gap = lam[j] - lam[i];
      if (fabs(gap) > thr) v = (M[(size_t)j * n + i] - M[(size_t)i * n + j]) / (2.0 * gap);
    }
    M[(size_t)j * n + i] = v;
    M[(size_t)i * n + j] = v;
  }
}

// X[:, c] *= alpha j_c (j = NULL: +1).  Grid (blocks, batch).
__global__ void k_scale_cols(int m, int n, double* __restrict__ X, int ldx, long long sx,
                             const int8_t* __restrict__ J, long long sj, double alpha) {
  const int b = blockIdx.y;
  X += (size_t)b * sx;
  if (J) J += (size_t)b * sj;
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    const double s = (J && J[c] < 0) ? -alpha : alpha;
    X[(size_t)c * ldx + r] *= s;
  }
}

}  // namespace jac

using namespace jac;

extern "C" int jacobi_eig_backward(int batch, int n, const double* lambda, long long s_lam, const double* U, int ldu,
                                   long long s_u, const double* lambda_bar, long long s_lbar, const double* U_bar,
                                   int ldub, long long s_ubar, double deg_tol, double* H_bar, int ldh, long long s_h,
                                   const double* G, int ldg, long long s_g, const int8_t* J, long long s_j,
                                   double* G_bar, int ldgb, long long s_gb, jac_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (batch < 0 || batch > 65535) return -1;
  if (n < 1 || n > 20000) return -2;
  if (!lambda) return -3;
  if (s_lam < n && batch > 1) return -4;
  if (!U) return -5;
  if (ldu < n) return -6;
  if (s_u < (long long)ldu * n && batch > 1) return -7;
  if (lambda_bar && s_lbar < n && batch > 1) return -9;
  if (U_bar && ldub < n) return -11;
  if (U_bar && s_ubar < (long long)ldub * n && batch > 1) return -12;
  if (!(deg_tol >= 0.0)) return -13;
  if (!H_bar) return -14;
  if (ldh < n) return -15;
  if (s_h < (long long)ldh * n && batch > 1) return -16;
  if (G_bar && !G) return -17;
  if (G && ldg < n) return -18;
  if (G && s_g < (long long)ldg * n && batch > 1) return -19;
  if (J && s_j < n && batch > 1) return -21;
  if (G_bar && ldgb < n) return -23;
  if (G_bar && s_gb < (long long)ldgb * n && batch > 1) return -24;
  if (batch == 0) return JAC_OK;
  const long long nn = (long long)n * n;
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, sizeof(double) * 2 * nn * batch, st) != cudaSuccess) {
    cudaGetLastError();
    return JAC_ENOMEM;
  }
  double* M = static_cast<double*>(scratch);
  double* T = M + nn * batch;
  int rg = 0;
  // M = U^T U_bar
  if (U_bar) rg |= oz_gemm_launch(n, n, n, U, ldu, 1, U_bar, ldub, nullptr, nullptr, M, n, 0, 0, s_u, s_ubar, nn, batch, st);
  const int eb = (int)std::min<long long>(1024, (nn + 255) / 256);
  k_bwd_mid<<<dim3(eb, batch), 256, 0, st>>>(n, M, nn, lambda, s_lam, lambda_bar, s_lbar, U_bar ? 1 : 0, deg_tol);
  // T = U K_s, H_bar = T U^T (symmetric: upper entries, mirrored)
  rg |= oz_gemm_launch(n, n, n, U, ldu, 0, M, n, nullptr, nullptr, T, n, 0, 0, s_u, nn, nn, batch, st);
  rg |= oz_gemm_launch(n, n, n, T, n, 0, U, ldu, nullptr, nullptr, H_bar, ldh, 1, 1, nn, s_u, s_h, batch, st);
  if (G_bar) {  // G_bar = 2 H_bar G J
    rg |= oz_gemm_launch(n, n, n, H_bar, ldh, 0, G, ldg, nullptr, nullptr, G_bar, ldgb, 0, 0, s_h, s_g, s_gb, batch, st);
    k_scale_cols<<<dim3(eb, batch), 256, 0, st>>>(n, n, G_bar, ldgb, s_gb, J, s_j, 2.0);
  }
  int status = (rg == 0 && cudaGetLastError() == cudaSuccess) ? JAC_OK : JAC_ECUDA;
  cudaFreeAsync(scratch, st);
  return status;
}
