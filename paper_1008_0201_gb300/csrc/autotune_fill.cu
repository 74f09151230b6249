// autotune_fill.cu -- synthetic inputs for the batched-width autotuner (no method arithmetic):
// counter-based uniforms (the splitmix64 finalizer of Steele, Lea and Flood) and Gaussians from
// them by the Box-Muller transform.
#include "jacobi_common.cuh"

namespace jac {

// x[i] = uniform in [-1, 1) from a counter-based hash of (seed, i) (splitmix64 finalizer).
__global__ void k_fill_uniform(double* __restrict__ x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

// x[i] = N(0, 1) by the Box-Muller transform of two such uniforms (in (0, 1] and [0, 1)).
__global__ void k_fill_gauss(double* __restrict__ x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long u[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(2 * i + h + 1);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      u[h] = z >> 11;
    }
    const double u1 = (double)(u[0] + 1) * 0x1.0p-53, u2 = (double)u[1] * 0x1.0p-53;
    x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

}  // namespace jac
