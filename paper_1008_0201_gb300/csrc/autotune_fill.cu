// autotune_fill.cu -- synthetic inputs for the batched-width autotuner (no method arithmetic).
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

}  // namespace jac
