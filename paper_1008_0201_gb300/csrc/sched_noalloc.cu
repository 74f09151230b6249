// sched_noalloc.cu -- the device scheduler for callers that cannot allocate device memory.
//
// jacobi_sched_pairs() takes the scratch of the per-cycle weight ordering (the rank-ordered
// pair list and the step count) from cudaMallocAsync.  Some callers cannot make that call: a
// process whose device memory is owned by an external pool or arena and must not grow behind
// its back, code that runs with a fixed memory budget (long-lived services that pre-reserve
// everything at start-up), or a caller that must not take the allocator's locks or trigger its
// implicit synchronization on the hot path.  jacobi_sched_pairs_noalloc() runs the same
// scheduling kernel with its scratch in a fixed array that lives in the library image instead.
#include <mutex>

#include "jacobi_common.cuh"
#include "jacobi_gb300.h"

namespace jac {
__global__ void k_sched_static(int nb, int ordering, int nsteps, int* pairs, int* counts);
__global__ void k_sched_rank(int nb, const double* w, int* order);
__global__ void k_sched_cycle_weight(int nb, int* order, int* pairs, int* counts, int max_steps, int* nsteps_out);
}  // namespace jac

namespace {

// Block counts up to 256, i.e. up to 256 * 255 / 2 = 32640 block pairs per cycle.
constexpr int kMaxNb = JAC_NOALLOC_MAX_NB;
constexpr int kMaxPairs = kMaxNb * (kMaxNb - 1) / 2;

// Scratch of the weight ordering: kMaxPairs ints for the ranked pair list, then the step count
// (~128 KiB).  Every device that loads the library holds this array until the process exits.
// In host code the name is only a host-side stand-in; kernels get its device address from
// cudaGetSymbolAddress below.
static __device__ __align__(256) int g_sched_scratch[kMaxPairs + 64];

std::mutex g_scratch_mutex;
int* g_scratch_addr[64] = {};  // device address of g_sched_scratch, per device ordinal

// Resolves the device address of the scratch array on the current device (once per device).
int scratch_on_current_device(int** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return JAC_ECUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sched_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return JAC_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<int*>(p);
  }
  *out = g_scratch_addr[dev];
  return JAC_OK;
}

}  // namespace

extern "C" int jacobi_sched_pairs_noalloc(int nb, int ordering, const double* weights, int* pairs, int* counts,
                                          int max_steps, int* nsteps, jac_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nb < 2 || (nb & 1) || nb > kMaxNb) return -1;  // beyond JAC_NOALLOC_MAX_NB: rejected
  if (ordering < 0 || ordering > 3) return -2;
  if (ordering == JAC_ORDER_CYCLE_WEIGHT && !weights) return -3;
  if (!pairs) return -4;
  if (!counts) return -5;
  const int need = (ordering == JAC_ORDER_ROUND_ROBIN) ? nb - 1 : (ordering == JAC_ORDER_CYCLE_WEIGHT ? 1 : nb);
  if (max_steps < need) return -6;
  if (!nsteps) return -7;
  if (ordering != JAC_ORDER_CYCLE_WEIGHT) {
    // the static orderings need no scratch
    jac::k_sched_static<<<need, 128, 0, st>>>(nb, ordering, need, pairs, counts);
    if (cudaGetLastError() != cudaSuccess) return JAC_ECUDA;
    *nsteps = need;
    return cudaStreamSynchronize(st) == cudaSuccess ? JAC_OK : JAC_ECUDA;
  }
  int* scratch = nullptr;
  if (int r = scratch_on_current_device(&scratch)) return r;
  int* order = scratch;
  int* dn = scratch + kMaxPairs;
  // the step count is the only value read back; start it at zero so that a failed launch
  // cannot return the previous call's count
  if (cudaMemsetAsync(dn, 0, sizeof(int), st) != cudaSuccess) return JAC_ECUDA;
  jac::k_sched_rank<<<(nb * (nb - 1) / 2 + 255) / 256, 256, sizeof(double) * nb, st>>>(nb, weights, order);
  jac::k_sched_cycle_weight<<<1, 1024, sizeof(int) * nb, st>>>(nb, order, pairs, counts, max_steps, dn);
  int status = (cudaGetLastError() == cudaSuccess) ? JAC_OK : JAC_ECUDA;
  int h = -1;
  if (cudaMemcpyAsync(&h, dn, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) status = JAC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) status = JAC_ECUDA;
  if (status == JAC_OK && h <= 0) status = JAC_EINTERNAL;
  *nsteps = h;
  return status;
}
