// capi.cu -- host driver of the sweep loop and the C ABI declared in include/jacobi_gb300.h.
//
// The driver does no numerics on the host.  It validates arguments, lays out the block
// partition (Sec. 3: widths differ by at most one), builds one descriptor per problem (a single
// solve is a batch of one) and launches, per sweep, the step kernels gram -> pivot -> update for
// every step of the ordering, then the sweep reduction.  The only values read back per sweep
// are one small record (single solve) or the number of problems still active (batch).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "jacobi_common.cuh"
#include "jacobi_gb300.h"

namespace jac {
__global__ void k_sched_static(int nb, int ordering, int nsteps, int* pairs, int* counts);
__global__ void k_sched_rank(int nb, const double* w, int* order);
__global__ void k_sched_cycle_weight(int nb, int* order, int* pairs, int* counts, int max_steps, int* nsteps_out);
__global__ void k_block_weights32(const float* G32, int mp, int nb, const int* boff, double* w);
__global__ void k_gram(const JacProb* probs, int s, int CS);
__global__ void k_update(const JacProb* probs, int s, int gslabs);
__global__ void k_gram32(const JacProb* probs, int s, int CS);
__global__ void k_update32(const JacProb* probs, int s, int gslabs);
int pivot_set_attributes();
void pivot_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s, const PivotParams& pp);
void fused_step_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                       const PivotParams& pp);
int fused_step_max_rows(int km);
int pivot64_set_attributes();
void pivot64_launch(int km, int max_half, int nprob, cudaStream_t st, const JacProb* probs, int s,
                    const PivotParams& pp);
__global__ void k_sweep_reduce(JacProb* probs, JacIO* io, SweepRecord* rec, int deactivate, int* remaining);
__global__ void k_cache_init(const JacProb* probs);
__global__ void k_cache_step(const JacProb* probs, int rec, int chk);
__global__ void k_sort_signs(const JacProb* probs, JacIO* io, int8_t* Js_all, const long long* js_off);
__global__ void k_apply_flags(JacProb* probs, const JacIO* io, int nprob);
__global__ void k_gather_in(const JacProb* probs, const JacIO* io);
__global__ void k_init_v(const JacProb* probs, const JacIO* io);
__global__ void k_check_finite(const JacProb* probs, JacIO* io);
__global__ void k_colnorm(const JacProb* probs, const JacIO* io);
__global__ void k_rank(const JacProb* probs, const JacIO* io);
__global__ void k_scatter(const JacProb* probs, const JacIO* io);
__global__ void k_gemm64(int Mr, int Nc, int K, const double* A, int lda, int transA, const double* B, int ldb,
                         const int8_t* sb, const int8_t* dsub, double* C, int ldc, int sym, int transB, long long sa,
                         long long sbb, long long sc);
__global__ void k_ns_correct(int Mr, int Nc, int K, const float* Af, int lda, const float* Bf, int ldb, double* V,
                             int ldv);
__global__ void k_cvt64to32(int rows, int cols, const double* src, int lds, float* dst, int ldd, const int8_t* rsign);
__global__ void k_cvt32to64(int rows, int cols, const float* src, int lds, double* dst, int ldd);
__global__ void k_absmax64(int n, const double* M, int ldm, unsigned long long* out);
__global__ void k_lowp_copy(const JacProb* probs, int to64);
__global__ void k_realify(int m, int n, const double2* G, int ldg, const int8_t* J, double* Gr, int8_t* Jr);
__global__ void k_complexify(int m, int n, const double* Gr, const double* lam_r, const double* Vr, double2* G, int ldg,
                             double* lambda, double2* U, int ldu, double2* V, int ldv, unsigned* bad);
__global__ void k_restructure(int h, int n, const double* in, double* out, const double* lam, int8_t* Jout);
__global__ void k_fill_uniform(double* x, long long n, unsigned long long seed);
__global__ void k_fill_gauss(double* x, long long n, unsigned long long seed);
__global__ void k_gram_oz(const JacProb* probs, int s, int CS);
__global__ void k_update_oz(const JacProb* probs, int s, int gslabs);
__global__ void k_gram32_tc(const JacProb* probs, int s, int CS, const __grid_constant__ CUtensorMap tmG);
__global__ void k_update32_tc(const JacProb* probs, int s, int gtiles, int tpc, const __grid_constant__ CUtensorMap tmG,
                              const __grid_constant__ CUtensorMap tmV);
__global__ void k_update_oz_tc(const JacProb* probs, int s);
__global__ void k_gram_oz_tc(const JacProb* probs, int s, int CS);
size_t tc_update_oz_smem_bytes();
size_t tc_gram_oz_smem_bytes();
size_t tc_gram32_smem_bytes();
size_t tc_update32_smem_bytes();
size_t oz_gram_smem_bytes();
size_t oz_update_smem_bytes();
int oz_gemm_launch(int Mr, int Nc, int K, const double* A, int lda, int transA, const double* B, int ldb,
                   const int8_t* sb, const int8_t* dsub, double* C, int ldc, int sym, int transB, long long sa,
                   long long sbb, long long sc, int batch, cudaStream_t st);
}  // namespace jac

using namespace jac;

namespace {

constexpr size_t kGramSmem = (size_t)(JAC_KMAX * (64 + 2) + JAC_KMAX * (JAC_KMAX + 1)) * sizeof(double);
constexpr size_t kUpdSmem = (size_t)(JAC_KMAX * (JAC_KMAX + 2) + 64 * (JAC_KMAX + 2)) * sizeof(double);

// ---- optional kernel timing (jacobi_profile_*) ------------------------------------------
std::mutex g_prof_mutex;
int g_prof_mask = 0;
double g_prof_ms[JAC_KERNEL_COUNT] = {};
long long g_prof_n[JAC_KERNEL_COUNT] = {};
std::vector<cudaEvent_t> g_prof_pool;

// Per-solve list of event pairs; events come from the process-wide pool.
struct ProfRun {
  int mask = 0;
  std::vector<std::pair<int, size_t>> marks;  // (kernel, index of the start event in evs)
  std::vector<cudaEvent_t> evs;
  void begin() {
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    mask = g_prof_mask;
  }
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_prof_mutex);
      if (!g_prof_pool.empty()) {
        e = g_prof_pool.back();
        g_prof_pool.pop_back();
      }
    }
    if (!e && cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    return e;
  }
  size_t pre(int k, cudaStream_t st) {
    if (!(mask & (1 << k))) return (size_t)-1;
    cudaEvent_t a = take(), b = take();
    if (!a || !b) return (size_t)-1;
    evs.push_back(a);
    evs.push_back(b);
    // external: inside a stream capture the record becomes a graph node that records the event
    // at every replay (a plain record would only order the capture)
    cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
    marks.emplace_back(k, evs.size() - 2);
    return evs.size() - 2;
  }
  void post(size_t idx, cudaStream_t st) {
    if (idx != (size_t)-1) cudaEventRecordWithFlags(evs[idx + 1], st, cudaEventRecordExternal);
  }
  void accumulate() {  // after the stream has been synchronized; the events stay with this run
    if (evs.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    for (auto& mk : marks) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[mk.second], evs[mk.second + 1]) == cudaSuccess && g_prof_mask) {
        g_prof_ms[mk.first] += ms;
        g_prof_n[mk.first] += 1;
      } else {
        cudaGetLastError();  // a timing failure must not surface as a later launch error
      }
    }
  }
  void release() {
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    for (auto e : evs) g_prof_pool.push_back(e);
    evs.clear();
    marks.clear();
  }
  void finish() {  // after the stream has been synchronized
    accumulate();
    release();
  }
};

std::mutex g_attr_mutex;
bool g_attr_done[64] = {};

int setup_attributes(int dev) {
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  if (dev < 0 || dev >= 64) return JAC_ECUDA;
  if (g_attr_done[dev]) return 0;
  bool ok = true;
  ok &= cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramSmem) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_gram_smem_bytes()) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_update_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_update_smem_bytes()) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gram32_smem_bytes()) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram32_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_update32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_update32_smem_bytes()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_update_oz_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_update_oz_smem_bytes()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram_oz_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_gram_oz_smem_bytes()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gram_oz_tc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  ok &= pivot_set_attributes() == 0;
  ok &= pivot64_set_attributes() == 0;
  ok &= cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return JAC_ECUDA;
  }
  g_attr_done[dev] = true;
  return 0;
}

// Carves one cudaMallocAsync block into 256-byte aligned pieces (a first pass with base == NULL
// only measures).
struct Arena {
  size_t off = 0;
  char* base = nullptr;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

// TMA tensor maps of the FP32 copies of one problem (FP32 sweeps on the tensor cores): 2-D
// column-major (rows contiguous), 32 x 32 boxes, 128-byte swizzle.  cuTensorMapEncodeTiled comes
// from the driver through the runtime's entry-point query (no link against the driver library).
struct TcMaps {
  CUtensorMap g32, v32;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
std::mutex g_encode_mutex;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_fn() {
  std::lock_guard<std::mutex> lk(g_encode_mutex);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

// rows x cols FP32, leading dimension ld (rows <= ld, ld * 4 a multiple of 16, base 16-byte aligned)
int encode_f32_map(CUtensorMap* m, float* base, int rows, int cols, int ld) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || !base || (ld * 4) % 16 || (reinterpret_cast<uintptr_t>(base) & 15)) return JAC_ECUDA;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
                 CUDA_SUCCESS
             ? 0
             : JAC_ECUDA;
}

int check_opts(const jac_opts& o, int argpos, bool batch) {
  if (o.block_w < 1 || o.block_w > JAC_WMAX) return -argpos;
  if (o.ordering < 0 || o.ordering > 3) return -argpos;
  if (batch && o.ordering == JAC_ORDER_CYCLE_WEIGHT) return -argpos;
  if (o.block_mode != JAC_BLOCK_FULL && o.block_mode != JAC_BLOCK_ORIENTED) return -argpos;
  if (o.factor != JAC_FACTOR_CHOL && o.factor != JAC_FACTOR_CHOL_DIAGPIV && o.factor != JAC_FACTOR_CHOL_SIGNPIV)
    return -argpos;
  if (o.precision < JAC_PREC_FP64 || o.precision > JAC_PREC_FP32_ONLY) return -argpos;
  if (batch && o.precision == JAC_PREC_FP32) return -argpos;
  if (o.max_sweeps < 1) return -argpos;
  if (o.want_v != 0 && o.want_v != 1) return -argpos;
  if (o.f64_products < JAC_F64_MMA || o.f64_products > JAC_F64_SPLIT16_TC) return -argpos;
  if (o.fused_step != 0 && o.fused_step != 1) return -argpos;
  return 0;
}

int compute_nb(int n, int w) {
  int nb = 2 * ((n + 2 * w - 1) / (2 * w));
  if (nb < 2) nb = 2;
  if (nb > n) nb = n & ~1;
  if (nb < 2) nb = 2;
  return nb;
}

// CTAs per pivot block of the Gram kernels (a cluster splitting the rows): the FP64 mma Gram is
// bound by the FP64 mma rate and takes every SM it can (>= 16 rows per CTA); the FP32 Gram is
// ~64x cheaper per row, so its CTAs keep >= 64 rows and the cluster reduction stays short
// (measured on the 512 x 512 workload: 64 rows per CTA beat 32, 128, 256 and 512).
int choose_cluster(int half, int mp, int min_rows) {
  int cs = 1;
  while (cs * 2 <= 16 && half * cs * 2 <= 2 * 152 && mp / (cs * 2) >= min_rows) cs *= 2;
  return cs;
}

template <class Kern, class... Args>
int launch_cluster(Kern kern, dim3 grid, int CS, int threads, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...) == cudaSuccess ? 0 : JAC_ECUDA;
}

// Block width of one problem of a batch, by size class.  Width rules: 0 = the whole problem is
// one pivot block (w = ceil(n/2), one step per sweep; needs n <= 64), else a fixed width w.
// Default: one block up to n = 64 (KM = 32 while n <= 32), blocks of 32 columns above (nb = 4,
// three round-robin steps of two pivot blocks).  jacobi_autotune_batched replaces the default
// per size class with the fastest rule it measures on the device.
std::mutex g_tune_mutex;
int g_tuned_rule[64][129];  // per device and order: -1 untuned, else a width rule
bool g_tune_init = false;

int width_of_rule(int rule, int n) { return rule == 0 ? (n + 1) / 2 : std::min(rule, (n + 1) / 2); }

int batch_width(int n) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    if (g_tune_init && dev >= 0 && dev < 64 && n >= 0 && n <= 128 && g_tuned_rule[dev][n] >= 0)
      return width_of_rule(g_tuned_rule[dev][n], n);
  }
  return n <= 64 ? (n + 1) / 2 : 32;
}

// Per-problem plan: sizes of its pieces.
struct Plan {
  int m, n, mp, np, nb, half, nsteps, km, ordering;
  bool want_v, have_vw, lowp;
  std::vector<int> boff;
};

void make_plan(Plan& P, int m, int n, int w, int ordering, bool want_v, bool have_vw, bool lowp) {
  P.m = m;
  P.n = n;
  P.mp = (m + 15) & ~15;
  P.np = (n + 15) & ~15;
  P.nb = compute_nb(n, w);
  P.half = P.nb / 2;
  P.ordering = ordering;
  P.nsteps = (ordering == JAC_ORDER_ROUND_ROBIN) ? P.nb - 1 : (ordering == JAC_ORDER_CYCLE_WEIGHT ? 2 * P.nb : P.nb);
  P.boff.resize(P.nb + 1);
  const int base = n / P.nb, rem = n % P.nb;
  int off = 0, wmax = 0;
  for (int b = 0; b < P.nb; ++b) {
    P.boff[b] = off;
    const int wb = base + (b < rem ? 1 : 0);
    wmax = std::max(wmax, wb);
    off += wb;
  }
  P.boff[P.nb] = off;
  P.km = (2 * wmax <= 32) ? 32 : 64;
  P.want_v = want_v;
  P.have_vw = have_vw;
  P.lowp = lowp;
}

// Device pieces of one problem (pointers into the arena).
void carve_problem(Arena& ar, const Plan& P, JacProb& d, JacIO& io, bool weights) {
  d.Gw = ar.take<double>((size_t)P.mp * P.n);
  d.Vw = P.have_vw ? ar.take<double>((size_t)P.np * P.n) : nullptr;
  d.G32 = (P.lowp || weights) ? ar.take<float>((size_t)P.mp * P.n) : nullptr;
  d.V32 = (P.lowp && P.have_vw) ? ar.take<float>((size_t)P.np * P.n) : nullptr;
  d.mp = P.mp;
  d.np = P.np;
  d.n = P.n;
  d.nb = P.nb;
  d.half = P.half;
  d.nsteps = P.nsteps;
  d.apld = P.km;
  d.Ap = ar.take<double>((size_t)P.half * P.km * P.km);
  d.vp = ar.take<double>((size_t)P.half * P.km * P.km);
  d.active = 1;
  d.skip = ar.take<int>(P.half);
  d.stats = ar.take<PairStat>((size_t)P.nsteps * P.half);
  d.cached = weights ? nullptr : ar.take<int>(P.half);  // pair cache: off for the weight ordering
  d.pver = weights ? nullptr : ar.take<int4>((size_t)P.nsteps * P.half);
  d.bver = weights ? nullptr : ar.take<int>(P.nb);
  io.perm_in = ar.take<int>(P.n);
  io.nrm2 = ar.take<double>(P.n);
  io.lam = ar.take<double>(P.n);
  io.rank = ar.take<int>(P.n);
  io.m = P.m;
  io.flags = 0;
  io.sweeps = 0;
  io.rotations = 0;
}

// One launch of the three step kernels for every problem of a class array.
// fallback = false leaves out the FP64 pivot kernel: blocks the FP32 pivot hands over are then
// not rotated in this step (the FP32 sweeps of the mixed mode switch to FP64 on a handover).
// Work split of the tensor-core FP32 update: 128-row tiles of G32 then V32, ysplit CTAs per pair.
struct TcSplit {
  int gtiles = 0, ysplit = 1, tpc = 1;
};

int launch_step(JacProb* dprobs, int count, int km, int max_half, int gslabs, int tslabs, int CS, int CS32, int s,
                bool lowp, bool fallback, const PivotParams& pp, cudaStream_t st, ProfRun& prof,
                long long& launches, const TcMaps* maps = nullptr, const TcSplit* tsp = nullptr,
                bool fused = false) {
  // the pair cache: record step s - 1, then mark the pairs of step s whose outcome is known
  k_cache_step<<<count, 256, 0, st>>>(dprobs, s - 1, s);
  int r = 0;
  if (lowp && fused) {
    // FP32 sweep step of small problems: Gram, pivot and update of each pair in one CTA (pivot.cu,
    // k_step_fused); a block it hands over takes the FP64 pivot, then the plain FP32 update,
    // which acts only on those blocks (the fused kernel marks its own pairs done)
    size_t pm = prof.pre(JAC_KERNEL_STEP_FUSED, st);
    fused_step_launch(km, max_half, count, st, dprobs, s, pp);
    if (fallback) pivot64_launch(km, max_half, count, st, dprobs, s, pp);
    prof.post(pm, st);
    if (fallback) {
      pm = prof.pre(JAC_KERNEL_UPDATE_LOWP, st);
      k_update32<<<dim3(max_half, tslabs, count), 256, 0, st>>>(dprobs, s, gslabs);
      prof.post(pm, st);
    }
    launches += fallback ? 4 : 2;
    return cudaGetLastError() == cudaSuccess ? 0 : JAC_ECUDA;
  }
  size_t pm = prof.pre(lowp ? JAC_KERNEL_GRAM_LOWP : JAC_KERNEL_GRAM, st);
  if (lowp && maps)
    r = launch_cluster(k_gram32_tc, dim3(max_half * CS32, count), CS32, 128, tc_gram32_smem_bytes(), st,
                       (const JacProb*)dprobs, s, CS32, maps->g32);
  else if (lowp)
    r = launch_cluster(k_gram32, dim3(max_half * CS32, count), CS32, 128, 0, st, (const JacProb*)dprobs, s, CS32);
  else if (pp.oz == 2)
    r = launch_cluster(k_gram_oz_tc, dim3(max_half * CS, count), CS, 512, tc_gram_oz_smem_bytes(), st,
                       (const JacProb*)dprobs, s, CS);
  else if (pp.oz)
    r = launch_cluster(k_gram_oz, dim3(max_half * CS, count), CS, 256, oz_gram_smem_bytes(), st,
                       (const JacProb*)dprobs, s, CS);
  else
    r = launch_cluster(k_gram, dim3(max_half * CS, count), CS, 128, kGramSmem, st, (const JacProb*)dprobs, s, CS);
  prof.post(pm, st);
  if (r) return r;
  pm = prof.pre(JAC_KERNEL_PIVOT, st);
  pivot_launch(km, max_half, count, st, dprobs, s, pp);
  if (fallback) pivot64_launch(km, max_half, count, st, dprobs, s, pp);  // blocks the FP32 kernel handed over
  prof.post(pm, st);
  pm = prof.pre(lowp ? JAC_KERNEL_UPDATE_LOWP : JAC_KERNEL_UPDATE, st);
  if (lowp && maps && tsp)
    k_update32_tc<<<dim3(max_half, tsp->ysplit, count), 128, tc_update32_smem_bytes(), st>>>(
        dprobs, s, tsp->gtiles, tsp->tpc, maps->g32, maps->v32);
  else if (lowp)
    k_update32<<<dim3(max_half, tslabs, count), 256, 0, st>>>(dprobs, s, gslabs);
  else if (pp.oz) {
    // tensor-core digit update: persistent CTAs (one per SM) over the (pair, 128-row tile) items
    // of each problem (tslabs counts 64-row slabs)
    const int items = max_half * ((tslabs + 1) / 2 + 1);
    const int nx = std::max(1, std::min(items, (152 + count - 1) / count));
    k_update_oz_tc<<<dim3(nx, 1, count), 512, tc_update_oz_smem_bytes(), st>>>(dprobs, s);
  }
  else
    k_update<<<dim3(max_half, tslabs, count), 128, kUpdSmem, st>>>(dprobs, s, gslabs);
  prof.post(pm, st);
  launches += fallback ? 5 : 4;
  return cudaGetLastError() == cudaSuccess ? 0 : JAC_ECUDA;
}

// One sweep's launches recorded once as a CUDA graph and replayed every sweep with the same
// parameters (the launches of a sweep differ only by the step index, which the graph holds).
// Capture runs on a private stream of the device (the caller's stream may be the legacy default
// stream, which cannot be captured); the graph is launched on the caller's stream.
std::mutex g_capture_mutex;
cudaStream_t g_capture_stream[64] = {};

struct SweepGraph {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels per replay
  ProfRun prof;            // event pairs recorded by the graph (kernel timing on), read per replay
  ~SweepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    prof.release();
  }
  // record(stream, launches&) issues the sweep's launches; returns 0 or a status
  template <class Fn>
  int build(Fn record) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return JAC_ECUDA;
    std::lock_guard<std::mutex> lk(g_capture_mutex);
    if (!g_capture_stream[dev] &&
        cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
      return JAC_ECUDA;
    cudaStream_t cs = g_capture_stream[dev];
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return JAC_ECUDA;
    long long n = 0;
    const int r = record(cs, n);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (r || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return r ? r : JAC_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      exec = nullptr;
      cudaGetLastError();
      return JAC_ECUDA;
    }
    launches = n;
    return 0;
  }
};

struct ArgPos {  // 1-based positions of the arguments in the public signature
  int m, n, dtype, G, ldg, J, opts, lambda, U, ldu, V, ldv;
};

// Extra device pieces of a single solve.
struct Single {
  JacProb* probs;
  JacIO* io;
  SweepRecord* rec;
  unsigned* flags;
  int8_t* Js;
  long long* jsoff;
  int* pairs;
  int* counts;
  double* weights;
  int* order;
  double* Mn;
  float* Mf;
  float* Vf;
  unsigned long long* mmax;
};

// ------------------------------------------------------------------ single solve
int solve_real(int m, int n, int dtype, void* Gv, int ldg, const int8_t* Jdev, const jac_opts* opts_in, double* lambda,
               void* Uv, int ldu, void* Vv, int ldv, jac_info* info, cudaStream_t st, const ArgPos& ap,
               const double* Vinit = nullptr, bool strict_stop = false) {
  jac_opts o;
  jacobi_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (info) std::memset(info, 0, sizeof(*info));
  auto fail_arg = [&](int pos) {
    if (info) info->status = -pos;
    return -pos;
  };
  if (m < 1) return fail_arg(ap.m);
  if (n < 1 || n > m || n > 20000) return fail_arg(ap.n);
  if (dtype != JAC_R64) return fail_arg(ap.dtype);
  if (!Gv) return fail_arg(ap.G);
  if (ldg < m) return fail_arg(ap.ldg);
  if (ap.J && !Jdev) return fail_arg(ap.J);
  if (int r = check_opts(o, ap.opts, false)) return fail_arg(-r);
  if (o.ordering == JAC_ORDER_CYCLE_WEIGHT && compute_nb(n, o.block_w) > JAC_CYCLE_WEIGHT_MAX_NB)
    return fail_arg(ap.opts);
  if (!lambda) return fail_arg(ap.lambda);
  if (Uv && ldu < m) return fail_arg(ap.ldu);
  if (Uv && Uv == Gv) return fail_arg(ap.U);
  if (o.want_v && !Vv) return fail_arg(ap.V);
  if (Vv && ldv < n) return fail_arg(ap.ldv);
  const bool fp32_only = (o.precision == JAC_PREC_FP32_ONLY);
  if (o.tol <= 0.0)
    o.tol = fp32_only ? std::max((double)n, 8.0 * std::sqrt((double)m)) * 5.9604644775390625e-08
                      : (double)n * 1.1102230246251565e-16;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JAC_ECUDA;
  if (int r = setup_attributes(dev)) return r;

  const bool weights = (o.ordering == JAC_ORDER_CYCLE_WEIGHT);
  const bool mixed = (o.precision == JAC_PREC_FP32);
  const bool lowp = mixed || fp32_only;
  const bool want_v = o.want_v != 0;
  const bool have_vw = want_v || mixed;  // the mixed mode needs V for G = G_in V
  Plan P;
  make_plan(P, m, n, o.block_w, o.ordering, want_v, have_vw, lowp);

  JacProb hp = {};
  JacIO hio = {};
  int* boff_dev = nullptr;
  Single L;
  auto carve_all = [&](Arena& A) {
    carve_problem(A, P, hp, hio, weights);
    boff_dev = A.take<int>(P.nb + 1);
    L.probs = A.take<JacProb>(1);
    L.io = A.take<JacIO>(1);
    L.rec = A.take<SweepRecord>(1);
    L.flags = A.take<unsigned>(1);
    L.Js = A.take<int8_t>(n);
    L.jsoff = A.take<long long>(1);
    L.pairs = A.take<int>((size_t)P.nsteps * P.half * 2);
    L.counts = A.take<int>(P.nsteps);
    L.weights = weights ? A.take<double>((size_t)P.nb * P.nb) : nullptr;
    L.order = weights ? A.take<int>(P.nb * (P.nb - 1) / 2) : nullptr;
    L.Mn = mixed ? A.take<double>((size_t)n * n) : nullptr;
    L.Mf = mixed ? A.take<float>((size_t)n * n) : nullptr;
    L.Vf = mixed ? A.take<float>((size_t)n * n) : nullptr;
    L.mmax = A.take<unsigned long long>(1);
  };
  Arena ar;
  carve_all(ar);
  void* base = nullptr;
  if (cudaMallocAsync(&base, ar.off, st) != cudaSuccess) {
    cudaGetLastError();
    return JAC_ENOMEM;
  }
  Arena ar2;
  ar2.base = static_cast<char*>(base);
  carve_all(ar2);
  hp.boff = boff_dev;
  hp.tol = o.tol;
  hp.Js = L.Js;
  hp.pairs = L.pairs;
  hp.counts = L.counts;
  hp.pflags = L.flags;
  hio.G = static_cast<double*>(Gv);
  hio.ldg = ldg;
  hio.J = Jdev;
  hio.lambda = lambda;
  hio.U = static_cast<double*>(Uv);
  hio.ldu = ldu;
  hio.V = want_v ? static_cast<double*>(Vv) : nullptr;
  hio.ldv = ldv;
  hio.Vinit = Vinit;
  hio.ldvi = n;

  int status = JAC_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  };
  const long long zero = 0;
  ck(cudaMemcpyAsync(boff_dev, P.boff.data(), sizeof(int) * (P.nb + 1), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.probs, &hp, sizeof(JacProb), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.io, &hio, sizeof(JacIO), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.jsoff, &zero, sizeof(long long), cudaMemcpyHostToDevice, st));
  ck(cudaMemsetAsync(L.flags, 0, sizeof(unsigned), st));

  // FP32 sweeps of a single solve run on the tensor cores (TMA tensor maps of the FP32 copies)
  TcMaps tmaps;
  TcSplit tsplit;
  bool use_tc = false;
  if (lowp && status == JAC_OK) {
    use_tc = encode_f32_map(&tmaps.g32, hp.G32, P.mp, n, P.mp) == 0;
    if (use_tc) use_tc = encode_f32_map(&tmaps.v32, hp.V32 ? hp.V32 : hp.G32, hp.V32 ? P.np : P.mp, n,
                                        hp.V32 ? P.np : P.mp) == 0;
    tsplit.gtiles = (P.mp + 127) / 128;
    const int ntiles = tsplit.gtiles + (hp.V32 ? (P.np + 127) / 128 : 0);
    tsplit.ysplit = std::max(1, std::min(ntiles, (2 * 152 + P.half - 1) / P.half));
    tsplit.tpc = (ntiles + tsplit.ysplit - 1) / tsplit.ysplit;
    tsplit.ysplit = (ntiles + tsplit.tpc - 1) / tsplit.tpc;
  }

  long long launches = 0;
  k_sort_signs<<<1, 32, 0, st>>>(L.probs, L.io, L.Js, L.jsoff);
  k_check_finite<<<dim3(std::min(1024, (int)(((size_t)m * n + 255) / 256)), 1), 256, 0, st>>>(L.probs, L.io);
  launches += 2;
  JacIO hio_back;
  ck(cudaMemcpyAsync(&hio_back, L.io, sizeof(JacIO), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  if (status == JAC_OK && (hio_back.flags & 2)) {
    cudaFreeAsync(base, st);
    cudaStreamSynchronize(st);
    return fail_arg(ap.J);
  }
  if (status == JAC_OK && (hio_back.flags & 1)) status = JAC_ENONFINITE;
  k_gather_in<<<dim3((P.mp + 255) / 256, n, 1), 256, 0, st>>>(L.probs, L.io);
  if (have_vw) k_init_v<<<dim3((P.np + 255) / 256, n, 1), 256, 0, st>>>(L.probs, L.io);
  k_cache_init<<<1, 256, 0, st>>>(L.probs);
  launches += have_vw ? 3 : 2;
  ck(cudaGetLastError());

  int nsteps = P.nsteps;
  if (status == JAC_OK && !weights) {
    k_sched_static<<<P.nsteps, 128, 0, st>>>(P.nb, o.ordering, P.nsteps, L.pairs, L.counts);
    ++launches;
    ck(cudaGetLastError());
  }
  // the digit-product Gram is ~20x cheaper per row than the FP64 mma one and takes a whole SM
  // (all 512 tensor-memory columns, ~165 KB of shared memory) per CTA, which works on groups of
  // 128 rows: >= 128 rows per CTA
  const bool split16 = o.f64_products != JAC_F64_MMA;
  const int CS = choose_cluster(P.half, P.mp, split16 ? (o.f64_products == JAC_F64_SPLIT16_TC ? 128 : 64) : 16),
            CS32 = choose_cluster(P.half, P.mp, 64);
  const int gslabs = (P.mp + 63) / 64;
  const int tslabs = gslabs + (have_vw ? (P.np + 63) / 64 : 0);
  const int ew_blocks = std::min(1024, (int)(((size_t)P.mp * n + 255) / 256));
  // FP32 sweeps of the mixed mode stop at the scaled off-norm the FP32 Gram still resolves (its
  // entries carry errors ~ eps_32 sqrt(m) relative to ||g_i|| ||g_j||)
  const double tau_lo = std::max(o.tol, 8.0 * 5.9604644775390625e-08 * std::sqrt((double)m));
  // FP32 sweeps of small problems: one fused kernel per step
  const bool fused = o.fused_step == 1 && P.mp <= fused_step_max_rows(P.km);
  int phase = mixed ? 1 : (fp32_only ? 4 : 3);  // 1: FP32 sweeps of the mixed mode, 3: FP64, 4: FP32 only
  if (lowp && status == JAC_OK) {
    k_lowp_copy<<<dim3(ew_blocks, 1), 256, 0, st>>>(L.probs, 0);  // FP64 layout -> FP32 copies
    launches += 1;
    ck(cudaGetLastError());
  }

  int sweeps = 0, converged = 0, lowp_sweeps = 0, ns_global = 0;
  long long rot_total = 0, piv_total = 0, piv_lowp = 0, cyc_total[4] = {0, 0, 0, 0}, ns_total = 0, inner_total = 0;
  long long ev_total = 0, ev_lowp = 0;
  double prev_max = 1e300;
  SweepRecord hrec = {};
  int last_steps = 0;
  ProfRun prof;
  prof.begin();
  double sweep_ms_h[64] = {};
  SweepGraph graphs[5];
  bool use_graphs = !weights;
  int phase_sweeps = 0;  // sweeps of the current (FP64 or FP32-only) phase
  for (int sw = 0; status == JAC_OK && n > 1 && sw < o.max_sweeps; ++sw) {
    const auto t_sweep = std::chrono::steady_clock::now();
    auto sweep_done = [&]() {
      if (sw < 64)
        sweep_ms_h[sw] =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_sweep).count();
    };
    const bool low = (phase == 1 || phase == 4);
    PivotParams pp;
    pp.tol = (phase == 1) ? tau_lo : o.tol;
    pp.tol_eps = 0.0;
    pp.tol_m = 0.0;
    pp.factor = o.factor;
    pp.ns_mode = low ? 0 : 1;
    pp.oriented = (o.block_mode == JAC_BLOCK_ORIENTED) ? 1 : 0;
    pp.oz = (o.f64_products == JAC_F64_SPLIT16) ? 1 : (o.f64_products == JAC_F64_SPLIT16_TC ? 2 : 0);
    if (weights) {
      const int npairs = P.nb * (P.nb - 1) / 2;
      if (!low) {
        k_cvt64to32<<<ew_blocks, 256, 0, st>>>(P.mp, n, hp.Gw, P.mp, hp.G32, P.mp, nullptr);
        ++launches;
      }
      int* nsteps_dev = reinterpret_cast<int*>(reinterpret_cast<char*>(L.probs) + offsetof(JacProb, nsteps));
      k_block_weights32<<<npairs, 256, 0, st>>>(hp.G32, P.mp, P.nb, boff_dev, L.weights);
      k_sched_rank<<<(npairs + 255) / 256, 256, sizeof(double) * P.nb, st>>>(P.nb, L.weights, L.order);
      k_sched_cycle_weight<<<1, 1024, sizeof(int) * P.nb, st>>>(P.nb, L.order, L.pairs, L.counts, P.nsteps,
                                                                nsteps_dev);
      launches += 3;
      ck(cudaGetLastError());
      ck(cudaMemcpyAsync(&nsteps, nsteps_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (status != JAC_OK) break;
      if (nsteps < 1 || nsteps > P.nsteps) {
        status = JAC_EINTERNAL;
        break;
      }
    }
    auto record = [&](cudaStream_t ss, long long& nl, ProfRun& pr) -> int {
      for (int s = 0; s < nsteps; ++s)
        if (int r = launch_step(L.probs, 1, P.km, P.half, gslabs, tslabs, CS, CS32, s, low, phase != 1, pp, ss, pr,
                                nl, use_tc ? &tmaps : nullptr, use_tc ? &tsplit : nullptr, fused))
          return r;
      k_cache_step<<<1, 256, 0, ss>>>(L.probs, -2, -1);  // record the last step of the sweep
      k_sweep_reduce<<<1, 256, 0, ss>>>(L.probs, L.io, L.rec, 0, nullptr);
      nl += 2;
      return cudaGetLastError() == cudaSuccess ? 0 : JAC_ECUDA;
    };
    // graphs: one per precision phase, unless the ordering is re-planned every sweep
    SweepGraph& sg = graphs[phase];
    if (use_graphs && !sg.exec) {
      sg.prof.begin();
      if (sg.build([&](cudaStream_t ss, long long& nl) { return record(ss, nl, sg.prof); })) {
        sg.prof.release();
        use_graphs = false;
      }
    }
    SweepGraph* replayed = nullptr;
    if (use_graphs && sg.exec) {
      if (cudaGraphLaunch(sg.exec, st) != cudaSuccess) status = JAC_ECUDA;
      launches += sg.launches;
      replayed = &sg;
    } else if (int r = record(st, launches, prof)) {
      status = r;
    }
    ck(cudaMemcpyAsync(&hrec, L.rec, sizeof(SweepRecord), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (replayed) replayed->prof.accumulate();
    if (status != JAC_OK) break;
    if (info && sweeps < 64) info->sweep_max_scaled[sweeps] = hrec.max_scaled;
    ++sweeps;
    last_steps = nsteps;
    rot_total += hrec.rotations;
    piv_total += hrec.pivots_rotated;
    if (phase == 1 || phase == 4) piv_lowp += hrec.pivots_rotated;
    ev_total += hrec.evaluated;
    if (phase == 1 || phase == 4) ev_lowp += hrec.evaluated;
    ns_total += hrec.ns_steps;
    inner_total += hrec.inner_sweeps;
    for (int u = 0; u < 4; ++u) cyc_total[u] += hrec.cyc[u];
    // a block the FP32 pivot could not factor or J-orthogonalize was handed over (and, in the
    // FP32 sweeps, left unrotated): the FP64 phase decides it
    bool lowp_singular = phase == 1 && (hrec.err & JAC_DEVERR_HANDOVER);
    if (hrec.err & JAC_DEVERR_TIMEOUT) {  // a bounded wait in a tensor-core kernel gave up
      status = JAC_EINTERNAL;
      break;
    }
    if (hrec.err & JAC_DEVERR_NOTPD) {
      if (phase != 1) {
        status = JAC_ENOTPD;
        break;
      }
      // a block whose FP32 Gram is singular at FP32 precision: the FP64 phase decides
      lowp_singular = true;
      static const int kActive = 1;
      ck(cudaMemsetAsync(L.flags, 0, sizeof(unsigned), st));
      ck(cudaMemcpyAsync(reinterpret_cast<char*>(L.probs) + offsetof(JacProb, active), &kActive, sizeof(int),
                         cudaMemcpyHostToDevice, st));
    }
    if (phase == 1) {
      ++lowp_sweeps;
      // leave the FP32 phase once the sweep has entered the quadratic regime (max scaled
      // off-diagonal below 1e-2): the switch itself resets the off-norm to the accuracy of the
      // FP32-accumulated V (~1e-4..1e-3 for the hyperbolic workload whatever the FP32 phase
      // reached), so further FP32 sweeps buy nothing.  Also when it has converged at tau_lo,
      // when the off-norm stalls, when a block is singular in FP32, or when only the sweeps the
      // polish needs are left.
      const bool stalled = hrec.max_scaled < 1e-3 && hrec.max_scaled > 0.5 * prev_max;
      const bool done = hrec.pivots_rotated == 0 || hrec.max_scaled < 1e-2 || stalled || lowp_singular ||
                        sw + 4 >= o.max_sweeps;
      prev_max = hrec.max_scaled;
      if (done) {
        // V (FP32) -> FP64, J-unitary by Newton-Schulz, then G = G_in V
        k_cvt32to64<<<ew_blocks, 256, 0, st>>>(P.np, n, hp.V32, P.np, hp.Vw, P.np);
        launches += 1;
        const dim3 gsym((n + 31) / 32, (n + 31) / 32, 1);
        for (int it = 0; it < 4 && status == JAC_OK; ++it) {
          if (split16)
            ck(oz_gemm_launch(n, n, n, hp.Vw, P.np, 1, hp.Vw, P.np, Jdev, L.Js, L.Mn, n, 1, 0, 0, 0, 0, 1, st)
                   ? cudaErrorLaunchFailure
                   : cudaSuccess);
          else
            k_gemm64<<<gsym, 128, 0, st>>>(n, n, n, hp.Vw, P.np, 1, hp.Vw, P.np, Jdev, L.Js, L.Mn, n, 1, 0, 0, 0, 0);
          ck(cudaMemsetAsync(L.mmax, 0, sizeof(unsigned long long), st));
          k_absmax64<<<std::min(1024, (n * n + 255) / 256), 256, 0, st>>>(n, L.Mn, n, L.mmax);
          unsigned long long hm = 0;
          ck(cudaMemcpyAsync(&hm, L.mmax, sizeof(hm), cudaMemcpyDeviceToHost, st));
          ck(cudaStreamSynchronize(st));
          launches += 2;
          double mm;
          std::memcpy(&mm, &hm, sizeof(mm));
          if (!(mm == mm) || mm > 0.25) {  // V32 too far from J-unitary to correct
            status = JAC_EINTERNAL;
            break;
          }
          if (mm <= 4e-16) break;
          // V <- V - V (J_c M) / 2, the correction in FP32
          k_cvt64to32<<<ew_blocks, 256, 0, st>>>(n, n, L.Mn, n, L.Mf, n, L.Js);
          k_cvt64to32<<<ew_blocks, 256, 0, st>>>(n, n, hp.Vw, P.np, L.Vf, n, nullptr);
          k_ns_correct<<<dim3((n + 63) / 64, (n + 63) / 64), 256, 0, st>>>(n, n, n, L.Vf, n, L.Mf, n, hp.Vw, P.np);
          launches += 3;
          ++ns_global;
          ck(cudaGetLastError());
          if (mm * mm + 1e-6 * mm <= 2e-16) break;
        }
        // G_int = G_in V (V rows are input columns): the FP64 factor the polish works on
        if (split16)
          ck(oz_gemm_launch(m, n, n, hio.G, ldg, 0, hp.Vw, P.np, nullptr, nullptr, hp.Gw, P.mp, 0, 0, 0, 0, 0, 1, st)
                 ? cudaErrorLaunchFailure
                 : cudaSuccess);
        else
          k_gemm64<<<dim3((m + 31) / 32, (n + 31) / 32, 1), 128, 0, st>>>(m, n, n, hio.G, ldg, 0, hp.Vw, P.np, nullptr,
                                                                          nullptr, hp.Gw, P.mp, 0, 0, 0, 0, 0);
        k_cache_init<<<1, 256, 0, st>>>(L.probs);  // G replaced: no earlier evaluation holds
        launches += 2;
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(st));
        phase = 3;
      }
      sweep_done();
      continue;
    }
    sweep_done();
    // converged: a sweep rotated nothing, or, from the second sweep of the phase on, its largest
    // scaled off-diagonal delta was so small that, by the quadratic convergence of the cyclic
    // method, the next sweep would rotate nothing (delta^2 <= 1e-6 tol: a margin of 10^6 on the
    // constant).  The first sweep of a phase does not qualify: its delta says nothing yet about
    // the rate.
    ++phase_sweeps;
    if (hrec.pivots_rotated == 0 ||
        (!strict_stop && phase_sweeps >= 2 && hrec.max_scaled * hrec.max_scaled <= 1e-6 * pp.tol)) {
      converged = 1;
      break;
    }
  }
  if (n == 1) converged = 1;
  if (status == JAC_OK && !converged) status = JAC_ENOTCONV;
  if (phase == 4 && (status == JAC_OK || status == JAC_ENOTCONV)) {
    k_lowp_copy<<<dim3(ew_blocks, 1), 256, 0, st>>>(L.probs, 1);  // FP32 result -> FP64 layout
    ++launches;
  }
  if (status == JAC_OK || status == JAC_ENOTCONV) {
    k_colnorm<<<dim3((n * 32 + 255) / 256, 1), 256, 0, st>>>(L.probs, L.io);
    k_rank<<<dim3((n + 255) / 256, 1), 256, sizeof(unsigned long long) * n, st>>>(L.probs, L.io);
    k_scatter<<<dim3(n, 1), 128, 0, st>>>(L.probs, L.io);
    launches += 3;
    if (cudaGetLastError() != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  }
  cudaFreeAsync(base, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  prof.finish();
  if (info) {
    for (int u = sweeps; u < 64; ++u) info->sweep_max_scaled[u] = 0.0;
    for (int u = 0; u < 64; ++u) info->sweep_ms[u] = (u < sweeps) ? sweep_ms_h[u] : 0.0;
    info->sweeps = sweeps;
    info->converged = converged;
    info->status = status;
    info->steps_per_sweep = last_steps;
    info->rotations = rot_total;
    info->pivots_rotated = piv_total;
    info->pivots_rotated_lowp = piv_lowp;
    info->pairs_evaluated = ev_total;
    info->pairs_evaluated_lowp = ev_lowp;
    info->max_scaled_off = hrec.max_scaled;
    info->off_rel = (hrec.trace > 0.0) ? std::sqrt(hrec.off2) / hrec.trace : 0.0;
    info->launches = launches;
    info->lowp_sweeps = lowp_sweeps;
    info->global_ns_steps = ns_global;
    info->pivot_ns_steps = ns_total;
    for (int u = 0; u < 4; ++u) info->pivot_cycles[u] = cyc_total[u];
    info->inner_sweeps = inner_total;
  }
  return status;
}

// ------------------------------------------------------------------ complex solve
// A complex problem is solved as the real problem of twice the order (complex.cu); the complex
// results are read off every other column of the ascending real result.
int solve_complex(int m, int n, void* Gv, int ldg, const int8_t* Jdev, const jac_opts* opts_in, double* lambda,
                  void* Uv, int ldu, void* Vv, int ldv, jac_info* info, cudaStream_t st, const ArgPos& ap) {
  jac_opts o;
  jacobi_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (info) std::memset(info, 0, sizeof(*info));
  auto fail_arg = [&](int pos) {
    if (info) info->status = -pos;
    return -pos;
  };
  if (m < 1) return fail_arg(ap.m);
  if (n < 1 || n > m || n > 10000) return fail_arg(ap.n);
  if (!Gv) return fail_arg(ap.G);
  if (ldg < m) return fail_arg(ap.ldg);
  if (ap.J && !Jdev) return fail_arg(ap.J);
  if (int r = check_opts(o, ap.opts, false)) return fail_arg(-r);
  if (o.ordering == JAC_ORDER_CYCLE_WEIGHT && compute_nb(2 * n, o.block_w) > JAC_CYCLE_WEIGHT_MAX_NB)
    return fail_arg(ap.opts);
  if (!lambda) return fail_arg(ap.lambda);
  if (Uv && ldu < m) return fail_arg(ap.ldu);
  if (Uv && Uv == Gv) return fail_arg(ap.U);
  if (o.want_v && !Vv) return fail_arg(ap.V);
  if (Vv && ldv < n) return fail_arg(ap.ldv);
  const bool want_v = o.want_v != 0;
  // the rotation threshold is that of the complex problem of order n (tol <= 0: n eps), not of
  // the real one of order 2n.  A complex entry g_i^* g_j has its real and imaginary parts in
  // two real Gram entries (columns [x_i; y_i] against [x_j; y_j] and [-y_j; x_j]), so the real
  // sweep uses tol / sqrt(2): every complex scaled off-diagonal entry then ends below tol
  if (o.tol <= 0.0)
    o.tol = (o.precision == JAC_PREC_FP32_ONLY) ? std::max((double)n, 8.0 * std::sqrt((double)m)) * 5.9604644775390625e-08
                                                : (double)n * 1.1102230246251565e-16;
  o.tol *= 0.70710678118654752;
  const size_t m2 = 2 * (size_t)m, n2 = 2 * (size_t)n;
  double *Gr = nullptr, *Gr2 = nullptr, *lam_r = nullptr, *Vr = nullptr, *Vr2 = nullptr;
  int8_t *Jr = nullptr, *Jr2 = nullptr;
  unsigned* bad = nullptr;
  auto carve = [&](Arena& A) {
    Jr2 = A.take<int8_t>(n2);
    Gr = A.take<double>(m2 * n2);
    Gr2 = A.take<double>(m2 * n2);
    lam_r = A.take<double>(n2);
    Vr = want_v ? A.take<double>(n2 * n2) : nullptr;
    Vr2 = want_v ? A.take<double>(n2 * n2) : nullptr;
    Jr = A.take<int8_t>(n2);
    bad = A.take<unsigned>(1);
  };
  Arena ar;
  carve(ar);
  void* base = nullptr;
  if (cudaMallocAsync(&base, ar.off, st) != cudaSuccess) {
    cudaGetLastError();
    if (info) info->status = JAC_ENOMEM;
    return JAC_ENOMEM;
  }
  Arena ar2;
  ar2.base = static_cast<char*>(base);
  carve(ar2);
  int status = JAC_OK;
  if (cudaMemsetAsync(bad, 0, sizeof(unsigned), st) != cudaSuccess) status = JAC_ECUDA;
  const int eb = (int)std::min<size_t>(4096, ((size_t)m * n + 255) / 256);
  k_realify<<<eb, 256, 0, st>>>(m, n, static_cast<const double2*>(Gv), ldg, Jdev, Gr, Jr);
  if (cudaGetLastError() != cudaSuccess) status = JAC_ECUDA;
  // pass 1: the sweep as requested
  if (status == JAC_OK)
    status = solve_real((int)m2, (int)n2, JAC_R64, Gr, (int)m2, Jr, &o, lam_r, nullptr, 0, Vr, (int)n2, info, st, ap);
  jac_info info1 = {};
  if (info) info1 = *info;
  double* Gres = Gr;
  double* Vres = Vr;
  // pass 2 (FP64, or FP32 for the FP32-only form): exact pairs from pass 1, started from its V
  if (status == JAC_OK) {
    const int eb2 = (int)std::min<size_t>(4096, (m2 * n + 255) / 256);
    k_restructure<<<eb2, 256, 0, st>>>(m, n, Gr, Gr2, lam_r, Jr2);  // signs of the output columns
    if (want_v)
      k_restructure<<<(int)std::min<size_t>(4096, (n2 * n + 255) / 256), 256, 0, st>>>(n, n, Vr, Vr2, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) status = JAC_ECUDA;
    jac_opts o2 = o;
    if (o2.precision == JAC_PREC_FP32) o2.precision = JAC_PREC_FP64;
    if (status == JAC_OK)
      status = solve_real((int)m2, (int)n2, JAC_R64, Gr2, (int)m2, Jr2, &o2, lam_r, nullptr, 0, Vr, (int)n2, info, st, ap,
                          want_v ? Vr2 : nullptr, /*strict_stop=*/true);
    if (info) {  // totals over both passes; the per-sweep maxima of pass 1, then of pass 2
      double merged[64], merged_ms[64];
      int t = 0;
      for (int u = 0; u < info1.sweeps && u < 64 && t < 64; ++u, ++t) {
        merged[t] = info1.sweep_max_scaled[u];
        merged_ms[t] = info1.sweep_ms[u];
      }
      for (int u = 0; u < info->sweeps && u < 64 && t < 64; ++u, ++t) {
        merged[t] = info->sweep_max_scaled[u];
        merged_ms[t] = info->sweep_ms[u];
      }
      for (; t < 64; ++t) merged[t] = merged_ms[t] = 0.0;
      for (int u = 0; u < 64; ++u) {
        info->sweep_max_scaled[u] = merged[u];
        info->sweep_ms[u] = merged_ms[u];
      }
      info->sweeps += info1.sweeps;
      info->rotations += info1.rotations;
      info->pivots_rotated += info1.pivots_rotated;
      info->pivots_rotated_lowp += info1.pivots_rotated_lowp;
      info->pairs_evaluated += info1.pairs_evaluated;
      info->pairs_evaluated_lowp += info1.pairs_evaluated_lowp;
      info->launches += info1.launches + 2;
      info->lowp_sweeps += info1.lowp_sweeps;
      info->global_ns_steps += info1.global_ns_steps;
      info->pivot_ns_steps += info1.pivot_ns_steps;
      info->inner_sweeps += info1.inner_sweeps;
      for (int u = 0; u < 4; ++u) info->pivot_cycles[u] += info1.pivot_cycles[u];
    }
    Gres = Gr2;
  }
  if (status == JAC_OK || status == JAC_ENOTCONV) {
    k_complexify<<<dim3((m + 127) / 128, n), 128, 0, st>>>(m, n, Gres, lam_r, Vres, static_cast<double2*>(Gv), ldg,
                                                          lambda, static_cast<double2*>(Uv), ldu,
                                                          want_v ? static_cast<double2*>(Vv) : nullptr, ldv, bad);
    unsigned hbad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      status = JAC_ECUDA;
    cudaFreeAsync(base, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) status = JAC_ECUDA;
    if (status == JAC_OK && hbad) status = JAC_EINTERNAL;
    if (info) {
      info->status = status;
      info->launches += 1;
    }
    return status;
  }
  cudaFreeAsync(base, st);
  cudaStreamSynchronize(st);
  return status;
}

int solve(int m, int n, int dtype, void* Gv, int ldg, const int8_t* Jdev, const jac_opts* opts_in, double* lambda,
          void* Uv, int ldu, void* Vv, int ldv, jac_info* info, cudaStream_t st, const ArgPos& ap) {
  if (dtype == JAC_C128) return solve_complex(m, n, Gv, ldg, Jdev, opts_in, lambda, Uv, ldu, Vv, ldv, info, st, ap);
  return solve_real(m, n, dtype, Gv, ldg, Jdev, opts_in, lambda, Uv, ldu, Vv, ldv, info, st, ap);
}

// ------------------------------------------------------------------ batched solve
// Problems are grouped by pivot class (KM = 32 or 64), largest order first inside a class; all
// problems advance sweep by sweep in the same launches, and converged ones drop out (active = 0)
// in the sweep reduction.
constexpr int kBatchChunk = 32768;  // grid y / z extents stay below 65536

int solve_batched(int batch, const int* m, const int* n, int dtype, void* const* G, const int* ldg,
                  const int8_t* const* J, const jac_opts* opts_in, double* const* lambda, void* const* U,
                  const int* ldu, void* const* V, const int* ldv, jac_info* info, cudaStream_t st) {
  if (batch > kBatchChunk) {  // consecutive chunks; the first failing status in input order wins
    int first = JAC_OK;
    for (int b0 = 0; b0 < batch; b0 += kBatchChunk) {
      const int c = std::min(kBatchChunk, batch - b0);
      auto off = [&](auto* p) { return p ? p + b0 : p; };
      const int r = solve_batched(c, off(m), off(n), dtype, off(G), off(ldg), off(J), opts_in, off(lambda), off(U),
                                  off(ldu), off(V), off(ldv), off(info), st);
      if (r < 0) return r;  // argument errors are found in the first chunk that has them
      if (r == JAC_ECUDA || r == JAC_ENOMEM) return r;
      if (first == JAC_OK) first = r;
    }
    return first;
  }
  jac_opts o;
  jacobi_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (batch < 0) return -1;
  if (batch == 0) return JAC_OK;
  if (!m) return -2;
  if (!n) return -3;
  if (dtype != JAC_R64) return -4;
  if (!G || !ldg) return !G ? -5 : -6;
  if (int r = check_opts(o, 8, true)) return r;
  if (!lambda) return -9;
  if (U && !ldu) return -11;
  if (o.want_v && (!V || !ldv)) return !V ? -12 : -13;
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1) return -2;
    if (n[b] < 1 || n[b] > m[b] || n[b] > 20000) return -3;
    if (!G[b]) return -5;
    if (ldg[b] < m[b]) return -6;
    if (!lambda[b]) return -9;
    if (U && U[b] && ldu[b] < m[b]) return -11;
    if (U && U[b] == G[b]) return -10;
    if (o.want_v && !V[b]) return -12;
    if (o.want_v && ldv[b] < n[b]) return -13;
  }
  if (info) std::memset(info, 0, sizeof(jac_info) * (size_t)batch);
  const bool fp32_only = (o.precision == JAC_PREC_FP32_ONLY);
  const bool want_v = o.want_v != 0;
  const bool have_vw = want_v;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JAC_ECUDA;
  if (int r = setup_attributes(dev)) return r;

  std::vector<Plan> plans(batch);
  for (int b = 0; b < batch; ++b) make_plan(plans[b], m[b], n[b], batch_width(n[b]), o.ordering, want_v, have_vw,
                                            fp32_only);
  // class order: KM 32 then 64; largest n first inside a class
  std::vector<int> order(batch);
  for (int b = 0; b < batch; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (plans[x].km != plans[y].km) return plans[x].km < plans[y].km;
    return plans[x].n > plans[y].n;
  });
  const int count32 = (int)std::count_if(plans.begin(), plans.end(), [](const Plan& p) { return p.km == 32; });
  const int count64 = batch - count32;
  std::map<int, std::pair<int*, int*>> tables;  // nb -> (pairs, counts)
  for (auto& p : plans) tables[p.nb] = {nullptr, nullptr};

  std::vector<JacProb> hp(batch);
  std::vector<JacIO> hio(batch);
  std::vector<long long> jsoff(batch);
  std::vector<int> boff_host;  // block offsets of every problem, concatenated
  std::vector<size_t> boff_at(batch);
  long long nsum = 0;
  for (int i = 0; i < batch; ++i) {
    jsoff[i] = nsum;
    nsum += plans[order[i]].n;
    boff_at[i] = boff_host.size();
    boff_host.insert(boff_host.end(), plans[order[i]].boff.begin(), plans[order[i]].boff.end());
  }
  int* d_boff = nullptr;
  JacProb* d_probs = nullptr;
  JacIO* d_io = nullptr;
  SweepRecord* d_rec = nullptr;
  unsigned* d_flags = nullptr;
  int8_t* d_Js = nullptr;
  long long* d_jsoff = nullptr;
  int* d_remaining = nullptr;
  auto carve_all = [&](Arena& A) {
    for (int i = 0; i < batch; ++i) carve_problem(A, plans[order[i]], hp[i], hio[i], false);
    d_boff = A.take<int>(boff_host.size());
    for (auto& kv : tables) {
      const int nb = kv.first;
      const int steps = (o.ordering == JAC_ORDER_ROUND_ROBIN) ? nb - 1 : nb;
      kv.second.first = A.take<int>((size_t)steps * (nb / 2) * 2);
      kv.second.second = A.take<int>(steps);
    }
    d_probs = A.take<JacProb>(batch);
    d_io = A.take<JacIO>(batch);
    d_rec = A.take<SweepRecord>(batch);
    d_flags = A.take<unsigned>(batch);
    d_Js = A.take<int8_t>(nsum);
    d_jsoff = A.take<long long>(batch);
    d_remaining = A.take<int>(1);
  };
  Arena ar;
  carve_all(ar);
  void* base = nullptr;
  if (cudaMallocAsync(&base, ar.off, st) != cudaSuccess) {
    cudaGetLastError();
    return JAC_ENOMEM;
  }
  Arena ar2;
  ar2.base = static_cast<char*>(base);
  carve_all(ar2);
  std::vector<int> boff_all;
  std::vector<std::pair<int*, size_t>> boff_pieces;
  for (int i = 0; i < batch; ++i) {
    const int b = order[i];
    const Plan& P = plans[b];
    hp[i].boff = d_boff + boff_at[i];
    hp[i].tol = (o.tol > 0.0) ? o.tol
                              : std::max((double)P.n, (fp32_only ? 8.0 : 0.0) * std::sqrt((double)P.mp)) *
                                    (fp32_only ? 5.9604644775390625e-08 : 1.1102230246251565e-16);
    hp[i].Js = d_Js + jsoff[i];
    hp[i].pairs = tables[P.nb].first;
    hp[i].counts = tables[P.nb].second;
    hp[i].pflags = d_flags + i;
    hio[i].G = static_cast<double*>(G[b]);
    hio[i].ldg = ldg[b];
    hio[i].J = J ? J[b] : nullptr;
    hio[i].lambda = lambda[b];
    hio[i].U = U ? static_cast<double*>(U[b]) : nullptr;
    hio[i].ldu = U ? ldu[b] : 0;
    hio[i].V = want_v ? static_cast<double*>(V[b]) : nullptr;
    hio[i].ldv = want_v ? ldv[b] : 0;
  }
  int status = JAC_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  };
  ck(cudaMemcpyAsync(d_boff, boff_host.data(), sizeof(int) * boff_host.size(), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(d_probs, hp.data(), sizeof(JacProb) * batch, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(d_io, hio.data(), sizeof(JacIO) * batch, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(d_jsoff, jsoff.data(), sizeof(long long) * batch, cudaMemcpyHostToDevice, st));
  ck(cudaMemsetAsync(d_flags, 0, sizeof(unsigned) * batch, st));
  for (auto& kv : tables) {
    const int nb = kv.first;
    const int steps = (o.ordering == JAC_ORDER_ROUND_ROBIN) ? nb - 1 : nb;
    k_sched_static<<<steps, 128, 0, st>>>(nb, o.ordering, steps, kv.second.first, kv.second.second);
  }
  int max_mp = 0, max_np = 0, max_n = 0;
  for (auto& p : plans) {
    max_mp = std::max(max_mp, p.mp);
    max_np = std::max(max_np, p.np);
    max_n = std::max(max_n, p.n);
  }
  k_sort_signs<<<batch, 32, 0, st>>>(d_probs, d_io, d_Js, d_jsoff);
  k_check_finite<<<dim3(8, batch), 256, 0, st>>>(d_probs, d_io);
  k_apply_flags<<<(batch + 255) / 256, 256, 0, st>>>(d_probs, d_io, batch);
  k_gather_in<<<dim3((max_mp + 255) / 256, max_n, batch), 256, 0, st>>>(d_probs, d_io);
  if (have_vw) k_init_v<<<dim3((max_np + 255) / 256, max_n, batch), 256, 0, st>>>(d_probs, d_io);
  k_cache_init<<<batch, 256, 0, st>>>(d_probs);
  if (fp32_only) k_lowp_copy<<<dim3(8, batch), 256, 0, st>>>(d_probs, 0);
  ck(cudaGetLastError());

  struct Cls {
    JacProb* probs;
    JacIO* io;
    SweepRecord* rec;
    int count, km, max_half, max_steps, gslabs, tslabs, max_mp;
  };
  std::vector<Cls> cls;
  auto add_cls = [&](int first, int count, int km) {
    if (count <= 0) return;
    Cls c{d_probs + first, d_io + first, d_rec + first, count, km, 0, 0, 0, 0, 0};
    for (int i = first; i < first + count; ++i) {
      const Plan& P = plans[order[i]];
      c.max_mp = std::max(c.max_mp, P.mp);
      c.max_half = std::max(c.max_half, P.half);
      c.max_steps = std::max(c.max_steps, P.nsteps);
      c.gslabs = std::max(c.gslabs, (P.mp + 63) / 64);
      c.tslabs = std::max(c.tslabs, (P.mp + 63) / 64 + (have_vw ? (P.np + 63) / 64 : 0));
    }
    cls.push_back(c);
  };
  add_cls(0, count32, 32);
  add_cls(count32, count64, 64);
  PivotParams pp;
  pp.tol = o.tol;  // <= 0: n eps of each problem
  pp.tol_eps = fp32_only ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  pp.tol_m = fp32_only ? 8.0 : 0.0;
  pp.factor = o.factor;
  pp.ns_mode = fp32_only ? 0 : 1;
  pp.oriented = (o.block_mode == JAC_BLOCK_ORIENTED) ? 1 : 0;
  pp.oz = (o.f64_products == JAC_F64_SPLIT16) ? 1 : (o.f64_products == JAC_F64_SPLIT16_TC ? 2 : 0);
  ProfRun prof;
  prof.begin();
  long long launches = 0;
  int sweeps = 0;
  SweepGraph graph;  // every sweep of a batch has the same launches
  bool use_graph = true;
  for (int sw = 0; status == JAC_OK && sw < o.max_sweeps; ++sw) {
    auto record = [&](cudaStream_t ss, long long& nl, ProfRun& pr) -> int {
      if (cudaMemsetAsync(d_remaining, 0, sizeof(int), ss) != cudaSuccess) return JAC_ECUDA;
      for (auto& c : cls) {
        for (int s = 0; s < c.max_steps; ++s)
          if (int r = launch_step(c.probs, c.count, c.km, c.max_half, c.gslabs, c.tslabs, 1, 1, s, fp32_only, true, pp,
                                  ss, pr, nl, nullptr, nullptr,
                                  o.fused_step == 1 && c.max_mp <= fused_step_max_rows(c.km)))
            return r;
        k_cache_step<<<c.count, 256, 0, ss>>>(c.probs, -2, -1);  // record the last step of the sweep
        k_sweep_reduce<<<c.count, 256, 0, ss>>>(c.probs, c.io, c.rec, 1, d_remaining);
        nl += 2;
      }
      return cudaGetLastError() == cudaSuccess ? 0 : JAC_ECUDA;
    };
    if (use_graph && !graph.exec) {
      graph.prof.begin();
      if (graph.build([&](cudaStream_t ss, long long& nl) { return record(ss, nl, graph.prof); })) {
        graph.prof.release();
        use_graph = false;
      }
    }
    bool replayed = false;
    if (use_graph && graph.exec) {
      if (cudaGraphLaunch(graph.exec, st) != cudaSuccess) status = JAC_ECUDA;
      launches += graph.launches;
      replayed = true;
    } else if (int r = record(st, launches, prof)) {
      status = r;
    }
    int remaining = 0;
    ck(cudaMemcpyAsync(&remaining, d_remaining, sizeof(int), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (replayed) graph.prof.accumulate();
    ++sweeps;
    if (remaining == 0) break;
  }
  if (fp32_only) k_lowp_copy<<<dim3(8, batch), 256, 0, st>>>(d_probs, 1);
  for (auto& c : cls) {
    int nmax = 0;
    for (int i = (int)(c.probs - d_probs); i < (int)(c.probs - d_probs) + c.count; ++i)
      nmax = std::max(nmax, plans[order[i]].n);
    k_colnorm<<<dim3((nmax * 32 + 255) / 256, c.count), 256, 0, st>>>(c.probs, c.io);
    k_rank<<<dim3((nmax + 255) / 256, c.count), 256, sizeof(unsigned long long) * nmax, st>>>(c.probs, c.io);
    k_scatter<<<dim3(nmax, c.count), 128, 0, st>>>(c.probs, c.io);
    launches += 3;
  }
  ck(cudaGetLastError());
  std::vector<JacProb> hp_back(batch);
  std::vector<JacIO> hio_back(batch);
  std::vector<unsigned> flags_back(batch);
  ck(cudaMemcpyAsync(hp_back.data(), d_probs, sizeof(JacProb) * batch, cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(hio_back.data(), d_io, sizeof(JacIO) * batch, cudaMemcpyDeviceToHost, st));
  ck(cudaMemcpyAsync(flags_back.data(), d_flags, sizeof(unsigned) * batch, cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(base, st);
  ck(cudaStreamSynchronize(st));
  prof.finish();
  int first_bad = JAC_OK;
  for (int i = 0; i < batch; ++i) {
    const int b = order[i];
    int s = JAC_OK;
    if (hio_back[i].flags & 2) s = -7;
    else if (hio_back[i].flags & 1) s = JAC_ENONFINITE;
    else if (flags_back[i] & JAC_DEVERR_TIMEOUT) s = JAC_EINTERNAL;
    else if (flags_back[i] & JAC_DEVERR_NOTPD) s = JAC_ENOTPD;
    else if (hp_back[i].active) s = JAC_ENOTCONV;
    if (status != JAC_OK) s = status;
    if (info) {
      info[b].status = s;
      info[b].converged = (s == JAC_OK) ? 1 : 0;
      info[b].sweeps = hio_back[i].sweeps;
      info[b].rotations = hio_back[i].rotations;
      info[b].steps_per_sweep = plans[b].nsteps;
      info[b].launches = (b == 0) ? launches : 0;
    }
    if (s != JAC_OK && first_bad == JAC_OK) first_bad = s;
  }
  (void)sweeps;
  return status != JAC_OK ? status : first_bad;
}

}  // namespace

extern "C" {

void jacobi_default_opts(jac_opts* o) {
  if (!o) return;
  o->block_w = 32;
  o->ordering = JAC_ORDER_ROUND_ROBIN;
  o->block_mode = JAC_BLOCK_FULL;
  o->factor = JAC_FACTOR_CHOL_SIGNPIV;
  o->precision = JAC_PREC_FP64;
  o->max_sweeps = 50;
  o->want_v = 1;
  o->tol = 0.0;
  o->f64_products = JAC_F64_SPLIT16;
  o->fused_step = 1;
}

const char* jacobi_status_string(int s) {
  if (s < 0) return "invalid argument";
  switch (s) {
    case JAC_OK: return "ok";
    case JAC_ENOTCONV: return "not converged within max_sweeps";
    case JAC_ENOTPD: return "pivot block not positive definite (G lacks full column rank)";
    case JAC_ENONFINITE: return "non-finite entry in G";
    case JAC_ECUDA: return "CUDA runtime error";
    case JAC_ENOMEM: return "device scratch allocation failed";
    case JAC_EINTERNAL: return "internal limit reached";
    default: return "unknown status";
  }
}

int jacobi_version(void) { return JAC_VERSION; }

int jacobi_profile_begin(int mask) {
  if (mask < 0 || mask >= (1 << JAC_KERNEL_COUNT)) return -1;
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  g_prof_mask = mask;
  for (int k = 0; k < JAC_KERNEL_COUNT; ++k) {
    g_prof_ms[k] = 0.0;
    g_prof_n[k] = 0;
  }
  return 0;
}

int jacobi_profile_read(int kernel, double* total_ms, long long* launches) {
  if (kernel < 0 || kernel >= JAC_KERNEL_COUNT) return -1;
  if (!total_ms) return -2;
  if (!launches) return -3;
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  *total_ms = g_prof_ms[kernel];
  *launches = g_prof_n[kernel];
  return 0;
}

int jacobi_profile_end(void) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  g_prof_mask = 0;
  for (auto e : g_prof_pool) cudaEventDestroy(e);
  g_prof_pool.clear();
  return 0;
}

int jacobi_hsvd(int m, int n, int dtype, void* G, int ldg, const int8_t* J, const jac_opts* opts, double* lambda,
                void* U, int ldu, void* V, int ldv, jac_info* info, jac_stream_t stream) {
  const ArgPos ap = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12};
  return solve(m, n, dtype, G, ldg, J, opts, lambda, U, ldu, V, ldv, info, (cudaStream_t)stream, ap);
}

int jacobi_eig_pd(int m, int n, int dtype, void* G, int ldg, const jac_opts* opts, double* lambda, void* U,
                  int ldu, void* V, int ldv, jac_info* info, jac_stream_t stream) {
  const ArgPos ap = {1, 2, 3, 4, 5, 0, 6, 7, 8, 9, 10, 11};
  return solve(m, n, dtype, G, ldg, nullptr, opts, lambda, U, ldu, V, ldv, info, (cudaStream_t)stream, ap);
}

int jacobi_eig_batched(int batch, const int* m, const int* n, int dtype, void* const* G, const int* ldg,
                       const int8_t* const* J, const jac_opts* opts, double* const* lambda, void* const* U,
                       const int* ldu, void* const* V, const int* ldv, jac_info* info, jac_stream_t stream) {
  return solve_batched(batch, m, n, dtype, G, ldg, J, opts, lambda, U, ldu, V, ldv, info, (cudaStream_t)stream);
}

int jacobi_autotune_batched(int count, int precision, int* rules, jac_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return JAC_ECUDA;
  if (count == 0) {  // back to the default widths on this device
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    if (g_tune_init)
      for (int n = 0; n <= 128; ++n) g_tuned_rule[dev][n] = -1;
    if (rules)
      for (int n = 0; n <= 128; ++n) rules[n] = -1;
    return JAC_OK;
  }
  if (count < 1 || count > 4096) return -1;
  if (precision != JAC_PREC_FP64 && precision != JAC_PREC_FP32_ONLY) return -2;
  // size classes and the width rules tried in each (rule 0: one pivot block); the first rule of
  // a class is its default (batch_width)
  struct Cls {
    int lo, hi;
    int rules[3];
  };
  const Cls classes[] = {{8, 16, {0, 8, -1}},      {17, 32, {0, 8, -1}},      {33, 48, {0, 16, 8}},
                         {49, 64, {0, 16, 32}},    {65, 96, {32, 16, -1}},    {97, 128, {32, 16, -1}}};
  int best_rule[129];
  for (int n = 0; n <= 128; ++n) best_rule[n] = -1;
  for (const Cls& c : classes)
    for (int n = c.lo; n <= c.hi; ++n) best_rule[n] = c.rules[0];
  jac_opts o;
  jacobi_default_opts(&o);
  o.precision = precision;
  o.want_v = 1;
  // one batch drawn like the batched workload: orders spread evenly over 8..128 (every class
  // present, sharing launches as in a real batch), square, Gaussian entries, round(0.3 n) signs
  // -1 at random positions of each problem
  std::vector<int> ms(count), ns(count), ld(count);
  std::vector<long long> offs(count + 1), joffs(count + 1);
  offs[0] = joffs[0] = 0;
  for (int b = 0; b < count; ++b) {
    ns[b] = ms[b] = ld[b] = 8 + (int)(((long long)b * 121) / count);
    offs[b + 1] = offs[b] + (long long)ns[b] * ns[b];
    joffs[b + 1] = joffs[b] + ns[b];
  }
  std::vector<int8_t> hJ((size_t)joffs[count], 1);
  {
    std::vector<int> idx;
    unsigned long long lcg = 0x5EED5EEDull;
    for (int b = 0; b < count; ++b) {  // partial Fisher-Yates shuffle of each problem's positions
      idx.resize(ns[b]);
      for (int i = 0; i < ns[b]; ++i) idx[i] = i;
      const int neg = (int)std::lround(0.3 * ns[b]);
      for (int i = 0; i < neg; ++i) {
        lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
        const int jx = i + (int)((lcg >> 33) % (unsigned long long)(ns[b] - i));
        std::swap(idx[i], idx[jx]);
        hJ[(size_t)(joffs[b] + idx[i])] = -1;
      }
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return JAC_ECUDA;
  int status = JAC_OK;
  void* base = nullptr;
  const size_t bytes = sizeof(double) * (3 * (size_t)offs[count] + (size_t)joffs[count]) + (size_t)joffs[count] + 256;
  if (cudaMallocAsync(&base, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return JAC_ENOMEM;
  }
  double* G0 = static_cast<double*>(base);
  double* Gw = G0 + offs[count];
  double* Vb = Gw + offs[count];
  double* lam = Vb + offs[count];
  int8_t* Jb = reinterpret_cast<int8_t*>(lam + joffs[count]);
  k_fill_gauss<<<1024, 256, 0, st>>>(G0, offs[count], 0x5EED5EEDull);
  cudaMemcpyAsync(Jb, hJ.data(), hJ.size(), cudaMemcpyHostToDevice, st);
  std::vector<void*> pG(count), pV(count);
  std::vector<double*> pl(count);
  std::vector<const int8_t*> pJ(count);
  for (int b = 0; b < count; ++b) {
    pG[b] = Gw + offs[b];
    pV[b] = Vb + offs[b];
    pl[b] = lam + joffs[b];
    pJ[b] = Jb + joffs[b];
  }
  // time of the whole batch under the given rules: best of two runs after a warm-up
  auto time_rules = [&](const int* rule) -> float {
    {
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      if (!g_tune_init) {
        for (int d = 0; d < 64; ++d)
          for (int n = 0; n <= 128; ++n) g_tuned_rule[d][n] = -1;
        g_tune_init = true;
      }
      for (int n = 0; n <= 128; ++n) g_tuned_rule[dev][n] = rule[n];
    }
    float t = 1e30f;
    for (int rep = 0; rep < 3 && status == JAC_OK; ++rep) {
      cudaMemcpyAsync(Gw, G0, sizeof(double) * offs[count], cudaMemcpyDeviceToDevice, st);
      cudaEventRecord(e0, st);
      const int rc = solve_batched(count, ms.data(), ns.data(), JAC_R64, pG.data(), ld.data(), pJ.data(), &o,
                                   pl.data(), nullptr, nullptr, pV.data(), ld.data(), nullptr, st);
      cudaEventRecord(e1, st);
      if (rc < 0 || rc == JAC_ECUDA || rc == JAC_ENOMEM) status = (rc < 0) ? JAC_EINTERNAL : rc;
      if (cudaEventSynchronize(e1) != cudaSuccess) status = JAC_ECUDA;
      float tr = 0.0f;
      cudaEventElapsedTime(&tr, e0, e1);
      if (rep > 0) t = std::min(t, tr);
    }
    return t;
  };
  // coordinate descent over the classes: a candidate replaces a class's current rule only when
  // the whole batch runs at least 3% faster with it (above run-to-run noise)
  float best_ms = time_rules(best_rule);
  for (const Cls& c : classes) {
    if (status != JAC_OK) break;
    for (int ri = 1; ri < 3 && status == JAC_OK; ++ri) {
      const int r = c.rules[ri];
      if (r < 0 || (r == 0 && c.hi > 64)) continue;
      int trial[129];
      for (int n = 0; n <= 128; ++n) trial[n] = best_rule[n];
      for (int n = c.lo; n <= c.hi; ++n) trial[n] = r;
      const float t = time_rules(trial);
      if (status == JAC_OK && t < 0.97f * best_ms) {
        best_ms = t;
        for (int n = c.lo; n <= c.hi; ++n) best_rule[n] = r;
      }
    }
  }
  cudaFreeAsync(base, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (int n = 0; n <= 128; ++n) g_tuned_rule[dev][n] = (status == JAC_OK) ? best_rule[n] : -1;
  }
  if (rules)
    for (int n = 0; n <= 128; ++n) rules[n] = (status == JAC_OK) ? best_rule[n] : -1;
  return status;
}

int jacobi_sched_pairs(int nb, int ordering, const double* weights, int* pairs, int* counts, int max_steps,
                       int* nsteps, jac_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nb < 2 || nb > 4096 || (nb & 1)) return -1;
  if (ordering == JAC_ORDER_CYCLE_WEIGHT && nb > JAC_CYCLE_WEIGHT_MAX_NB) return -1;
  if (ordering < 0 || ordering > 3) return -2;
  if (ordering == JAC_ORDER_CYCLE_WEIGHT && !weights) return -3;
  if (!pairs) return -4;
  if (!counts) return -5;
  const int need = (ordering == JAC_ORDER_ROUND_ROBIN) ? nb - 1 : (ordering == JAC_ORDER_CYCLE_WEIGHT ? 1 : nb);
  if (max_steps < need) return -6;
  if (!nsteps) return -7;
  if (ordering != JAC_ORDER_CYCLE_WEIGHT) {
    k_sched_static<<<need, 128, 0, st>>>(nb, ordering, need, pairs, counts);
    if (cudaGetLastError() != cudaSuccess) return JAC_ECUDA;
    *nsteps = need;
    return cudaStreamSynchronize(st) == cudaSuccess ? JAC_OK : JAC_ECUDA;
  }
  const int npairs = nb * (nb - 1) / 2;
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, sizeof(int) * (npairs + 1), st) != cudaSuccess) return JAC_ENOMEM;
  int* order = static_cast<int*>(scratch);
  int* dn = order + npairs;
  k_sched_rank<<<(npairs + 255) / 256, 256, sizeof(double) * nb, st>>>(nb, weights, order);
  k_sched_cycle_weight<<<1, 1024, sizeof(int) * nb, st>>>(nb, order, pairs, counts, max_steps, dn);
  int status = (cudaGetLastError() == cudaSuccess) ? JAC_OK : JAC_ECUDA;
  int h = -1;
  if (cudaMemcpyAsync(&h, dn, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) status = JAC_ECUDA;
  cudaFreeAsync(scratch, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) status = JAC_ECUDA;
  if (status == JAC_OK && h < 0) status = JAC_EINTERNAL;
  *nsteps = h;
  return status;
}

}  // extern "C"
