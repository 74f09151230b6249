// capi.cu -- host driver of the sweep loop and the C ABI declared in include/jacobi_gb300.h.
//
// The driver does no numerics on the host: it validates arguments, sorts J into
// diag(I, -I) (Algorithms 3.2 / 3.4 assume that order), lays out the block partition
// (Sec. 3: widths differ by at most one), launches the device scheduler, and then per sweep
// the step kernels gram -> pivot -> update for every step, followed by the sweep reduction,
// whose small record is the only value read back per sweep.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "jacobi_common.cuh"
#include "jacobi_gb300.h"

namespace jac {
__global__ void k_sched_static(int nb, int ordering, int nsteps, int* pairs, int* counts);
__global__ void k_sched_cycle_weight(int nb, const double* w, int* order_g, int* pairs, int* counts, int max_steps,
                                     int* nsteps_out);
__global__ void k_block_weights32(const float* G32, int mp, int nb, const int* boff, double* w);
__global__ void k_gram32(JacStepArgs a, const float* G32, const int* step_pairs, const int* step_count, int CS,
                         double* Ap);
__global__ void k_update32(JacStepArgs a, float* G32, float* V32, const int* step_pairs, const int* step_count,
                           const double* vp, const int* skip, int gslabs);
__global__ void k_gemm64(int Mr, int Nc, int K, const double* A, int lda, int transA, const double* B, int ldb,
                         const int8_t* sb, const int8_t* dsub, double* C, int ldc, int sym);
__global__ void k_ns_correct(int Mr, int Nc, int K, const float* Af, int lda, const float* Bf, int ldb, double* V,
                             int ldv);
__global__ void k_cvt64to32(int rows, int cols, const double* src, int lds, float* dst, int ldd, const int8_t* rsign);
__global__ void k_cvt32to64(int rows, int cols, const float* src, int lds, double* dst, int ldd);
__global__ void k_absmax64(int n, const double* M, int ldm, unsigned long long* out);
__global__ void k_gram(JacStepArgs a, const int* step_pairs, const int* step_count, int CS, double* Ap);
__global__ void k_update(JacStepArgs a, const int* step_pairs, const int* step_count, const double* vp,
                         const int* skip, int gslabs);
__global__ void k_pivot(JacStepArgs a, const int* step_pairs, const int* step_count, const double* Ap,
                        PivotParams pp, double* vp, int* skip, PairStat* stats, unsigned* err);
__global__ void k_sweep_reduce(const PairStat* stats, const int* counts, int nsteps, int half, int nb,
                               const unsigned* err, SweepRecord* rec);
__global__ void k_gather_in(const double* G, int ldg, int m, int mp, const int* perm_in, double* Gw);
__global__ void k_init_v(int n, int np, const int* perm_in, double* Vw);
__global__ void k_check_finite(const double* G, int ldg, int m, int n, unsigned* err);
__global__ void k_colnorm(const double* Gw, int mp, int n, const int8_t* Js, double* nrm2, double* lam);
__global__ void k_rank(const double* lam, int n, int* rank);
__global__ void k_scatter(const double* Gw, int mp, int m, const double* Vw, int np, int n, const double* nrm2,
                          const double* lam, const int* rank, double* lambda, double* G, int ldg, double* U,
                          int ldu, double* V, int ldv);
size_t pivot_smem_bytes();
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
  // record before / after one launch of kernel k
  size_t pre(int k, cudaStream_t st) {
    if (!(mask & (1 << k))) return (size_t)-1;
    cudaEvent_t a = take(), b = take();
    if (!a || !b) return (size_t)-1;
    evs.push_back(a);
    evs.push_back(b);
    cudaEventRecord(a, st);
    marks.emplace_back(k, evs.size() - 2);
    return evs.size() - 2;
  }
  void post(size_t idx, cudaStream_t st) {
    if (idx != (size_t)-1) cudaEventRecord(evs[idx + 1], st);
  }
  // after the stream has been synchronized
  void finish() {
    if (evs.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mutex);
    for (auto& mk : marks) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[mk.second], evs[mk.second + 1]) == cudaSuccess && g_prof_mask) {
        g_prof_ms[mk.first] += ms;
        g_prof_n[mk.first] += 1;
      }
    }
    for (auto e : evs) g_prof_pool.push_back(e);
    evs.clear();
    marks.clear();
  }
};

std::mutex g_attr_mutex;
bool g_attr_done[64] = {};

int setup_attributes(int dev) {
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  if (dev < 0 || dev >= 64) return JAC_ECUDA;
  if (g_attr_done[dev]) return 0;
  if (cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramSmem) != cudaSuccess)
    return JAC_ECUDA;
  if (cudaFuncSetAttribute(k_gram, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return JAC_ECUDA;
  if (cudaFuncSetAttribute(k_gram32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return JAC_ECUDA;
  if (cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem) != cudaSuccess)
    return JAC_ECUDA;
  if (cudaFuncSetAttribute(k_pivot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pivot_smem_bytes()) !=
      cudaSuccess)
    return JAC_ECUDA;
  if (cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) != cudaSuccess)
    return JAC_ECUDA;
  g_attr_done[dev] = true;
  return 0;
}

// Carves one cudaMallocAsync block into 256-byte aligned pieces.
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

struct Layout {
  double *Gw, *Vw, *Ap, *vp, *weights, *nrm2, *lam, *Mn;
  float *G32, *V32, *Mf, *Vf;
  int *boff, *perm_in, *pairs, *counts, *skip, *order, *nsteps, *rank;
  int8_t *Js, *Jin;
  PairStat* stats;
  SweepRecord* rec;
  unsigned* err;
  unsigned long long* mmax;
};

size_t carve(Arena& ar, Layout& L, int m, int mp, int np, int n, int nb, int max_steps, bool have_vw, bool weights,
             bool need_g32, bool mixed) {
  (void)m;
  const int half = nb / 2;
  const int npairs = nb * (nb - 1) / 2;
  L.Gw = ar.take<double>((size_t)mp * n);
  L.Vw = have_vw ? ar.take<double>((size_t)np * n) : nullptr;
  L.Ap = ar.take<double>((size_t)half * JAC_KMAX * JAC_KMAX);
  L.vp = ar.take<double>((size_t)half * JAC_KMAX * JAC_KMAX);
  L.weights = weights ? ar.take<double>((size_t)nb * nb) : nullptr;
  L.nrm2 = ar.take<double>(n);
  L.lam = ar.take<double>(n);
  L.Mn = mixed ? ar.take<double>((size_t)n * n) : nullptr;
  L.G32 = need_g32 ? ar.take<float>((size_t)mp * n) : nullptr;
  L.V32 = mixed ? ar.take<float>((size_t)np * n) : nullptr;
  L.Mf = mixed ? ar.take<float>((size_t)n * n) : nullptr;
  L.Vf = mixed ? ar.take<float>((size_t)n * n) : nullptr;
  L.boff = ar.take<int>(nb + 1);
  L.perm_in = ar.take<int>(n);
  L.pairs = ar.take<int>((size_t)max_steps * half * 2);
  L.counts = ar.take<int>(max_steps);
  L.skip = ar.take<int>(half);
  L.order = weights ? ar.take<int>(npairs) : nullptr;
  L.nsteps = ar.take<int>(1);
  L.rank = ar.take<int>(n);
  L.Js = ar.take<int8_t>(n);
  L.Jin = ar.take<int8_t>(n);
  L.stats = ar.take<PairStat>((size_t)max_steps * half);
  L.rec = ar.take<SweepRecord>(1);
  L.err = ar.take<unsigned>(1);
  L.mmax = ar.take<unsigned long long>(1);
  return ar.off;
}

int choose_cluster(int half, int mp) {
  int cs = 1;
  while (cs * 2 <= 16 && half * cs * 2 <= 2 * 152 && mp / (cs * 2) >= 16) cs *= 2;
  return cs;
}

template <class Kern, class... Args>
int launch_cluster(Kern kern, int half, int CS, int threads, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(half * CS);
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

// Validates the options; returns 0 or the (negative) argument position of opts.
int check_opts(const jac_opts& o, int argpos) {
  if (o.block_w < 1 || o.block_w > JAC_WMAX) return -argpos;
  if (o.ordering < 0 || o.ordering > 3) return -argpos;
  if (o.block_mode != JAC_BLOCK_FULL) return -argpos;
  if (o.factor != JAC_FACTOR_CHOL && o.factor != JAC_FACTOR_CHOL_SIGNPIV) return -argpos;
  if (o.precision != JAC_PREC_FP64 && o.precision != JAC_PREC_FP32) return -argpos;
  if (o.max_sweeps < 1) return -argpos;
  if (o.want_v != 0 && o.want_v != 1) return -argpos;
  return 0;
}

int compute_nb(int n, int w) {
  int nb = 2 * ((n + 2 * w - 1) / (2 * w));
  if (nb < 2) nb = 2;
  if (nb > n) nb = n & ~1;
  if (nb < 2) nb = 2;
  return nb;
}

struct ArgPos {  // 1-based positions of the arguments in the public signature
  int m, n, dtype, G, ldg, J, opts, lambda, U, ldu, V, ldv;
};

int solve(int m, int n, int dtype, void* Gv, int ldg, const int8_t* Jdev, const jac_opts* opts_in, double* lambda,
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
  if (n < 1 || n > m || n > 20000) return fail_arg(ap.n);
  if (dtype != JAC_R64) return fail_arg(ap.dtype);
  if (!Gv) return fail_arg(ap.G);
  if (ldg < m) return fail_arg(ap.ldg);
  if (ap.J && !Jdev) return fail_arg(ap.J);
  if (int r = check_opts(o, ap.opts)) return fail_arg(-r);
  if (!lambda) return fail_arg(ap.lambda);
  if (Uv && ldu < m) return fail_arg(ap.ldu);
  if (Uv && Uv == Gv) return fail_arg(ap.U);
  if (o.want_v && !Vv) return fail_arg(ap.V);
  if (Vv && ldv < n) return fail_arg(ap.ldv);
  if (o.tol <= 0.0) o.tol = (double)n * 1.1102230246251565e-16;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JAC_ECUDA;
  if (int r = setup_attributes(dev)) return r;

  // signs on the host (needed for the internal sort)
  std::vector<int8_t> Jh(n, 1);
  if (ap.J) {
    if (cudaMemcpyAsync(Jh.data(), Jdev, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) return JAC_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return JAC_ECUDA;
    for (int k = 0; k < n; ++k)
      if (Jh[k] != 1 && Jh[k] != -1) return fail_arg(ap.J);
  }
  std::vector<int> perm_in;
  perm_in.reserve(n);
  for (int k = 0; k < n; ++k)
    if (Jh[k] > 0) perm_in.push_back(k);
  for (int k = 0; k < n; ++k)
    if (Jh[k] < 0) perm_in.push_back(k);
  std::vector<int8_t> Js(n);
  for (int k = 0; k < n; ++k) Js[k] = Jh[perm_in[k]];

  const int mp = (m + 15) & ~15, np = (n + 15) & ~15;
  const int nb = compute_nb(n, o.block_w);
  const int half = nb / 2;
  std::vector<int> boff(nb + 1);
  {
    const int base = n / nb, rem = n % nb;
    int off = 0;
    for (int b = 0; b < nb; ++b) {
      boff[b] = off;
      off += base + (b < rem ? 1 : 0);
    }
    boff[nb] = off;
  }
  const bool weights = (o.ordering == JAC_ORDER_CYCLE_WEIGHT);
  const bool mixed = (o.precision == JAC_PREC_FP32);
  const int max_steps = (o.ordering == JAC_ORDER_ROUND_ROBIN) ? nb - 1 : (weights ? 2 * nb : nb);
  const bool want_v = o.want_v != 0;
  const bool have_vw = want_v || mixed;  // the mixed mode needs V internally for G = G_in V
  const bool need_g32 = mixed || weights;

  Arena ar;
  Layout L;
  const size_t bytes = carve(ar, L, m, mp, np, n, nb, max_steps, have_vw, weights, need_g32, mixed);
  void* base = nullptr;
  if (cudaMallocAsync(&base, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return JAC_ENOMEM;
  }
  Arena ar2;
  ar2.base = static_cast<char*>(base);
  carve(ar2, L, m, mp, np, n, nb, max_steps, have_vw, weights, need_g32, mixed);

  int status = JAC_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  };
  ck(cudaMemcpyAsync(L.boff, boff.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.perm_in, perm_in.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.Js, Js.data(), n, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(L.Jin, Jh.data(), n, cudaMemcpyHostToDevice, st));
  ck(cudaMemsetAsync(L.err, 0, sizeof(unsigned), st));

  long long launches = have_vw ? 3 : 2;
  const double* G = static_cast<const double*>(Gv);
  const int ew_blocks = std::min(1024, (int)(((size_t)mp * n + 255) / 256));
  k_check_finite<<<std::min(1024, (int)(((size_t)m * n + 255) / 256)), 256, 0, st>>>(G, ldg, m, n, L.err);
  k_gather_in<<<dim3((mp + 255) / 256, n), 256, 0, st>>>(G, ldg, m, mp, L.perm_in, L.Gw);
  if (have_vw) k_init_v<<<dim3((np + 255) / 256, n), 256, 0, st>>>(n, np, L.perm_in, L.Vw);
  ck(cudaGetLastError());
  unsigned herr = 0;
  ck(cudaMemcpyAsync(&herr, L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  if (status == JAC_OK && (herr & JAC_DEVERR_NONFINITE)) status = JAC_ENONFINITE;

  int nsteps = max_steps;
  if (status == JAC_OK && !weights) {
    k_sched_static<<<max_steps, 128, 0, st>>>(nb, o.ordering, max_steps, L.pairs, L.counts);
    ++launches;
    ck(cudaGetLastError());
  }

  JacStepArgs args;
  args.Gw = L.Gw;
  args.mp = mp;
  args.Vw = L.Vw;
  args.np = np;
  args.n = n;
  args.nb = nb;
  args.boff = L.boff;
  args.Js = L.Js;
  args.pairs = L.pairs;
  args.counts = L.counts;
  args.half = half;
  const int CS = choose_cluster(half, mp);
  const int gslabs = (mp + 63) / 64;
  const int vslabs = have_vw ? (np + 63) / 64 : 0;
  // FP32 phase: stop at the scaled off-norm the FP32 Gram still resolves (its entries carry
  // errors ~ eps_32 sqrt(m) relative to ||g_i|| ||g_j||)
  const double tau_lo = std::max(o.tol, 8.0 * 5.9604644775390625e-08 * std::sqrt((double)m));
  int phase = mixed ? 1 : 3;
  if (mixed && status == JAC_OK) {
    k_cvt64to32<<<ew_blocks, 256, 0, st>>>(mp, n, L.Gw, mp, L.G32, mp, nullptr);
    k_cvt64to32<<<ew_blocks, 256, 0, st>>>(np, n, L.Vw, np, L.V32, np, nullptr);
    launches += 2;
    ck(cudaGetLastError());
  }

  int sweeps = 0, converged = 0, lowp_sweeps = 0, ns_global = 0;
  long long rot_total = 0, piv_total = 0, cyc_total[4] = {0, 0, 0, 0}, ns_total = 0, inner_total = 0;
  double prev_max = 1e300;
  SweepRecord hrec = {};
  int last_steps = 0;
  ProfRun prof;
  prof.begin();
  for (int sw = 0; status == JAC_OK && n > 1 && sw < o.max_sweeps; ++sw) {
    const bool low = (phase == 1);
    PivotParams pp;
    pp.tol = low ? tau_lo : o.tol;
    pp.factor = o.factor;
    pp.ns_mode = low ? 0 : 1;
    if (weights) {
      const int npairs = nb * (nb - 1) / 2;
      if (!low) {
        k_cvt64to32<<<ew_blocks, 256, 0, st>>>(mp, n, L.Gw, mp, L.G32, mp, nullptr);
        ++launches;
      }
      k_block_weights32<<<npairs, 256, 0, st>>>(L.G32, mp, nb, L.boff, L.weights);
      k_sched_cycle_weight<<<1, 1024, sizeof(int) * nb, st>>>(nb, L.weights, L.order, L.pairs, L.counts,
                                                              max_steps, L.nsteps);
      launches += 2;
      ck(cudaGetLastError());
      ck(cudaMemcpyAsync(&nsteps, L.nsteps, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (status != JAC_OK) break;
      if (nsteps < 1 || nsteps > max_steps) {
        status = JAC_EINTERNAL;
        break;
      }
    }
    for (int s = 0; s < nsteps && status == JAC_OK; ++s) {
      const int* sp = L.pairs + (size_t)s * half * 2;
      const int* sc = L.counts + s;
      size_t pm = prof.pre(JAC_KERNEL_GRAM, st);
      if (low) {
        if (int r = launch_cluster(k_gram32, half, CS, 128, 0, st, args, (const float*)L.G32, sp, sc, CS, L.Ap))
          status = r;
      } else {
        if (int r = launch_cluster(k_gram, half, CS, 128, kGramSmem, st, args, sp, sc, CS, L.Ap)) status = r;
      }
      prof.post(pm, st);
      pm = prof.pre(JAC_KERNEL_PIVOT, st);
      k_pivot<<<half, 1024, pivot_smem_bytes(), st>>>(args, sp, sc, L.Ap, pp, L.vp, L.skip,
                                                      L.stats + (size_t)s * half, L.err);
      prof.post(pm, st);
      pm = prof.pre(JAC_KERNEL_UPDATE, st);
      if (low) {
        k_update32<<<dim3(half, gslabs + vslabs), 256, 0, st>>>(args, L.G32, L.V32, sp, sc, L.vp, L.skip, gslabs);
      } else {
        k_update<<<dim3(half, gslabs + vslabs), 128, kUpdSmem, st>>>(args, sp, sc, L.vp, L.skip, gslabs);
      }
      prof.post(pm, st);
      launches += 3;
      ck(cudaGetLastError());
    }
    k_sweep_reduce<<<1, 256, 0, st>>>(L.stats, L.counts, nsteps, half, nb, L.err, L.rec);
    ++launches;
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(&hrec, L.rec, sizeof(SweepRecord), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (status != JAC_OK) break;
    if (info && sweeps < 64) info->sweep_max_scaled[sweeps] = hrec.max_scaled;
    ++sweeps;
    last_steps = nsteps;
    rot_total += hrec.rotations;
    piv_total += hrec.pivots_rotated;
    ns_total += hrec.ns_steps;
    inner_total += hrec.inner_sweeps;
    for (int u = 0; u < 4; ++u) cyc_total[u] += hrec.cyc[u];
    if (hrec.err & JAC_DEVERR_NOTPD) {
      status = JAC_ENOTPD;
      break;
    }
    if (low) {
      ++lowp_sweeps;
      // leave the FP32 phase when it has converged at tau_lo, when the off-norm stalls, or
      // when only the sweeps the polish needs are left
      const bool stalled = hrec.max_scaled < 1e-3 && hrec.max_scaled > 0.5 * prev_max;
      const bool done = hrec.pivots_rotated == 0 || stalled || sw + 4 >= o.max_sweeps;
      prev_max = hrec.max_scaled;
      if (done) {
        // phase 2: V (FP32) -> FP64, J-unitary by Newton-Schulz, then G = G_in V
        k_cvt32to64<<<ew_blocks, 256, 0, st>>>(np, n, L.V32, np, L.Vw, np);
        launches += 1;
        const dim3 gsym((n + 31) / 32, (n + 31) / 32);
        for (int it = 0; it < 4 && status == JAC_OK; ++it) {
          k_gemm64<<<gsym, 128, 0, st>>>(n, n, n, L.Vw, np, 1, L.Vw, np, L.Jin, L.Js, L.Mn, n, 1);
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
          k_cvt64to32<<<ew_blocks, 256, 0, st>>>(n, n, L.Vw, np, L.Vf, n, nullptr);
          k_ns_correct<<<dim3((n + 63) / 64, (n + 63) / 64), 256, 0, st>>>(n, n, n, L.Vf, n, L.Mf, n, L.Vw, np);
          launches += 3;
          ++ns_global;
          ck(cudaGetLastError());
          if (mm * mm + 1e-6 * mm <= 2e-16) break;
        }
        // G_int = G_in V (V rows are input columns): the FP64 factor the polish works on
        k_gemm64<<<dim3((m + 31) / 32, (n + 31) / 32), 128, 0, st>>>(m, n, n, G, ldg, 0, L.Vw, np, nullptr,
                                                                     nullptr, L.Gw, mp, 0);
        ++launches;
        ck(cudaGetLastError());
        phase = 3;
      }
      continue;
    }
    if (hrec.pivots_rotated == 0) {
      converged = 1;
      break;
    }
  }
  if (n == 1) converged = 1;
  if (status == JAC_OK && !converged) status = JAC_ENOTCONV;

  if (status == JAC_OK || status == JAC_ENOTCONV) {
    k_colnorm<<<(n * 32 + 255) / 256, 256, 0, st>>>(L.Gw, mp, n, L.Js, L.nrm2, L.lam);
    k_rank<<<(n + 255) / 256, 256, sizeof(unsigned long long) * n, st>>>(L.lam, n, L.rank);
    k_scatter<<<n, 128, 0, st>>>(L.Gw, mp, m, L.Vw, np, n, L.nrm2, L.lam, L.rank, lambda, static_cast<double*>(Gv),
                                 ldg, static_cast<double*>(Uv), ldu, want_v ? static_cast<double*>(Vv) : nullptr,
                                 ldv);
    launches += 3;
    if (cudaGetLastError() != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  }
  cudaFreeAsync(base, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && status == JAC_OK) status = JAC_ECUDA;
  prof.finish();
  if (info) {
    for (int u = sweeps; u < 64; ++u) info->sweep_max_scaled[u] = 0.0;
    info->sweeps = sweeps;
    info->converged = converged;
    info->status = status;
    info->steps_per_sweep = last_steps;
    info->rotations = rot_total;
    info->pivots_rotated = piv_total;
    info->max_scaled_off = hrec.max_scaled;
    info->off_rel = (hrec.trace > 0.0) ? std::sqrt(hrec.off2) / hrec.trace : 0.0;
    info->launches = launches;
    info->lowp_sweeps = lowp_sweeps;
    info->global_ns_steps = ns_global;
    info->pivot_ns_steps = ns_total;
    info->inner_sweeps = inner_total;
    for (int u = 0; u < 4; ++u) info->pivot_cycles[u] = cyc_total[u];
  }
  return status;
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

int jacobi_version(void) { return 100; }

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

int jacobi_sched_pairs(int nb, int ordering, const double* weights, int* pairs, int* counts, int max_steps,
                       int* nsteps, jac_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nb < 2 || nb > 4096 || (nb & 1)) return -1;
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
  k_sched_cycle_weight<<<1, 1024, sizeof(int) * nb, st>>>(nb, weights, order, pairs, counts, max_steps, dn);
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
