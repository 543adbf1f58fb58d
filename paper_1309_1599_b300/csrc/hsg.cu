// libhsg: host side of the C ABI declared in include/hsg.h.
//
// Owns every device buffer, validates arguments before touching state,
// enqueues the kernels of kernels.cuh on the context's stream and replays one
// Monte Carlo step (Sec. III, App. A.1) from captured CUDA graphs.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; a no-op unless a profiler is attached

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/hsg.h"
#include "fused.cuh"
#include "persistent.cuh"
#include "transfer.cuh"
#include "sequential.cuh"
#include "measure.cuh"
#include "kernels.cuh"

using namespace hsg;

namespace {

thread_local std::string g_last_error;

hsg_status fail(hsg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define HSG_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(HSG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

struct Bucket {
  int L = 0, N = 0, S_b = 0, G = 0;
  std::vector<int> samples;   // global sample ids, in order
  int* d_samples = nullptr;
  float* d_spins[2] = {nullptr, nullptr};  // [S_b][G][3][N][V]; [1] only with the fused sweep
  int cur = 0;                // which of d_spins holds the current spins
  void* d_J = nullptr;        // f32 [S_b][3][N][6], f16 [S_b][3][N][8] or bimodal u8 [S_b][3][N]
  int sweep_chunks = 0;       // blocks per lattice group in a half-sweep
  bool fused = false;         // sweeps use k_sweep_fused (ping-pong buffers)
  int band_rows = 0, n_bands = 0;  // fused-sweep tiling
  int gp_or = 1, gp_hb = 1;   // fused sweep: lattice groups per CTA (each thread updates all)
                              // of the overrelaxation and heat-bath kernels
  size_t fused_smem = 0;      // dynamic shared memory of the larger of the two fused kernels
  double* d_epart = nullptr;  // [S_b*R][max(sweep_chunks, n_bands)]
  int m_chunks = 0, P = 0;
  bool m_warp = false;        // measurement: one warp per unit (small lattices)
  double* d_mpart = nullptr;  // [S_b][NT][P][m_chunks][kNQ]
  float* d_phase = nullptr;   // [L][2]
  int res_js = 0;             // resident steps: bonds in global memory (0), resident as
                              // stored (1) or resident as FP32 (2)
  size_t res_smem = 0;        // resident steps: dynamic shared memory per CTA
  int res_gp = 1;             // resident steps: lattice groups per work item
  int res_threads = 512;      // resident steps: threads per CTA
  int res_gsub = 0;           // resident steps: lattice groups per CTA (N_T/V: whole sets)
  int res_sets = 1;           // resident steps: whole replica sets per CTA (> 1 only in a joint launch)
};

}  // namespace

// An NVTX range around a public call that enqueues device work, named after
// the call, so a timeline profiler shows where each step's stages begin.
// Replays of captured steps appear as the one hsg_run_steps range.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Lets the other translation units of the library report through
// hsg_last_error().
void hsg_record_error(const std::string& msg) { g_last_error = msg; }

struct hsg_ctx {
  int S = 0, n_rep = 0, NT = 0, R = 0, V = 1, prec = HSG_F32, layout = 0, n_or = 0;
  float bimodal_D = 0.0f;      // HSG_BIMODAL: magnitude of the anisotropic couplings
  int measure_every = 0;
  uint64_t seed = 0;
  std::vector<int> Ls;
  std::vector<double> beta;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<Bucket> buckets;
  std::vector<int> sample_bucket, sample_local;
  int* d_perm = nullptr;        // [S][n_rep][NT] temperature -> slot
  int* d_temp_of = nullptr;     // [S][R] slot -> temperature
  double* d_beta = nullptr;     // [NT]
  float* d_beta_f = nullptr;    // [NT]
  double* d_E = nullptr;        // [S][R]
  double* d_obs = nullptr;      // [S][NT][HSG_NOBS]
  long long* d_counts = nullptr;  // [S][NT]
  long long* d_pt_acc = nullptr;  // [S][n_rep][max(NT-1,1)]
  uint32_t* d_counters = nullptr; // [0] HB sweeps, [1] PT sweeps
  float* d_stage = nullptr;     // staging for spins [max N][3]
  float* d_big = nullptr;       // staging for whole-sample transfers (grown on demand)
  size_t big_cap = 0;           // floats in d_big
  uint32_t* d_tmp_u32 = nullptr;
  bool energy_valid = false;
  uint64_t counters[3] = {0, 0, 0};
  // Captured steps, by [parity of the fused buckets' buffer index][measure?].
  cudaGraphExec_t g_step[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  uint64_t g_step_launches[2][2] = {{0, 0}, {0, 0}};  // kernels per graph replay
  int* d_status = nullptr;     // device status word (HSG_ETIMEOUT from bounded waits)
  bool persistent = false;     // run_steps keeps replica sets resident in shared memory
  bool persistent_joint = false;  // ... with all lattice sizes in one launch
  bool res_split = false;      // some replica set spans several CTAs: one step per launch, PT outside
  bool res_pair = false;       // the resident steps of both buckets run in one launch
  int pair_a = -1, pair_b = -1;  // joint launch: bucket of the first CTAs, bucket of the others
  bool pair_special = false;   // joint launch: the L = 12 with L = 8 specialisation
  int pair_threads = 0;        // joint launch: threads per CTA
  size_t pair_smem = 0;        // joint launch: dynamic shared memory per CTA
  std::vector<std::array<int, 2>> pair_cands;  // joint launch: feasible (sets per CTA, bond
                                               // residency) of the smaller size, planned first
  long long timeout_cycles = 0;
  int sweep_kernel = 0;
  uint64_t launches = 0;       // kernels enqueued by this context so far
  uint64_t* launch_sink = nullptr;  // where enqueue helpers count launches
};

namespace {

uint2 philox_key(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

size_t bond_bytes(int prec) { return prec == HSG_F16 ? 16 : prec == HSG_BIMODAL ? 1 : 24; }

template <int K>
using IC = std::integral_constant<int, K>;

// Calls f(IC<V>, IC<PREC>) for a context's layout (lattices per element) and
// coupling format; every branch must return the same type.
template <typename F>
decltype(auto) dispatch(int V, int prec, F&& f) {
  if (V == 2) {
    if (prec == HSG_F16) return f(IC<2>{}, IC<kPrecF16>{});
    if (prec == HSG_BIMODAL) return f(IC<2>{}, IC<kPrecBimodal>{});
    return f(IC<2>{}, IC<kPrecF32>{});
  }
  if (prec == HSG_F16) return f(IC<1>{}, IC<kPrecF16>{});
  if (prec == HSG_BIMODAL) return f(IC<1>{}, IC<kPrecBimodal>{});
  return f(IC<1>{}, IC<kPrecF32>{});
}

void free_ctx(hsg_ctx* h) {
  if (!h) return;
  for (int a = 0; a < 2; ++a)
    for (int m = 0; m < 2; ++m)
      if (h->g_step[a][m]) cudaGraphExecDestroy(h->g_step[a][m]);
  cudaFree(h->d_status);
  for (Bucket& b : h->buckets) {
    cudaFree(b.d_samples);
    cudaFree(b.d_spins[0]);  // d_spins[1] lies in the same allocation
    cudaFree(b.d_J);
    cudaFree(b.d_epart);
    cudaFree(b.d_mpart);
    cudaFree(b.d_phase);
  }
  cudaFree(h->d_perm);
  cudaFree(h->d_temp_of);
  cudaFree(h->d_beta);
  cudaFree(h->d_beta_f);
  cudaFree(h->d_E);
  cudaFree(h->d_obs);
  cudaFree(h->d_counts);
  cudaFree(h->d_pt_acc);
  cudaFree(h->d_counters);
  cudaFree(h->d_stage);
  cudaFree(h->d_big);
  cudaFree(h->d_tmp_u32);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

template <typename T>
hsg_status dalloc(T** p, size_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(HSG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return HSG_OK;
}

#define HSG_TRY(expr)                  \
  do {                                 \
    hsg_status st_ = (expr);           \
    if (st_ != HSG_OK) return st_;     \
  } while (0)

int acc_stride(const hsg_ctx* h) { return h->NT > 1 ? h->NT - 1 : 1; }

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit belongs to the kernel, not to a context: every
// context of the process launches the same kernels, so the limit only ever
// grows (a context needing less must not lower it under another context's
// captured launches).
hsg_status raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limits;
  int dev = 0;
  HSG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limits[{dev, fn}];
  if (bytes <= cur) return HSG_OK;
  HSG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)));
  cur = bytes;
  return HSG_OK;
}

// Storage position of the natural site i = x + L*(y + L*z) (parity-split rows,
// as on the device).
size_t storage_site(size_t i, int L) {
  const size_t x = i % L, row = i / L;
  return row * L + (x & 1) * (L / 2) + (x >> 1);
}

// ----------------------------------------------------------------------------
// Enqueue helpers (stream-ordered; used directly and under graph capture)
// ----------------------------------------------------------------------------
BucketView view(const Bucket& b) {
  BucketView v;
  v.spins = b.d_spins[b.cur];
  v.J = b.d_J;
  v.sample_ids = b.d_samples;
  v.L = b.L;
  v.N = b.N;
  v.S_b = b.S_b;
  v.G = b.G;
  v.D = 0.0f;
  return v;
}

template <int KIND>
hsg_status launch_half(hsg_ctx* h, const Bucket& b, int colour, bool energy, cudaStream_t st) {
  SweepParams p;
  p.b = view(b);
  p.b.D = h->bimodal_D;
  p.colour = colour;
  p.chunks = b.sweep_chunks;
  p.R = h->R;
  p.temp_of = h->d_temp_of;
  p.beta_f = h->d_beta_f;
  p.key = philox_key(h->seed);
  p.counters = h->d_counters;
  p.e_partial = energy ? b.d_epart : nullptr;
  const unsigned grid = static_cast<unsigned>(b.S_b * b.G * b.sweep_chunks);
  *h->launch_sink += 1;
  dispatch(h->V, h->prec, [&](auto v, auto pr) {
    k_sweep_half<KIND, decltype(v)::value, decltype(pr)::value, true><<<grid, kSweepThreads, 0, st>>>(p);
    return 0;
  });
  HSG_CUDA(cudaGetLastError());
  return HSG_OK;
}

// The fused-sweep kernel for a tiling: compile-time specialisations for the
// common ones (L = 64 and L = 32 in bands of 8 rows), the run-time-geometry
// kernel otherwise; gp lattice groups per CTA (2 only with two lattices per
// element).
using FusedKernel = void (*)(FusedParams);

template <int KIND, int V, int PREC, int GP>
FusedKernel fused_kernel_gp(int L, int band_rows) {
  if (L == 64 && band_rows == 8) return k_sweep_fused<KIND, V, PREC, 64, 8, GP>;
  if (L == 32 && band_rows == 8) return k_sweep_fused<KIND, V, PREC, 32, 8, GP>;
  return k_sweep_fused<KIND, V, PREC, 0, 0, GP>;
}

template <int KIND, int V, int PREC>
FusedKernel fused_kernel(int L, int band_rows, int gp) {
  if constexpr (V == 2) {
    if (gp == 2) return fused_kernel_gp<KIND, V, PREC, 2>(L, band_rows);
  }
  return fused_kernel_gp<KIND, V, PREC, 1>(L, band_rows);
}

// Every fused kernel of (KIND, V, PREC) with gp groups per CTA.
template <int KIND, int V, int PREC>
std::vector<FusedKernel> fused_kernels(int gp) {
  std::vector<FusedKernel> v;
  for (const int L : {64, 32, 0}) v.push_back(fused_kernel<KIND, V, PREC>(L, L > 0 ? 8 : 0, gp));
  return v;
}

template <int KIND, int V, int PREC>
void fused_kernel_launch(const FusedParams& p, int gp, unsigned grid, unsigned block, size_t smem,
                         cudaStream_t st) {
  fused_kernel<KIND, V, PREC>(p.L, p.band_rows, gp)<<<grid, block, smem, st>>>(p);
}

// Dynamic shared memory of the fused kernel: a ring of kFusedSlots planes of
// gp lattice groups, each the band plus two halo rows per side (or whole
// planes), three components of L * V floats per row.
size_t fused_smem_bytes(int L, int V, int gp, int band_rows) {
  const int rows = (band_rows == L) ? L : band_rows + 4;
  return static_cast<size_t>(kFusedSlots) * 3 * gp * rows * L * V * sizeof(float);
}

// One whole sweep (both colours) of a bucket with the fused kernel; reads the
// current buffer, writes the other, then flips the bucket's buffer index.
// With probe_timeout the kernel only exercises its bounded-wait failure path
// (it writes no spins and the buffer index is kept).
template <int KIND>
hsg_status launch_fused(hsg_ctx* h, Bucket& b, bool energy, cudaStream_t st, bool probe_timeout = false,
                        long long timeout = 0) {
  FusedParams p;
  p.in = b.d_spins[b.cur];
  p.out = b.d_spins[b.cur ^ 1];
  p.J = b.d_J;
  p.sample_ids = b.d_samples;
  p.L = b.L;
  p.N = b.N;
  p.G = b.G;
  p.R = h->R;
  p.band_rows = b.band_rows;
  p.n_bands = b.n_bands;
  p.temp_of = h->d_temp_of;
  p.beta_f = h->d_beta_f;
  p.key = philox_key(h->seed);
  p.counters = h->d_counters;
  p.e_partial = energy ? b.d_epart : nullptr;
  p.status = h->d_status;
  p.timeout = timeout > 0 ? timeout : h->timeout_cycles;
  p.probe_timeout = probe_timeout ? 1 : 0;
  p.D = h->bimodal_D;
  const int rows_t = (b.band_rows == b.L) ? b.L : b.band_rows + 2;
  const unsigned block = static_cast<unsigned>(((rows_t * (b.L / 2)) + 31) / 32 * 32);
  const int gp = (KIND == kHB) ? b.gp_hb : b.gp_or;
  const unsigned grid = static_cast<unsigned>(b.S_b * (b.G / gp) * b.n_bands);
  const size_t smem = fused_smem_bytes(b.L, h->V, gp, b.band_rows);
  *h->launch_sink += 1;
  dispatch(h->V, h->prec, [&](auto v, auto pr) {
    fused_kernel_launch<KIND, decltype(v)::value, decltype(pr)::value>(p, gp, grid, block, smem, st);
    return 0;
  });
  HSG_CUDA(cudaGetLastError());
  if (!probe_timeout) b.cur ^= 1;
  return HSG_OK;
}

template <int KIND, int V, int PREC>
hsg_status allow_fused_smem(size_t bytes) {
  for (const int gp : {1, 2})
    for (FusedKernel fn : fused_kernels<KIND, V, PREC>(gp))
      HSG_TRY(raise_smem_limit(reinterpret_cast<const void*>(fn), bytes));
  return HSG_OK;
}

// Smallest block limit over a kind's fused kernels with gp groups per CTA, as
// the CUDA driver reports it for their register use; 0 if unknown.
template <int KIND, int V, int PREC>
int fused_max_threads_one(int gp) {
  int best = 1 << 30;
  for (FusedKernel fn : fused_kernels<KIND, V, PREC>(gp)) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = std::min(best, a.maxThreadsPerBlock);
  }
  return best;
}

// Largest block the fused kernels (heat-bath and overrelaxation) with gp
// groups per CTA can launch with, as the CUDA driver reports it for their
// register use; 0 if unknown.
int fused_max_threads(int V, int prec, int gp) {
  return dispatch(V, prec, [gp](auto v, auto pr) {
    constexpr int VV = decltype(v)::value, P = decltype(pr)::value;
    const int a = fused_max_threads_one<kHB, VV, P>(gp), b = fused_max_threads_one<kOR, VV, P>(gp);
    return std::min(std::min(a, b), kFusedMaxThreads);
  });
}

hsg_status allow_fused_smem_all(int V, int prec, size_t bytes) {
  return dispatch(V, prec, [&](auto v, auto pr) {
    constexpr int VV = decltype(v)::value, P = decltype(pr)::value;
    const hsg_status a = allow_fused_smem<kHB, VV, P>(bytes);
    return a != HSG_OK ? a : allow_fused_smem<kOR, VV, P>(bytes);
  });
}

// Tiling of the fused sweep for lattice size L, V lattices per element and gp
// lattice groups per CTA: whole planes for L <= 24, else the smallest band of
// rows (a divisor of L, at least 8) within the thread and shared-memory
// limits, else whole planes if they fit.  False: use the two-pass half-sweep
// kernel.
bool plan_fused(int L, int V, int gp, int max_threads, int want, int* band_rows, size_t* smem) {
  const size_t max_smem = 200 * 1024;
  auto smem_for = [&](int rows) {
    return static_cast<size_t>(kFusedSlots) * 3 * gp * rows * L * V * sizeof(float);
  };
  if (gp != 1 && (gp != 2 || V != 2)) return false;
  // blocks are rounded up to whole warps
  auto threads_for = [&](int rows) { return (rows * (L / 2) + 31) / 32 * 32; };
  if (max_threads <= 0) return false;
  if (want > 0) {  // a requested band: whole planes, or a divisor of L of at least 8 rows
    const bool full = (want == L);
    if (!full && (want < 8 || L % want != 0 || (L * V) % 4 != 0)) return false;
    const int rows_t = full ? L : want + 2, rows_s = full ? L : want + 4;
    if (threads_for(rows_t) > max_threads || smem_for(rows_s) > max_smem) return false;
    *band_rows = want;
    *smem = smem_for(rows_s);
    return true;
  }
  const bool planes_fit = threads_for(L) <= max_threads && smem_for(L) <= max_smem;
  // small lattices: whole planes, no halo rows (at L = 24 they ran 24% faster
  // per step than 8-row bands; at L = 32 8-row bands win)
  if (planes_fit && L <= 24) {
    *band_rows = L;
    *smem = smem_for(L);
    return true;
  }
  // the smallest band that tiles L: more, smaller CTAs per SM overlap their
  // per-plane barriers (8-row bands ran faster than 16-row ones at L = 64,
  // and than whole planes at L = 32)
  if ((L * V) % 4 == 0) {  // 16-byte rows for the bulk copies
    for (int B = 8; B <= L / 2; ++B) {
      if (L % B != 0) continue;
      if (threads_for(B + 2) <= max_threads && smem_for(B + 4) <= max_smem) {
        *band_rows = B;
        *smem = smem_for(B + 4);
        return true;
      }
    }
  }
  if (planes_fit) {
    *band_rows = L;
    *smem = smem_for(L);
    return true;
  }
  return false;
}

// Resident-step kernel for (V, precision, bond residency, L, groups per
// item): L = 8 and 12 have compile-time specialisations when the bonds are
// resident, and with two lattices per element also two-group items (gp = 2);
// L = 16 and 20 have them for every bond residency.
template <int V, int PREC, int JS>
void* persistent_fn_L(int L, int gp) {
  // L = 16 and 20: parts of replica sets (one or two groups per CTA)
  if (L == 16) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 16>);
  if (L == 20) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 20>);
  if constexpr (JS == 0) {
    return reinterpret_cast<void*>(k_persistent<V, PREC, 0, 0>);
  } else {
    if constexpr (V == 2) {
      if (gp == 2 && L == 8) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 8, 2>);
      if (gp == 2 && L == 12) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 12, 2>);
    }
    if (L == 8) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 8>);
    if (L == 12) return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 12>);
    return reinterpret_cast<void*>(k_persistent<V, PREC, JS, 0>);
  }
}

template <int V, int PREC>
void* persistent_fn_js(int js, int L, int gp) {
  if (js == 0) return persistent_fn_L<V, PREC, 0>(L, 1);
  if constexpr (PREC == kPrecF32) {
    return persistent_fn_L<V, PREC, 1>(L, gp);  // FP32 bonds are resident as stored
  } else {
    return js == 1 ? persistent_fn_L<V, PREC, 1>(L, gp) : persistent_fn_L<V, PREC, 2>(L, gp);
  }
}

void* persistent_kernel(int V, int prec, int js, int L, int gp) {
  return dispatch(V, prec, [&](auto v, auto pr) {
    return persistent_fn_js<decltype(v)::value, decltype(pr)::value>(js, L, gp);
  });
}

// The joint resident kernel of two buckets: the L = 12 with L = 8
// specialisation (two lattices per element, L = 12 bonds resident as stored,
// the L = 8 bucket's bonds as stored (jsb = 1) or as FP32 (jsb = 2), two
// groups per work item), or the generic one (run-time L, bonds from global
// memory, one group per item).
template <int V, int PREC>
void* pair_fn(bool special, int jsb) {
  if constexpr (V == 2) {
    if (special) {
      if constexpr (PREC == kPrecF32) {
        return reinterpret_cast<void*>(k_persistent_pair<V, PREC, 1, 12, 2, 1, 8, 2>);
      } else {
        return jsb == 2 ? reinterpret_cast<void*>(k_persistent_pair<V, PREC, 1, 12, 2, 2, 8, 2>)
                        : reinterpret_cast<void*>(k_persistent_pair<V, PREC, 1, 12, 2, 1, 8, 2>);
      }
    }
  }
  return reinterpret_cast<void*>(k_persistent_pair<V, PREC, 0, 0, 1, 0, 0, 1>);
}

void* pair_kernel(int V, int prec, bool special, int jsb) {
  return dispatch(V, prec, [&](auto v, auto pr) {
    return pair_fn<decltype(v)::value, decltype(pr)::value>(special, jsb);
  });
}

// Lattice groups per work item of the resident kernel: two where a
// specialisation exists and the groups a CTA holds pair up.
int persistent_gp(int V, int g_sub, int js, int L) {
  return (V == 2 && js != 0 && (L == 8 || L == 12) && g_sub % 2 == 0) ? 2 : 1;
}

// Threads of a resident CTA: 512 for the generic kernel; for an L
// specialisation the warp count from 16 to its limit that takes the fewest
// rounds over `items` work items of hN sites each (warps split evenly over
// the items in flight, 32 sites per warp and round), the smallest such.
int persistent_threads(int items, int hN, int max_threads) {
  if (max_threads >= kPersistentMaxThreads) return 512;
  int best_w = 16;
  long best = -1;
  for (int W = 16; W <= max_threads / 32; ++W) {
    const int wpg = W >= items ? W / items : 1;
    const int gpp = W / wpg;
    const long rounds = static_cast<long>((items + gpp - 1) / gpp) * ((hN + 32 * wpg - 1) / (32 * wpg));
    if (best < 0 || rounds < best) {
      best = rounds;
      best_w = W;
    }
  }
  return 32 * best_w;
}

// Plans the resident steps of every bucket.  A CTA holds G_sub lattice groups
// of one replica set: the whole set (N_T/V groups) when it fits, so PT runs
// in the kernel; otherwise the divisor of the set that keeps the most groups
// resident per SM (ties: more CTAs per SM), one step per launch with PT
// outside.  Shared memory per CTA: spins 12 V G_sub N bytes, plus the bonds
// (3 N per sample) when they fit beside them -- converted to FP32 (JS = 2)
// unless that lowers the CTAs per SM, else as stored (JS = 1) -- or read from
// global memory (JS = 0).
hsg_status plan_persistent(hsg_ctx* h) {
  int dev = 0, optin = 0;
  HSG_CUDA(cudaGetDevice(&dev));
  HSG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int G_set = h->NT / h->V;
  h->res_split = false;
  for (Bucket& b : h->buckets) {
    const size_t stored = h->prec == HSG_F16 ? 12 : h->prec == HSG_BIMODAL ? 1 : 24;
    const size_t bond_bytes[3] = {0, stored, 24};
    int best_js = -1, best_occ = 0, best_threads = 0, best_gsub = 0;
    size_t best_smem = 0;
    for (int g_sub = G_set; g_sub >= 1; --g_sub) {
      if (G_set % g_sub != 0) continue;
      if (best_js >= 0 && best_gsub == G_set) break;  // a whole set fits: keep PT in the kernel
      const size_t spins = static_cast<size_t>(12) * h->V * g_sub * b.N;
      for (int js = (h->prec == HSG_F32 ? 1 : 2); js >= 0; --js) {
        const int gp = persistent_gp(h->V, g_sub, js, b.L);
        void* fn = persistent_kernel(h->V, h->prec, js, b.L, gp);
        cudaFuncAttributes fa;
        HSG_CUDA(cudaFuncGetAttributes(&fa, fn));
        const size_t budget = static_cast<size_t>(optin) - fa.sharedSizeBytes;
        const size_t smem = spins + 3 * static_cast<size_t>(b.N) * bond_bytes[js];
        if (smem > budget) continue;
        HSG_TRY(raise_smem_limit(fn, budget));
        int occ = 0;
        const int threads = persistent_threads(g_sub / gp, b.N / 2, fa.maxThreadsPerBlock);
        HSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
        if (occ < 1) continue;
        // groups resident per SM first, then CTAs per SM
        const long score = static_cast<long>(occ) * g_sub * 1024 + occ;
        const long best = static_cast<long>(best_occ) * best_gsub * 1024 + best_occ;
        if (best_js < 0 || score > best) {
          best_js = js;
          best_occ = occ;
          best_smem = smem;
          best_threads = threads;
          best_gsub = g_sub;
        }
      }
    }
    if (best_js < 0) return fail(HSG_EINVAL, "a lattice group does not fit in shared memory");
    b.res_js = best_js;
    b.res_smem = best_smem;
    b.res_gsub = best_gsub;
    b.res_gp = persistent_gp(h->V, best_gsub, best_js, b.L);
    b.res_threads = best_threads;
    b.res_sets = 1;
    if (best_gsub < G_set) h->res_split = true;
  }
  h->res_pair = false;
  return HSG_OK;
}

// Plans the resident steps of a two-bucket context as one launch: bucket a
// (the larger L) holds one replica set per CTA as planned alone; bucket b
// holds as many whole replica sets of one sample per CTA (a divisor of
// n_replicas) as fit in the shared memory bucket a's CTAs take, so the
// launch's one block shape and shared-memory size serve both.  HSG_EINVAL if
// a replica set cannot be held whole or the buckets do not fit.
hsg_status plan_joint(hsg_ctx* h) {
  if (h->buckets.size() == 1) return HSG_OK;  // one lattice size: one launch already
  if (h->buckets.size() > 2) return fail(HSG_EINVAL, "one resident launch holds at most two lattice sizes");
  if (h->res_split)
    return fail(HSG_EINVAL, "one launch for all lattice sizes needs every replica set held whole by a CTA");
  int dev = 0, optin = 0;
  HSG_CUDA(cudaGetDevice(&dev));
  HSG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int ia = h->buckets[0].N >= h->buckets[1].N ? 0 : 1, ib = 1 - ia;
  Bucket& A = h->buckets[ia];
  Bucket& B = h->buckets[ib];
  const size_t stored = h->prec == HSG_F16 ? 12 : h->prec == HSG_BIMODAL ? 1 : 24;
  const size_t bond_bytes[3] = {0, stored, 24};
  const int G_set = h->NT / h->V;
  // The L = 12 with L = 8 specialisation keeps bucket a's bonds resident as
  // stored; where that does not fit one CTA (FP32 bonds beside eight
  // temperatures of spins), or for other sizes, the generic joint kernel
  // reads the bonds from global memory.
  bool special = false;
  size_t smem_a = 0;
  int jsa = 0;
  for (const bool sp : {h->V == 2 && A.L == 12 && B.L == 8, false}) {
    jsa = sp ? 1 : 0;
    smem_a = static_cast<size_t>(12) * h->V * G_set * A.N + 3 * static_cast<size_t>(A.N) * bond_bytes[jsa];
    std::vector<int> jsbs;
    if (sp && h->prec != HSG_F32) jsbs.push_back(2);
    jsbs.push_back(sp ? 1 : 0);
    // every (sets per CTA, bond residency) of bucket b that fits in the
    // shared memory bucket a's CTAs take; the first (most sets, FP32 bonds
    // first) is the plan until the autotuner times the others
    h->pair_cands.clear();
    for (int k = h->n_rep; k >= 1; --k) {
      if (h->n_rep % k != 0 || k * h->NT > kMaxTempsResident) continue;
      for (const int jsb : jsbs) {
        const size_t smem_b =
            static_cast<size_t>(12) * h->V * k * G_set * B.N + 3 * static_cast<size_t>(B.N) * bond_bytes[jsb];
        if (smem_b <= smem_a) h->pair_cands.push_back({k, jsb});
      }
    }
    bool fits = !h->pair_cands.empty();
    for (const auto& c : h->pair_cands) {
      cudaFuncAttributes fc;
      HSG_CUDA(cudaFuncGetAttributes(&fc, pair_kernel(h->V, h->prec, sp, c[1])));
      if (smem_a + fc.sharedSizeBytes > static_cast<size_t>(optin)) fits = false;
    }
    if (fits) {
      special = sp;
      break;
    }
    h->pair_cands.clear();
  }
  if (h->pair_cands.empty())
    return fail(HSG_EINVAL, "a replica set of L = " + std::to_string(A.L) + " does not fit one CTA of the joint launch");
  for (const auto& c : h->pair_cands) {
    void* f = pair_kernel(h->V, h->prec, special, c[1]);
    cudaFuncAttributes fc;
    HSG_CUDA(cudaFuncGetAttributes(&fc, f));
    HSG_TRY(raise_smem_limit(f, static_cast<size_t>(optin) - fc.sharedSizeBytes));
  }
  const int best_k = h->pair_cands[0][0], best_jsb = h->pair_cands[0][1];
  const size_t best_smem = smem_a;
  void* fn = pair_kernel(h->V, h->prec, special, best_jsb);
  cudaFuncAttributes fa;
  HSG_CUDA(cudaFuncGetAttributes(&fa, fn));
  const int threads = std::min(fa.maxThreadsPerBlock, std::max(A.res_threads, B.res_threads)) / 32 * 32;
  int occ = 0;
  HSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, best_smem));
  if (occ < 1) return fail(HSG_EINVAL, "the joint resident launch does not fit an SM");
  A.res_js = jsa;
  A.res_gp = special ? 2 : 1;
  A.res_gsub = G_set;
  A.res_sets = 1;
  B.res_js = best_jsb;
  B.res_gp = special ? 2 : 1;
  B.res_gsub = best_k * G_set;
  B.res_sets = best_k;
  A.res_smem = B.res_smem = best_smem;
  A.res_threads = B.res_threads = threads;
  h->res_pair = true;
  h->pair_a = ia;
  h->pair_b = ib;
  h->pair_special = special;
  h->pair_threads = threads;
  h->pair_smem = best_smem;
  return HSG_OK;
}

hsg_status enqueue_bump(hsg_ctx* h, uint32_t dhb, uint32_t dpt, cudaStream_t st);

// Launch arguments of the resident-step kernel for one bucket (the state
// buffers of the context; the tuner substitutes scratch copies).
PersistentParams persistent_params(hsg_ctx* h, const Bucket& b, int steps) {
  PersistentParams p;
  p.spins = b.d_spins[b.cur];
  p.J = b.d_J;
  p.sample_ids = b.d_samples;
  p.L = b.L;
  p.N = b.N;
  p.G = b.G;
  p.R = h->R;
  p.n_rep = h->n_rep;
  p.NT = h->NT;
  p.n_or = h->n_or;
  p.steps = steps;
  p.beta = h->d_beta;
  p.E = h->d_E;
  p.perm = h->d_perm;
  p.temp_of = h->d_temp_of;
  p.accepted = h->d_pt_acc;
  p.key = philox_key(h->seed);
  p.counters = h->d_counters;
  p.D = h->bimodal_D;
  p.G_sub = b.res_gsub;
  p.sets = b.res_sets;
  p.pt = h->res_split ? 0 : 1;
  p.warps = b.res_threads / 32;
  return p;
}

hsg_status launch_persistent(hsg_ctx* h, const Bucket& b, PersistentParams p, int gp, int threads,
                             cudaStream_t st) {
  p.warps = threads / 32;
  void* args[] = {&p};
  *h->launch_sink += 1;
  const int n_sub = h->NT / h->V / p.G_sub;  // CTAs per replica set
  HSG_CUDA(cudaLaunchKernel(persistent_kernel(h->V, h->prec, b.res_js, b.L, gp),
                            dim3(b.S_b * h->n_rep * n_sub), dim3(threads), args, b.res_smem, st));
  return HSG_OK;
}

// The joint launch: bucket pair_a's CTAs (one replica set each) first, then
// bucket pair_b's (res_sets whole sets of one sample each).
hsg_status launch_pair(hsg_ctx* h, PersistentParams pa, PersistentParams pb, int threads, cudaStream_t st) {
  const Bucket& A = h->buckets[h->pair_a];
  const Bucket& B = h->buckets[h->pair_b];
  int ctas_a = A.S_b * h->n_rep;
  const int ctas_b = B.S_b * (h->n_rep / B.res_sets);
  void* args[] = {&pa, &pb, &ctas_a};
  *h->launch_sink += 1;
  HSG_CUDA(cudaLaunchKernel(pair_kernel(h->V, h->prec, h->pair_special, B.res_js), dim3(ctas_a + ctas_b),
                            dim3(threads), args, h->pair_smem, st));
  return HSG_OK;
}

hsg_status enqueue_pt(hsg_ctx* h, cudaStream_t st);

// `steps` whole Monte Carlo steps with the lattices resident in shared
// memory: one launch per bucket (and, when replica sets span several CTAs,
// one step per call with the PT sweep as its own kernel), then the sweep
// counters advance.
hsg_status enqueue_persistent(hsg_ctx* h, int steps, cudaStream_t st) {
  if (h->res_split && steps != 1) return fail(HSG_ESTATE, "split replica sets run one step per launch");
  if (h->res_pair) {
    HSG_TRY(launch_pair(h, persistent_params(h, h->buckets[h->pair_a], steps),
                        persistent_params(h, h->buckets[h->pair_b], steps), h->pair_threads, st));
  } else {
    for (const Bucket& b : h->buckets)
      HSG_TRY(launch_persistent(h, b, persistent_params(h, b, steps), b.res_gp, b.res_threads, st));
  }
  if (h->res_split) HSG_TRY(enqueue_pt(h, st));
  return enqueue_bump(h, static_cast<uint32_t>(steps), static_cast<uint32_t>(steps), st);
}

hsg_status enqueue_bump(hsg_ctx* h, uint32_t dhb, uint32_t dpt, cudaStream_t st) {
  *h->launch_sink += 1;
  k_bump_counters<<<1, 1, 0, st>>>(h->d_counters, dhb, dpt);
  HSG_CUDA(cudaGetLastError());
  return HSG_OK;
}

hsg_status enqueue_hb_sweep(hsg_ctx* h, cudaStream_t st) {
  for (Bucket& b : h->buckets) {
    if (b.fused) {
      HSG_TRY(launch_fused<kHB>(h, b, false, st));
    } else {
      HSG_TRY(launch_half<kHB>(h, b, 0, false, st));
      HSG_TRY(launch_half<kHB>(h, b, 1, false, st));
    }
  }
  return HSG_OK;
}

// E = sum of each lattice's partials; `from_sweep` selects the partial layout
// of the sweep kernels (fused: one per band) over that of the energy pass.
hsg_status enqueue_energy_finalize(hsg_ctx* h, bool from_sweep, cudaStream_t st) {
  for (const Bucket& b : h->buckets) {
    const int n_lat = b.S_b * h->R;
    const int threads = 256;
    const int blocks = (n_lat * 32 + threads - 1) / threads;
    const int chunks = (from_sweep && b.fused) ? b.n_bands : b.sweep_chunks;
    *h->launch_sink += 1;
    k_energy_finalize<<<blocks, threads, 0, st>>>(b.d_epart, chunks, n_lat, b.d_samples, h->R, h->d_E);
    HSG_CUDA(cudaGetLastError());
  }
  return HSG_OK;
}

// n overrelaxation sweeps; the white half of the last one writes energies.
hsg_status enqueue_or_sweeps(hsg_ctx* h, int n, cudaStream_t st) {
  for (int s = 0; s < n; ++s) {
    const bool last = (s == n - 1);
    for (Bucket& b : h->buckets) {
      if (b.fused) {
        HSG_TRY(launch_fused<kOR>(h, b, last, st));
      } else {
        HSG_TRY(launch_half<kOR>(h, b, 0, false, st));
        HSG_TRY(launch_half<kOR>(h, b, 1, last, st));
      }
    }
  }
  if (n > 0) HSG_TRY(enqueue_energy_finalize(h, true, st));
  return HSG_OK;
}

hsg_status enqueue_energy(hsg_ctx* h, cudaStream_t st) {
  for (const Bucket& b : h->buckets) HSG_TRY(launch_half<kEnergyOnly>(h, b, 1, true, st));
  return enqueue_energy_finalize(h, false, st);
}

hsg_status enqueue_pt(hsg_ctx* h, cudaStream_t st) {
  const int n_sets = h->S * h->n_rep;
  *h->launch_sink += 1;
  if (h->NT <= kPtWarpMaxTemps) {
    k_pt_sweep_warp<<<n_sets, 32, 0, st>>>(h->n_rep, h->NT, h->R, h->d_beta, h->d_E, h->d_perm, h->d_temp_of,
                                           h->d_pt_acc, philox_key(h->seed), h->d_counters);
  } else {
    const int threads = 128;
    k_pt_sweep<<<(n_sets + threads - 1) / threads, threads, 0, st>>>(
        n_sets, h->n_rep, h->NT, h->R, h->d_beta, h->d_E, h->d_perm, h->d_temp_of, h->d_pt_acc,
        philox_key(h->seed), h->d_counters);
  }
  HSG_CUDA(cudaGetLastError());
  return HSG_OK;
}

hsg_status enqueue_measure(hsg_ctx* h, cudaStream_t st) {
  for (const Bucket& b : h->buckets) {
    MeasureParams p;
    p.b = view(b);
    p.b.D = h->bimodal_D;
    p.R = h->R;
    p.n_rep = h->n_rep;
    p.NT = h->NT;
    p.P = b.P;
    p.chunks = b.m_chunks;
    p.perm = h->d_perm;
    p.beta = h->d_beta;
    p.phase = b.d_phase;
    p.partial = b.d_mpart;
    const unsigned grid = static_cast<unsigned>(b.S_b * h->NT * b.P * b.m_chunks);
    *h->launch_sink += 2;
    const int n_units = b.S_b * h->NT * b.P;
    const unsigned wgrid = static_cast<unsigned>((n_units + kMeasureThreads / 32 - 1) / (kMeasureThreads / 32));
    dispatch(h->V, h->prec, [&](auto v, auto pr) {
      constexpr int VV = decltype(v)::value, P = decltype(pr)::value;
      if (b.m_warp) k_measure_warp<VV, P><<<wgrid, kMeasureThreads, measure_block_smem(b.L), st>>>(p, n_units);
      else k_measure<VV, P><<<grid, kMeasureThreads, measure_block_smem(b.L), st>>>(p);
      return 0;
    });
    HSG_CUDA(cudaGetLastError());
    const int units = b.S_b * h->NT;
    k_measure_finalize<<<(units + 127) / 128, 128, 0, st>>>(b.d_mpart, b.d_samples, b.S_b, h->NT, b.P, b.m_chunks,
                                                           h->n_rep, h->R, b.N, h->d_perm, h->d_E, h->d_obs,
                                                           h->d_counts);
    HSG_CUDA(cudaGetLastError());
  }
  return HSG_OK;
}

// One Monte Carlo step: HB sweep, n_or OR sweeps (energies fused into the
// last), energies, PT, optional measurement, counters.
hsg_status enqueue_step(hsg_ctx* h, bool with_measure, cudaStream_t st) {
  HSG_TRY(enqueue_hb_sweep(h, st));
  if (h->n_or > 0) HSG_TRY(enqueue_or_sweeps(h, h->n_or, st));
  else HSG_TRY(enqueue_energy(h, st));
  if (h->NT > 1) HSG_TRY(enqueue_pt(h, st));
  if (with_measure) HSG_TRY(enqueue_measure(h, st));
  return enqueue_bump(h, 1, 1, st);
}

// Buffer index of the buckets swept by the fused kernel (they all flip
// together, so one parity describes them); 0 if there are none.
int fused_parity(const hsg_ctx* h) {
  for (const Bucket& b : h->buckets)
    if (b.fused) return b.cur;
  return 0;
}

// Captures one step starting from fused-buffer parity `par`; the buckets'
// buffer indices are left as they were.
hsg_status capture_graph(hsg_ctx* h, int par, bool with_measure, cudaGraphExec_t* out, uint64_t* n_kernels) {
  cudaGraph_t graph = nullptr;
  std::vector<int> saved;
  for (Bucket& b : h->buckets) {
    saved.push_back(b.cur);
    if (b.fused) b.cur = par;
  }
  HSG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  *n_kernels = 0;
  h->launch_sink = n_kernels;
  hsg_status st = enqueue_step(h, with_measure, h->cap_stream);
  h->launch_sink = &h->launches;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  for (size_t j = 0; j < h->buckets.size(); ++j) h->buckets[j].cur = saved[j];
  if (st != HSG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(HSG_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(HSG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return HSG_OK;
}

// HSG_ETIMEOUT if a kernel recorded an expired bounded wait since the last
// check (the word is then cleared); call after synchronising the stream.
hsg_status status_check(hsg_ctx* h) {
  int st = 0;
  HSG_CUDA(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    HSG_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    return fail(HSG_ETIMEOUT, "a device-side wait gave up (timeout_cycles exceeded); that launch did not complete");
  }
  return HSG_OK;
}

hsg_status check_sample(const hsg_ctx* h, int sample) {
  if (sample < 0 || sample >= h->S) return fail(HSG_EINVAL, "sample index out of range");
  return HSG_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* hsg_last_error(void) { return g_last_error.c_str(); }

int hsg_version(void) { return HSG_VERSION; }

hsg_status hsg_lattice_create(const hsg_config* cfg, hsg_t* out) {
  if (!out) return fail(HSG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(HSG_EINVAL, "cfg is NULL");
  if (cfg->n_samples < 1 || !cfg->L) return fail(HSG_EINVAL, "n_samples must be >= 1 and L non-NULL");
  if (cfg->n_replicas < 1 || cfg->n_temps < 1 || !cfg->beta)
    return fail(HSG_EINVAL, "n_replicas and n_temps must be >= 1 and beta non-NULL");
  if (cfg->coupling_prec != HSG_F32 && cfg->coupling_prec != HSG_F16 && cfg->coupling_prec != HSG_BIMODAL)
    return fail(HSG_EINVAL, "coupling_prec must be HSG_F32, HSG_F16 or HSG_BIMODAL");
  if (cfg->coupling_prec == HSG_BIMODAL && !(cfg->bimodal_D >= 0.0 && cfg->bimodal_D < 1e30))
    return fail(HSG_EINVAL, "bimodal_D must be finite and >= 0");
  if (cfg->layout != HSG_LAYOUT_PLAIN && cfg->layout != HSG_LAYOUT_BATCHED)
    return fail(HSG_EINVAL, "layout must be HSG_LAYOUT_PLAIN or HSG_LAYOUT_BATCHED");
  if (cfg->n_or < 0 || cfg->measure_every < 0) return fail(HSG_EINVAL, "n_or and measure_every must be >= 0");
  if (cfg->sweep_kernel != HSG_SWEEP_AUTO && cfg->sweep_kernel != HSG_SWEEP_TWO_PASS)
    return fail(HSG_EINVAL, "sweep_kernel must be HSG_SWEEP_AUTO or HSG_SWEEP_TWO_PASS");
  if (cfg->band_rows < 0 || (cfg->band_rows > 0 && cfg->sweep_kernel != HSG_SWEEP_AUTO))
    return fail(HSG_EINVAL, "band_rows must be 0, or > 0 with the fused sweep");
  if (cfg->persistent < 0 || cfg->persistent > 2) return fail(HSG_EINVAL, "persistent must be 0, 1 or 2");
  if (cfg->persistent) {
    if (cfg->n_temps > kMaxTempsResident) return fail(HSG_EINVAL, "persistent steps need n_temps <= 64");
    if (cfg->layout == HSG_LAYOUT_BATCHED && cfg->n_temps % 2 != 0)
      return fail(HSG_EINVAL, "persistent steps need n_temps to be a multiple of the lattices per element");
    // the smallest resident unit is one lattice group (V lattices)
    const size_t vl = cfg->layout == HSG_LAYOUT_BATCHED ? 2 : 1;
    for (int s = 0; s < cfg->n_samples; ++s) {
      const size_t Ls = cfg->L[s];
      if (12 * vl * Ls * Ls * Ls > 224 * 1024)
        return fail(HSG_EINVAL, "a lattice group (12 V L^3 bytes) does not fit in shared memory");
    }
  }
  for (int s = 0; s < cfg->n_samples; ++s) {
    const int L = cfg->L[s];
    if (L < 4 || L > 512 || (L & 1)) return fail(HSG_EINVAL, "each L must be even and in [4, 512]");
  }
  for (int k = 0; k < cfg->n_temps; ++k) {
    if (!(cfg->beta[k] >= 0.0) || !(cfg->beta[k] < 1e300))
      return fail(HSG_EINVAL, "beta must be finite and >= 0");
    if (k > 0 && !(cfg->beta[k] > cfg->beta[k - 1])) return fail(HSG_EINVAL, "beta must be strictly increasing");
  }
  const long long R = static_cast<long long>(cfg->n_replicas) * cfg->n_temps;
  const int V = cfg->layout == HSG_LAYOUT_BATCHED ? 2 : 1;
  if (R % V != 0) return fail(HSG_EINVAL, "the batched layout needs an even number of lattices per sample");
  if (cfg->fused_groups < 0 || cfg->fused_groups > 2 ||
      (cfg->fused_groups > 0 && cfg->sweep_kernel != HSG_SWEEP_AUTO))
    return fail(HSG_EINVAL, "fused_groups must be 0, or 1 or 2 with the fused sweep");
  if (cfg->fused_groups == 2 && (V != 2 || R % 4 != 0))
    return fail(HSG_EINVAL, "fused_groups = 2 needs the batched layout and a multiple of 4 lattices per sample");
  if (R * cfg->n_samples > 0x7fffffffLL) return fail(HSG_EINVAL, "too many lattices");

  hsg_ctx* h = new (std::nothrow) hsg_ctx();
  if (!h) return fail(HSG_ENOMEM, "host allocation failed");
  h->S = cfg->n_samples;
  h->n_rep = cfg->n_replicas;
  h->NT = cfg->n_temps;
  h->R = static_cast<int>(R);
  h->V = V;
  h->prec = cfg->coupling_prec;
  h->bimodal_D = cfg->coupling_prec == HSG_BIMODAL ? static_cast<float>(cfg->bimodal_D) : 0.0f;
  h->layout = cfg->layout;
  h->n_or = cfg->n_or;
  h->measure_every = cfg->measure_every;
  h->seed = cfg->seed;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  h->timeout_cycles = cfg->timeout_cycles > 0 ? cfg->timeout_cycles : 4000000000LL;
  h->sweep_kernel = cfg->sweep_kernel;
  h->persistent = cfg->persistent != 0;
  h->persistent_joint = cfg->persistent == 2;
  h->launch_sink = &h->launches;
  h->Ls.assign(cfg->L, cfg->L + cfg->n_samples);
  h->beta.assign(cfg->beta, cfg->beta + cfg->n_temps);

  auto bail = [&](hsg_status st) {
    std::string msg = g_last_error;
    free_ctx(h);
    g_last_error = msg;
    return st;
  };

  // Buckets: samples grouped by L, in order of first appearance.
  h->sample_bucket.assign(h->S, -1);
  h->sample_local.assign(h->S, -1);
  for (int s = 0; s < h->S; ++s) {
    int bi = -1;
    for (size_t j = 0; j < h->buckets.size(); ++j)
      if (h->buckets[j].L == h->Ls[s]) bi = static_cast<int>(j);
    if (bi < 0) {
      h->buckets.emplace_back();
      bi = static_cast<int>(h->buckets.size()) - 1;
      h->buckets[bi].L = h->Ls[s];
    }
    h->sample_bucket[s] = bi;
    h->sample_local[s] = static_cast<int>(h->buckets[bi].samples.size());
    h->buckets[bi].samples.push_back(s);
  }

  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fail(HSG_ECUDA, "cudaStreamCreate failed");
    return bail(HSG_ECUDA);
  }

  size_t max_N = 0, max_fused_smem = 0;
  for (Bucket& b : h->buckets) {
    b.N = b.L * b.L * b.L;
    b.S_b = static_cast<int>(b.samples.size());
    b.G = h->R / V;
    b.sweep_chunks = (b.N / 2 + kSweepThreads - 1) / kSweepThreads;
    b.gp_or = b.gp_hb = cfg->fused_groups > 0 ? cfg->fused_groups : 1;
    b.fused = (h->sweep_kernel == HSG_SWEEP_AUTO) &&
              plan_fused(b.L, V, b.gp_or, fused_max_threads(V, h->prec, b.gp_or), cfg->band_rows,
                         &b.band_rows, &b.fused_smem);
    if ((cfg->band_rows > 0 || cfg->fused_groups > 0) && !b.fused) {
      fail(HSG_EINVAL, "band_rows / fused_groups do not tile L = " + std::to_string(b.L) + " within the limits");
      return bail(HSG_EINVAL);
    }
    b.n_bands = b.fused ? b.L / b.band_rows : 0;
    // the shared-memory limit is a property of the kernel, not of the bucket:
    // raise it to what the largest tiling in this context needs
    if (b.fused) max_fused_smem = std::max(max_fused_smem, b.fused_smem);
    b.P = (h->n_rep + 1) / 2;
    const int units = b.S_b * h->NT * b.P;
    const int by_size = std::max(1, b.N / (kMeasureThreads * 16));
    const int by_fill = std::max(1, (2 * 148 + units - 1) / units);
    // small lattices (N < 4096): one warp per unit (m_chunks = 1)
    b.m_warp = b.N < kMeasureThreads * 16;
    b.m_chunks = b.m_warp ? 1 : std::max(1, std::min(by_size, by_fill));
    max_N = std::max<size_t>(max_N, b.N);
    const size_t n_spin = static_cast<size_t>(b.S_b) * h->R * 3 * b.N;
    hsg_status st;
    if ((st = dalloc(&b.d_samples, b.S_b)) != HSG_OK) return bail(st);
    // The fused sweep reads one spin buffer and writes the other at nearly
    // the same offsets.  Both share one allocation, the second starting half
    // a 2 MiB page (mod 2 MiB) after the first: with the two at equal offsets
    // modulo 2 MiB (separate allocations) the L = 64 overrelaxation sweep
    // ran 2.8% slower on some boxes and builds.
    size_t pad = 0;
    if (b.fused) {
      const size_t page = size_t(2) << 20, rem = (n_spin * sizeof(float)) % page;
      pad = ((page / 2 + page - rem) % page) / sizeof(float);
    }
    if ((st = dalloc(&b.d_spins[0], b.fused ? 2 * n_spin + pad : n_spin)) != HSG_OK) return bail(st);
    if (b.fused) b.d_spins[1] = b.d_spins[0] + n_spin + pad;
    const size_t jbytes = static_cast<size_t>(b.S_b) * 3 * b.N * bond_bytes(h->prec);
    if ((st = dalloc(reinterpret_cast<char**>(&b.d_J), jbytes)) != HSG_OK) return bail(st);
    if ((st = dalloc(&b.d_epart, static_cast<size_t>(b.S_b) * h->R * std::max(b.sweep_chunks, b.n_bands))) != HSG_OK)
      return bail(st);
    if ((st = dalloc(&b.d_mpart, static_cast<size_t>(units) * b.m_chunks * kNQ)) != HSG_OK) return bail(st);
    if ((st = dalloc(&b.d_phase, 2 * static_cast<size_t>(b.L))) != HSG_OK) return bail(st);
    if (cudaMemcpy(b.d_samples, b.samples.data(), sizeof(int) * b.S_b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b.d_J, 0, jbytes) != cudaSuccess) {
      cudaGetLastError();
      fail(HSG_ECUDA, "initialising bucket buffers failed");
      return bail(HSG_ECUDA);
    }
    std::vector<float> ph(2 * b.L);
    for (int x = 0; x < b.L; ++x) {
      const double a = 2.0 * 3.14159265358979323846 * x / b.L;
      ph[2 * x] = static_cast<float>(std::cos(a));
      ph[2 * x + 1] = static_cast<float>(std::sin(a));
    }
    if (cudaMemcpy(b.d_phase, ph.data(), sizeof(float) * 2 * b.L, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      fail(HSG_ECUDA, "phase table upload failed");
      return bail(HSG_ECUDA);
    }
    const size_t per_block = static_cast<size_t>(b.N) * V;
    k_fill_spins<<<static_cast<unsigned>((n_spin + 255) / 256), 256>>>(b.d_spins[0], per_block, n_spin);
  }

  if (max_fused_smem > 0 && allow_fused_smem_all(V, h->prec, max_fused_smem) != HSG_OK) return bail(HSG_ECUDA);
  if (h->persistent) {
    hsg_status ps = plan_persistent(h);
    if (ps == HSG_OK && h->persistent_joint) ps = plan_joint(h);
    if (ps != HSG_OK) return bail(ps);
  }
  {
    // both measurement kernels keep their accumulators in shared memory
    size_t msmem = 0;
    for (const Bucket& b : h->buckets) msmem = std::max(msmem, measure_block_smem(b.L));
    if (msmem > 0) {
      const hsg_status e = dispatch(h->V, h->prec, [&](auto v, auto pr) {
        constexpr int VV = decltype(v)::value, P = decltype(pr)::value;
        const hsg_status a = raise_smem_limit(reinterpret_cast<const void*>(k_measure<VV, P>), msmem);
        return a != HSG_OK ? a : raise_smem_limit(reinterpret_cast<const void*>(k_measure_warp<VV, P>), msmem);
      });
      if (e != HSG_OK) return bail(e);
    }
  }
  const size_t S = h->S, NT = h->NT;
  hsg_status st;
  if ((st = dalloc(&h->d_perm, S * h->n_rep * NT)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_temp_of, S * h->R)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_beta, NT)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_beta_f, NT)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_E, S * h->R)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_obs, S * NT * HSG_NOBS)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_counts, S * NT)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_pt_acc, S * h->n_rep * acc_stride(h))) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_counters, 2)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_status, 1)) != HSG_OK) return bail(st);
  if ((st = dalloc(&h->d_stage, 3 * max_N)) != HSG_OK) return bail(st);

  std::vector<int> perm(S * h->n_rep * NT), temp_of(S * h->R);
  for (size_t s = 0; s < S; ++s)
    for (int r = 0; r < h->n_rep; ++r)
      for (size_t k = 0; k < NT; ++k) {
        const int slot = r * static_cast<int>(NT) + static_cast<int>(k);
        perm[(s * h->n_rep + r) * NT + k] = slot;
        temp_of[s * h->R + slot] = static_cast<int>(k);
      }
  std::vector<float> bf(NT);
  for (size_t k = 0; k < NT; ++k) bf[k] = static_cast<float>(h->beta[k]);
  if (cudaMemcpy(h->d_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_temp_of, temp_of.data(), sizeof(int) * temp_of.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_beta, h->beta.data(), sizeof(double) * NT, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_beta_f, bf.data(), sizeof(float) * NT, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->d_E, 0, sizeof(double) * S * h->R) != cudaSuccess ||
      cudaMemset(h->d_obs, 0, sizeof(double) * S * NT * HSG_NOBS) != cudaSuccess ||
      cudaMemset(h->d_counts, 0, sizeof(long long) * S * NT) != cudaSuccess ||
      cudaMemset(h->d_pt_acc, 0, sizeof(long long) * S * h->n_rep * acc_stride(h)) != cudaSuccess ||
      cudaMemset(h->d_counters, 0, sizeof(uint32_t) * 2) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    fail(HSG_ECUDA, std::string("initialising context buffers failed: ") + cudaGetErrorString(e));
    return bail(HSG_ECUDA);
  }
  *out = h;
  return HSG_OK;
}

void hsg_destroy(hsg_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_ctx(h);
}

hsg_status hsg_synchronize(hsg_t h) {
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

hsg_status hsg_selftest_wait_timeout(hsg_t h, long long timeout_cycles) {
  if (!h || timeout_cycles <= 0) return fail(HSG_EINVAL, "bad handle or timeout_cycles <= 0");
  Bucket* fb = nullptr;
  for (Bucket& b : h->buckets)
    if (b.fused) fb = &b;
  if (!fb) return fail(HSG_ESTATE, "no bucket uses the fused sweep, which holds the bounded waits");
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_TRY(status_check(h));
  HSG_TRY(launch_fused<kOR>(h, *fb, false, h->stream, true, timeout_cycles));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

// Device address of the couplings of context sample `sample`.
static char* sample_coupling_ptr(hsg_t h, int sample) {
  const Bucket& b = h->buckets[h->sample_bucket[sample]];
  const size_t per_sample = 3 * static_cast<size_t>(b.N) * bond_bytes(h->prec);
  return static_cast<char*>(b.d_J) + static_cast<size_t>(h->sample_local[sample]) * per_sample;
}

// One bimodal bond as its six FP32 entries (the kernels' decoding).
static void decode_bimodal_host(uint8_t bits, float D, float* j) {
  const float eps = (bits & 1u) ? -1.0f : 1.0f;
  float d[6];
  for (int k = 0; k < 6; ++k) d[k] = ((bits >> (k + 1)) & 1u) ? -D : D;
  j[0] = eps + d[0];
  j[1] = eps + d[1];
  j[2] = eps + d[2];
  j[3] = d[3];
  j[4] = d[4];
  j[5] = d[5];
}

// Largest staging buffer for whole-sample transfers (floats): 256 MiB.
constexpr size_t kBigStageFloats = static_cast<size_t>(64) << 20;

// Makes d_big hold min(want, kBigStageFloats) floats (growing it after the
// stream has drained); returns that count in *got.
static hsg_status big_stage(hsg_t h, size_t want, size_t* got) {
  const size_t n = std::min(want, kBigStageFloats);
  if (h->big_cap < n) {
    HSG_CUDA(cudaStreamSynchronize(h->stream));
    cudaFree(h->d_big);
    h->d_big = nullptr;
    h->big_cap = 0;
    HSG_TRY(dalloc(&h->d_big, n));
    h->big_cap = n;
  }
  *got = n;
  return HSG_OK;
}

hsg_status hsg_set_couplings(hsg_t h, int sample, const float* J6) {
  NvtxRange nvtx_range("hsg_set_couplings");
  if (!h || !J6) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  if (h->prec == HSG_BIMODAL) return fail(HSG_EINVAL, "bimodal contexts take hsg_set_couplings_bimodal");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const long long N = b.N;
  // FP32 [N][3][6] to the device in chunks of whole sites; the packing kernel
  // permutes them to storage order and rounds to the storage precision
  size_t cap = 0;
  HSG_TRY(big_stage(h, 18 * static_cast<size_t>(N), &cap));
  const long long per = static_cast<long long>(cap / 18);
  void* dst = sample_coupling_ptr(h, sample);
  for (long long i0 = 0; i0 < N; i0 += per) {
    const long long n = std::min(per, N - i0);
    HSG_CUDA(cudaMemcpyAsync(h->d_big, J6 + 18 * i0, sizeof(float) * 18 * n, cudaMemcpyHostToDevice, h->stream));
    const unsigned blocks = static_cast<unsigned>((3 * n + 255) / 256);
    if (h->prec == HSG_F32) k_pack_couplings<kPrecF32><<<blocks, 256, 0, h->stream>>>(h->d_big, dst, b.L, i0, n);
    else k_pack_couplings<kPrecF16><<<blocks, 256, 0, h->stream>>>(h->d_big, dst, b.L, i0, n);
    HSG_CUDA(cudaGetLastError());
  }
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_set_couplings_bimodal(hsg_t h, int sample, const uint8_t* bits) {
  if (!h || !bits) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  if (h->prec != HSG_BIMODAL) return fail(HSG_EINVAL, "the context does not store bimodal couplings");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const size_t N = b.N;
  std::vector<uint8_t> buf(3 * N);
  for (size_t i = 0; i < N; ++i)
    for (int mu = 0; mu < 3; ++mu) {
      const uint8_t v = bits[i * 3 + mu];
      if (v & 0x80u) return fail(HSG_EINVAL, "bit 7 of a bimodal bond is set");
      buf[mu * N + storage_site(i, b.L)] = v;
    }
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_CUDA(cudaMemcpy(sample_coupling_ptr(h, sample), buf.data(), buf.size(), cudaMemcpyHostToDevice));
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_get_couplings_bimodal(hsg_t h, int sample, uint8_t* bits_out) {
  if (!h || !bits_out) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  if (h->prec != HSG_BIMODAL) return fail(HSG_EINVAL, "the context does not store bimodal couplings");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const size_t N = b.N;
  std::vector<uint8_t> buf(3 * N);
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_CUDA(cudaMemcpy(buf.data(), sample_coupling_ptr(h, sample), buf.size(), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < N; ++i)
    for (int mu = 0; mu < 3; ++mu) bits_out[i * 3 + mu] = buf[mu * N + storage_site(i, b.L)];
  return HSG_OK;
}

hsg_status hsg_get_couplings(hsg_t h, int sample, float* J6) {
  if (!h || !J6) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const size_t N = b.N;
  std::vector<char> buf(3 * N * bond_bytes(h->prec));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_CUDA(cudaMemcpy(buf.data(), sample_coupling_ptr(h, sample), buf.size(), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < N; ++i)
    for (int mu = 0; mu < 3; ++mu) {
      const size_t d = mu * N + storage_site(i, b.L);
      float* out = J6 + (i * 3 + mu) * 6;
      if (h->prec == HSG_BIMODAL) {
        decode_bimodal_host(reinterpret_cast<const uint8_t*>(buf.data())[d], h->bimodal_D, out);
        continue;
      }
      for (int e = 0; e < 6; ++e) {
        if (h->prec == HSG_F32) out[e] = reinterpret_cast<const float*>(buf.data())[d * 6 + e];
        else out[e] = __half2float(reinterpret_cast<const __half*>(buf.data())[d * 8 + e]);
      }
    }
  return HSG_OK;
}

static hsg_status spin_slot_args(hsg_t h, int sample, int slot) {
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  HSG_TRY(check_sample(h, sample));
  if (slot < 0 || slot >= h->R) return fail(HSG_EINVAL, "slot out of range");
  return HSG_OK;
}

hsg_status hsg_set_spins(hsg_t h, int sample, int slot, const float* s) {
  HSG_TRY(spin_slot_args(h, sample, slot));
  if (!s) return fail(HSG_EINVAL, "spins pointer is NULL");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  float* base = b.d_spins[b.cur] + (static_cast<size_t>(sb) * b.G + slot / h->V) * 3 * static_cast<size_t>(b.N) * h->V;
  HSG_CUDA(cudaMemcpyAsync(h->d_stage, s, sizeof(float) * 3 * b.N, cudaMemcpyHostToDevice, h->stream));
  k_scatter_spins<<<(b.N + 255) / 256, 256, 0, h->stream>>>(h->d_stage, base, b.L, h->V, slot % h->V);
  HSG_CUDA(cudaGetLastError());
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_get_spins(hsg_t h, int sample, int slot, float* s_out) {
  HSG_TRY(spin_slot_args(h, sample, slot));
  if (!s_out) return fail(HSG_EINVAL, "output pointer is NULL");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  const float* base =
      b.d_spins[b.cur] + (static_cast<size_t>(sb) * b.G + slot / h->V) * 3 * static_cast<size_t>(b.N) * h->V;
  k_gather_spins<<<(b.N + 255) / 256, 256, 0, h->stream>>>(base, h->d_stage, b.L, h->V, slot % h->V);
  HSG_CUDA(cudaGetLastError());
  HSG_CUDA(cudaMemcpyAsync(s_out, h->d_stage, sizeof(float) * 3 * b.N, cudaMemcpyDeviceToHost, h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

hsg_status hsg_set_spins_sample(hsg_t h, int sample, const float* s) {
  NvtxRange nvtx_range("hsg_set_spins_sample");
  if (!h || !s) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  float* spins_s = b.d_spins[b.cur] + static_cast<size_t>(sb) * b.G * 3 * static_cast<size_t>(b.N) * h->V;
  const long long total = static_cast<long long>(h->R) * b.N;  // (slot, site) records of 3 floats
  size_t cap = 0;
  HSG_TRY(big_stage(h, 3 * static_cast<size_t>(total), &cap));
  const long long per = static_cast<long long>(cap / 3);
  for (long long q0 = 0; q0 < total; q0 += per) {
    const long long n = std::min(per, total - q0);
    HSG_CUDA(cudaMemcpyAsync(h->d_big, s + 3 * q0, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    k_scatter_spins_many<<<static_cast<unsigned>((n + 255) / 256), 256, 0, h->stream>>>(h->d_big, spins_s, b.L,
                                                                                          h->V, q0, n);
    HSG_CUDA(cudaGetLastError());
  }
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_get_spins_sample(hsg_t h, int sample, float* s_out) {
  NvtxRange nvtx_range("hsg_get_spins_sample");
  if (!h || !s_out) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  const float* spins_s = b.d_spins[b.cur] + static_cast<size_t>(sb) * b.G * 3 * static_cast<size_t>(b.N) * h->V;
  const long long total = static_cast<long long>(h->R) * b.N;
  size_t cap = 0;
  HSG_TRY(big_stage(h, 3 * static_cast<size_t>(total), &cap));
  const long long per = static_cast<long long>(cap / 3);
  for (long long q0 = 0; q0 < total; q0 += per) {
    const long long n = std::min(per, total - q0);
    k_gather_spins_many<<<static_cast<unsigned>((n + 255) / 256), 256, 0, h->stream>>>(spins_s, h->d_big, b.L, h->V,
                                                                                         q0, n);
    HSG_CUDA(cudaGetLastError());
    HSG_CUDA(cudaMemcpyAsync(s_out + 3 * q0, h->d_big, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  }
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

hsg_status hsg_set_spins_device(hsg_t h, int sample, int slot, const float* d_s) {
  HSG_TRY(spin_slot_args(h, sample, slot));
  if (!d_s) return fail(HSG_EINVAL, "spins pointer is NULL");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  float* base = b.d_spins[b.cur] + (static_cast<size_t>(sb) * b.G + slot / h->V) * 3 * static_cast<size_t>(b.N) * h->V;
  k_scatter_spins<<<(b.N + 255) / 256, 256, 0, h->stream>>>(d_s, base, b.L, h->V, slot % h->V);
  HSG_CUDA(cudaGetLastError());
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_get_spins_device(hsg_t h, int sample, int slot, float* d_out) {
  HSG_TRY(spin_slot_args(h, sample, slot));
  if (!d_out) return fail(HSG_EINVAL, "output pointer is NULL");
  Bucket& b = h->buckets[h->sample_bucket[sample]];
  const int sb = h->sample_local[sample];
  const float* base =
      b.d_spins[b.cur] + (static_cast<size_t>(sb) * b.G + slot / h->V) * 3 * static_cast<size_t>(b.N) * h->V;
  k_gather_spins<<<(b.N + 255) / 256, 256, 0, h->stream>>>(base, d_out, b.L, h->V, slot % h->V);
  HSG_CUDA(cudaGetLastError());
  return HSG_OK;
}

hsg_status hsg_sweep_hb(hsg_t h, int n) {
  NvtxRange nvtx_range("hsg_sweep_hb");
  if (!h || n < 0) return fail(HSG_EINVAL, "bad handle or n < 0");
  for (int s = 0; s < n; ++s) {
    HSG_TRY(enqueue_hb_sweep(h, h->stream));
    HSG_TRY(enqueue_bump(h, 1, 0, h->stream));
    h->counters[0] += 1;
  }
  if (n > 0) h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_sweep_or(hsg_t h, int n) {
  NvtxRange nvtx_range("hsg_sweep_or");
  if (!h || n < 0) return fail(HSG_EINVAL, "bad handle or n < 0");
  if (n == 0) return HSG_OK;
  HSG_TRY(enqueue_or_sweeps(h, n, h->stream));
  h->energy_valid = true;
  return HSG_OK;
}

// Shared memory of the sequential sweep: one lattice group in natural order.
static constexpr size_t kSeqMaxSmem = 200 * 1024;

hsg_status hsg_sweep_or_sequential(hsg_t h, int n) {
  NvtxRange nvtx_range("hsg_sweep_or_sequential");
  if (!h || n < 0) return fail(HSG_EINVAL, "bad handle or n < 0");
  size_t smem_max = 0;
  for (const Bucket& b : h->buckets) {
    const size_t smem = sizeof(float) * 3 * static_cast<size_t>(b.N) * h->V;
    if (smem > kSeqMaxSmem)
      return fail(HSG_EINVAL, "sequential sweep: a lattice group of L = " + std::to_string(b.L) +
                                  " does not fit in shared memory (12 V L^3 <= 200 KiB)");
    smem_max = std::max(smem_max, smem);
  }
  if (n == 0) return HSG_OK;
  HSG_TRY((dispatch(h->V, h->prec, [&](auto v, auto pr) {
    return raise_smem_limit(reinterpret_cast<const void*>(k_sweep_or_seq<decltype(v)::value, decltype(pr)::value>),
                            smem_max);
  })));
  for (const Bucket& b : h->buckets) {
    SeqParams p;
    p.b = view(b);
    p.b.D = h->bimodal_D;
    p.n_sweeps = n;
    const size_t smem = sizeof(float) * 3 * static_cast<size_t>(b.N) * h->V;
    const unsigned grid = static_cast<unsigned>(b.S_b * b.G);
    *h->launch_sink += 1;
    dispatch(h->V, h->prec, [&](auto v, auto pr) {
      k_sweep_or_seq<decltype(v)::value, decltype(pr)::value><<<grid, kSeqThreads, smem, h->stream>>>(p);
      return 0;
    });
    HSG_CUDA(cudaGetLastError());
  }
  h->energy_valid = false;
  return HSG_OK;
}

hsg_status hsg_energy(hsg_t h) {
  NvtxRange nvtx_range("hsg_energy");
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  HSG_TRY(enqueue_energy(h, h->stream));
  h->energy_valid = true;
  return HSG_OK;
}

hsg_status hsg_get_energies(hsg_t h, double* E_out) {
  if (!h || !E_out) return fail(HSG_EINVAL, "NULL argument");
  if (!h->energy_valid) HSG_TRY(hsg_energy(h));
  HSG_CUDA(cudaMemcpyAsync(E_out, h->d_E, sizeof(double) * h->S * h->R, cudaMemcpyDeviceToHost, h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

hsg_status hsg_set_energies(hsg_t h, const double* E) {
  if (!h || !E) return fail(HSG_EINVAL, "NULL argument");
  HSG_CUDA(cudaMemcpyAsync(h->d_E, E, sizeof(double) * h->S * h->R, cudaMemcpyHostToDevice, h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  h->energy_valid = true;
  return HSG_OK;
}

hsg_status hsg_pt_swap(hsg_t h) {
  NvtxRange nvtx_range("hsg_pt_swap");
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  if (!h->energy_valid) HSG_TRY(hsg_energy(h));
  if (h->NT > 1) HSG_TRY(enqueue_pt(h, h->stream));
  HSG_TRY(enqueue_bump(h, 0, 1, h->stream));
  h->counters[1] += 1;
  return HSG_OK;
}

hsg_status hsg_get_perm(hsg_t h, int* perm_out) {
  if (!h || !perm_out) return fail(HSG_EINVAL, "NULL argument");
  HSG_CUDA(cudaMemcpyAsync(perm_out, h->d_perm, sizeof(int) * h->S * h->n_rep * h->NT, cudaMemcpyDeviceToHost,
                           h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return HSG_OK;
}

hsg_status hsg_set_perm(hsg_t h, const int* perm) {
  if (!h || !perm) return fail(HSG_EINVAL, "NULL argument");
  const int NT = h->NT;
  std::vector<int> temp_of(static_cast<size_t>(h->S) * h->R);
  for (int s = 0; s < h->S; ++s)
    for (int r = 0; r < h->n_rep; ++r) {
      std::vector<char> seen(NT, 0);
      for (int k = 0; k < NT; ++k) {
        const int slot = perm[(static_cast<size_t>(s) * h->n_rep + r) * NT + k];
        if (slot < r * NT || slot >= (r + 1) * NT || seen[slot - r * NT])
          return fail(HSG_EINVAL, "perm must map each replica's temperatures onto that replica's slots");
        seen[slot - r * NT] = 1;
        temp_of[static_cast<size_t>(s) * h->R + slot] = k;
      }
    }
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_CUDA(cudaMemcpy(h->d_perm, perm, sizeof(int) * h->S * h->n_rep * NT, cudaMemcpyHostToDevice));
  HSG_CUDA(cudaMemcpy(h->d_temp_of, temp_of.data(), sizeof(int) * temp_of.size(), cudaMemcpyHostToDevice));
  return HSG_OK;
}

hsg_status hsg_get_pt_accepts(hsg_t h, long long* acc_out) {
  if (!h || !acc_out) return fail(HSG_EINVAL, "NULL argument");
  HSG_CUDA(cudaMemcpyAsync(acc_out, h->d_pt_acc, sizeof(long long) * h->S * h->n_rep * acc_stride(h),
                           cudaMemcpyDeviceToHost, h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return HSG_OK;
}

hsg_status hsg_measure(hsg_t h) {
  NvtxRange nvtx_range("hsg_measure");
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  if (!h->energy_valid) HSG_TRY(hsg_energy(h));
  return enqueue_measure(h, h->stream);
}

hsg_status hsg_run_steps(hsg_t h, int n_steps) {
  NvtxRange nvtx_range("hsg_run_steps");
  if (!h || n_steps < 0) return fail(HSG_EINVAL, "bad handle or n_steps < 0");
  if (n_steps == 0) return HSG_OK;
  if (h->persistent) {
    int left = n_steps;
    while (left > 0) {
      // bounded launches: at most kMaxStepsPerLaunch steps each, one when
      // replica sets span several CTAs (PT between launches)
      int k = std::min(left, h->res_split ? 1 : kMaxStepsPerLaunch);
      if (h->measure_every > 0) {
        const uint64_t m = static_cast<uint64_t>(h->measure_every);
        k = static_cast<int>(std::min<uint64_t>(k, m - h->counters[2] % m));
      }
      HSG_TRY(enqueue_persistent(h, k, h->stream));
      h->counters[0] += k;
      h->counters[1] += k;
      h->counters[2] += k;
      left -= k;
      if (h->measure_every > 0 && h->counters[2] % static_cast<uint64_t>(h->measure_every) == 0)
        HSG_TRY(enqueue_measure(h, h->stream));
    }
    h->energy_valid = true;
    return HSG_OK;
  }
  // sweeps per step: one heat-bath sweep plus n_or overrelaxation sweeps;
  // each fused sweep flips the buffer index
  const int flips = (1 + h->n_or) & 1;
  for (int s = 0; s < n_steps; ++s) {
    const uint64_t next = h->counters[2] + 1;
    const int m = (h->measure_every > 0 && (next % static_cast<uint64_t>(h->measure_every)) == 0) ? 1 : 0;
    const int par = fused_parity(h);
    if (!h->g_step[par][m]) HSG_TRY(capture_graph(h, par, m != 0, &h->g_step[par][m], &h->g_step_launches[par][m]));
    HSG_CUDA(cudaGraphLaunch(h->g_step[par][m], h->stream));
    h->launches += h->g_step_launches[par][m];
    for (Bucket& b : h->buckets)
      if (b.fused) b.cur ^= flips;
    h->counters[0] += 1;
    h->counters[1] += 1;
    h->counters[2] = next;
  }
  h->energy_valid = true;
  return HSG_OK;
}

hsg_status hsg_read_observables(hsg_t h, double* obs_out, long long* counts_out) {
  NvtxRange nvtx_range("hsg_read_observables");
  if (!h || !obs_out) return fail(HSG_EINVAL, "NULL argument");
  const size_t n = static_cast<size_t>(h->S) * h->NT;
  HSG_CUDA(cudaMemcpyAsync(obs_out, h->d_obs, sizeof(double) * n * HSG_NOBS, cudaMemcpyDeviceToHost, h->stream));
  if (counts_out)
    HSG_CUDA(cudaMemcpyAsync(counts_out, h->d_counts, sizeof(long long) * n, cudaMemcpyDeviceToHost, h->stream));
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  return status_check(h);
}

hsg_status hsg_reset_observables(hsg_t h) {
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  const size_t n = static_cast<size_t>(h->S) * h->NT;
  HSG_CUDA(cudaMemsetAsync(h->d_obs, 0, sizeof(double) * n * HSG_NOBS, h->stream));
  HSG_CUDA(cudaMemsetAsync(h->d_counts, 0, sizeof(long long) * n, h->stream));
  HSG_CUDA(cudaMemsetAsync(h->d_pt_acc, 0, sizeof(long long) * h->S * h->n_rep * acc_stride(h), h->stream));
  return HSG_OK;
}

hsg_status hsg_get_counters(hsg_t h, uint64_t out[3]) {
  if (!h || !out) return fail(HSG_EINVAL, "NULL argument");
  for (int j = 0; j < 3; ++j) out[j] = h->counters[j];
  return HSG_OK;
}

hsg_status hsg_get_sweep_plan(hsg_t h, int sample, int out[5]) {
  if (!h || !out) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  const Bucket& b = h->buckets[h->sample_bucket[sample]];
  out[0] = b.fused ? 1 : 0;
  out[1] = b.fused ? b.band_rows : 0;
  out[2] = b.fused ? 1 : 2;
  out[3] = b.fused ? b.gp_or : 0;
  out[4] = b.fused ? b.gp_hb : 0;
  return HSG_OK;
}

hsg_status hsg_get_resident_plan(hsg_t h, int sample, int out[6]) {
  if (!h || !out) return fail(HSG_EINVAL, "NULL argument");
  HSG_TRY(check_sample(h, sample));
  const Bucket& b = h->buckets[h->sample_bucket[sample]];
  out[0] = h->persistent ? b.res_js : 0;
  out[1] = h->persistent ? b.res_gp : 0;
  out[2] = h->persistent ? b.res_threads : 0;
  out[3] = h->persistent ? b.res_gsub : 0;
  out[4] = h->persistent ? b.res_sets : 0;
  out[5] = h->res_pair ? 1 : 0;
  return HSG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: the candidate tilings of each bucket, timed on the context's own
// couplings and spins without changing its state, the fastest kept and
// remembered for the process.
// ---------------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;
// (kind, L, V, precision, N_T, bond residency) -> (band rows, overrelaxation
// groups, heat-bath groups) or (gp, threads, 0)
std::map<std::array<int, 6>, std::array<int, 3>> g_tune_cache;

bool tune_lookup(const std::array<int, 6>& key, std::array<int, 3>* val) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const auto it = g_tune_cache.find(key);
  if (it == g_tune_cache.end()) return false;
  *val = it->second;
  return true;
}

void tune_store(const std::array<int, 6>& key, const std::array<int, 3>& val) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = val;
}

// Mean device time (ms) of `reps` calls of `launch` after one untimed call.
template <typename F>
hsg_status time_ms(hsg_ctx* h, cudaEvent_t e0, cudaEvent_t e1, int reps, F&& launch, float* ms) {
  HSG_TRY(launch());
  HSG_CUDA(cudaEventRecord(e0, h->stream));
  for (int r = 0; r < reps; ++r) HSG_TRY(launch());
  HSG_CUDA(cudaEventRecord(e1, h->stream));
  HSG_CUDA(cudaEventSynchronize(e1));
  HSG_CUDA(cudaEventElapsedTime(ms, e0, e1));
  *ms /= static_cast<float>(reps);
  return status_check(h);
}

// Streaming buckets: every band height that tiles L (and whole planes)
// within the fused kernel's limits, timed as overrelaxation sweeps whose
// output buffer is discarded (the input buffer stays the state), and the
// two-pass half-sweeps (band 0), timed on a copy of the state in the other
// buffer.  The two-pass kernel wins where the fused z-march has too few
// CTAs to fill the GPU (few small lattices).
hsg_status tune_fused(hsg_ctx* h, Bucket& b, cudaEvent_t e0, cudaEvent_t e1) {
  const std::array<int, 6> key = {0, b.L, h->V, h->prec, b.S_b * h->R, 0};
  std::array<int, 3> got;
  const bool remembered = tune_lookup(key, &got);
  // two lattice groups per CTA need the batched layout and whole group pairs
  const bool two_groups = (h->V == 2 && h->R % 4 == 0);
  auto set_plan = [&](int band, int gp_or, int gp_hb) -> hsg_status {
    b.band_rows = band;
    b.n_bands = b.L / band;
    b.gp_or = gp_or;
    b.gp_hb = gp_hb;
    b.fused_smem = std::max(fused_smem_bytes(b.L, h->V, gp_or, band), fused_smem_bytes(b.L, h->V, gp_hb, band));
    return allow_fused_smem_all(h->V, h->prec, b.fused_smem);
  };
  if (remembered) {  // nothing to time
    if (got[0] == 0) {
      b.fused = false;
      return HSG_OK;
    }
    return set_plan(got[0], got[1], got[2]);
  }
  // The overrelaxation sweep (n_or of them per step) decides the band height
  // and the two-pass alternative; candidates (band rows, groups per CTA),
  // the current plan first so that ties keep it.
  std::vector<std::array<int, 2>> cands;
  cands.push_back({b.band_rows, b.gp_or});
  for (const int gp : {1, 2}) {
    if (gp == 2 && !two_groups) continue;
    for (int B = 8; B <= b.L; ++B)
      if (b.L % B == 0 && !(B == b.band_rows && gp == b.gp_or)) cands.push_back({B, gp});
  }
  int best_band = b.band_rows, best_gp = b.gp_or;
  float best_ms = -1.0f;
  for (const auto& cand : cands) {
    int br = 0;
    size_t sm = 0;
    if (!plan_fused(b.L, h->V, cand[1], fused_max_threads(h->V, h->prec, cand[1]), cand[0], &br, &sm)) continue;
    HSG_TRY(set_plan(br, cand[1], b.gp_hb));
    float ms = 0.0f;
    HSG_TRY(time_ms(h, e0, e1, 3, [&]() -> hsg_status {
      HSG_TRY(launch_fused<kOR>(h, b, false, h->stream));
      b.cur ^= 1;  // keep reading the state; the other buffer is scratch
      return HSG_OK;
    }, &ms));
    // a new choice must win by 2%, so timing noise does not move the plan
    if (best_ms < 0.0f || ms < 0.98f * best_ms) {
      best_ms = ms;
      best_band = br;
      best_gp = cand[1];
    }
  }
  {  // the two-pass half-sweeps, timed on a copy of the state in the other buffer
    const size_t bytes = sizeof(float) * static_cast<size_t>(b.S_b) * h->R * 3 * b.N;
    HSG_CUDA(cudaMemcpyAsync(b.d_spins[b.cur ^ 1], b.d_spins[b.cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    b.cur ^= 1;
    float ms = 0.0f;
    const hsg_status st = time_ms(h, e0, e1, 3, [&]() -> hsg_status {
      HSG_TRY(launch_half<kOR>(h, b, 0, false, h->stream));
      return launch_half<kOR>(h, b, 1, false, h->stream);
    }, &ms);
    b.cur ^= 1;
    HSG_TRY(st);
    if (best_ms < 0.0f || ms < 0.98f * best_ms) {
      b.fused = false;  // the state stays in the current buffer
      tune_store(key, {0, 1, 1});
      return HSG_OK;
    }
  }
  // The heat-bath sweep keeps the band and picks its own groups per CTA.
  int best_hb = b.gp_hb;
  if (two_groups) {
    float hb_ms = -1.0f;
    for (const int gp : {b.gp_hb, 3 - b.gp_hb}) {
      int br = 0;
      size_t sm = 0;
      if (!plan_fused(b.L, h->V, gp, fused_max_threads(h->V, h->prec, gp), best_band, &br, &sm)) continue;
      HSG_TRY(set_plan(best_band, best_gp, gp));
      float ms = 0.0f;
      HSG_TRY(time_ms(h, e0, e1, 3, [&]() -> hsg_status {
        HSG_TRY(launch_fused<kHB>(h, b, false, h->stream));
        b.cur ^= 1;
        return HSG_OK;
      }, &ms));
      if (hb_ms < 0.0f || ms < 0.98f * hb_ms) {
        hb_ms = ms;
        best_hb = gp;
      }
    }
  }
  HSG_TRY(set_plan(best_band, best_gp, best_hb));
  tune_store(key, {best_band, best_gp, best_hb});
  return HSG_OK;
}

// Resident buckets: groups per work item and threads per CTA, timed as
// stretches of whole steps on scratch copies of the state (spins, labels,
// energies, acceptances), so the context's state is untouched.
hsg_status tune_persistent(hsg_ctx* h, Bucket& b, cudaEvent_t e0, cudaEvent_t e1) {
  const std::array<int, 6> key = {1, b.L, h->V, h->prec, h->NT * 256 + b.res_gsub, b.res_js};
  std::array<int, 3> got;
  if (tune_lookup(key, &got)) {
    b.res_gp = got[0];
    b.res_threads = got[1];
    return HSG_OK;
  }
  int dev = 0, optin = 0;
  HSG_CUDA(cudaGetDevice(&dev));
  HSG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t S = h->S, n_spin = static_cast<size_t>(b.S_b) * h->R * 3 * b.N;
  float* sp = nullptr;
  int *perm = nullptr, *temp_of = nullptr;
  double* E = nullptr;
  long long* acc = nullptr;
  hsg_status st = dalloc(&sp, n_spin);
  if (st == HSG_OK) st = dalloc(&perm, S * h->n_rep * h->NT);
  if (st == HSG_OK) st = dalloc(&temp_of, S * h->R);
  if (st == HSG_OK) st = dalloc(&E, S * h->R);
  if (st == HSG_OK) st = dalloc(&acc, S * h->n_rep * acc_stride(h));
  auto run = [&]() -> hsg_status {
    HSG_CUDA(cudaMemcpyAsync(sp, b.d_spins[b.cur], n_spin * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    HSG_CUDA(cudaMemcpyAsync(perm, h->d_perm, S * h->n_rep * h->NT * sizeof(int), cudaMemcpyDeviceToDevice,
                             h->stream));
    HSG_CUDA(cudaMemsetAsync(acc, 0, S * h->n_rep * acc_stride(h) * sizeof(long long), h->stream));
    // as in the run: one step per launch when replica sets span several CTAs
    const int steps = h->res_split ? 1
                                   : (h->measure_every > 0 && h->measure_every <= kMaxStepsPerLaunch)
                                         ? h->measure_every
                                         : 10;
    PersistentParams p = persistent_params(h, b, steps);
    p.spins = sp;
    p.perm = perm;
    p.temp_of = temp_of;
    p.E = E;
    p.accepted = acc;
    const int gp_max = persistent_gp(h->V, b.res_gsub, b.res_js, b.L);
    float best_ms = -1.0f;
    int best_gp = b.res_gp, best_threads = b.res_threads;
    std::vector<std::array<int, 2>> cands = {{b.res_gp, b.res_threads}};  // current plan first
    for (int gp = 1; gp <= gp_max; ++gp)
      for (const int W : {16, 18, 20, 22, 24, 28, 32})
        if (gp != b.res_gp || 32 * W != b.res_threads) cands.push_back({gp, 32 * W});
    for (const auto& c : cands) {
      void* fn = persistent_kernel(h->V, h->prec, b.res_js, b.L, c[0]);
      cudaFuncAttributes fa;
      HSG_CUDA(cudaFuncGetAttributes(&fa, fn));
      if (c[1] > fa.maxThreadsPerBlock) continue;
      HSG_TRY(raise_smem_limit(fn, static_cast<size_t>(optin) - fa.sharedSizeBytes));
      int occ = 0;
      HSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c[1], b.res_smem));
      if (occ < 1) continue;
      float ms = 0.0f;
      HSG_TRY(time_ms(h, e0, e1, 2, [&]() { return launch_persistent(h, b, p, c[0], c[1], h->stream); }, &ms));
      if (best_ms < 0.0f || ms < 0.98f * best_ms) {
        best_ms = ms;
        best_gp = c[0];
        best_threads = c[1];
      }
    }
    b.res_gp = best_gp;
    b.res_threads = best_threads;
    tune_store(key, {best_gp, best_threads, 0});
    return HSG_OK;
  };
  if (st == HSG_OK) st = run();
  cudaStreamSynchronize(h->stream);
  cudaFree(sp);
  cudaFree(perm);
  cudaFree(temp_of);
  cudaFree(E);
  cudaFree(acc);
  return st;
}

// The joint resident launch: threads per CTA, timed on scratch copies of
// both buckets' spins, labels, energies and acceptances.
hsg_status tune_pair(hsg_ctx* h, cudaEvent_t e0, cudaEvent_t e1) {
  Bucket& A = h->buckets[h->pair_a];
  Bucket& B = h->buckets[h->pair_b];
  const int G_set = h->NT / h->V;
  auto set_b = [&](int k, int jsb) {
    B.res_sets = k;
    B.res_gsub = k * G_set;
    B.res_js = jsb;
  };
  const std::array<int, 6> key = {2, A.L * 1024 + B.L, h->V, h->prec, h->NT * 256 + h->n_rep, 0};
  std::array<int, 3> got;
  if (tune_lookup(key, &got)) {
    set_b(got[0] >> 2, got[0] & 3);
    A.res_threads = got[1];
    B.res_threads = got[2];
    h->pair_threads = std::max(got[1], got[2]);
    return HSG_OK;
  }
  const size_t S = h->S;
  const size_t na = static_cast<size_t>(A.S_b) * h->R * 3 * A.N, nb = static_cast<size_t>(B.S_b) * h->R * 3 * B.N;
  float *spa = nullptr, *spb = nullptr;
  int *perm = nullptr, *temp_of = nullptr;
  double* E = nullptr;
  long long* acc = nullptr;
  hsg_status st = dalloc(&spa, na);
  if (st == HSG_OK) st = dalloc(&spb, nb);
  if (st == HSG_OK) st = dalloc(&perm, S * h->n_rep * h->NT);
  if (st == HSG_OK) st = dalloc(&temp_of, S * h->R);
  if (st == HSG_OK) st = dalloc(&E, S * h->R);
  if (st == HSG_OK) st = dalloc(&acc, S * h->n_rep * acc_stride(h));
  auto run = [&]() -> hsg_status {
    HSG_CUDA(cudaMemcpyAsync(spa, A.d_spins[A.cur], na * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    HSG_CUDA(cudaMemcpyAsync(spb, B.d_spins[B.cur], nb * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    HSG_CUDA(cudaMemcpyAsync(perm, h->d_perm, S * h->n_rep * h->NT * sizeof(int), cudaMemcpyDeviceToDevice,
                             h->stream));
    const int steps = (h->measure_every > 0 && h->measure_every <= kMaxStepsPerLaunch) ? h->measure_every : 10;
    PersistentParams pa = persistent_params(h, A, steps), pb = persistent_params(h, B, steps);
    for (PersistentParams* p : {&pa, &pb}) {
      p->perm = perm;
      p->temp_of = temp_of;
      p->E = E;
      p->accepted = acc;
    }
    pa.spins = spa;
    pb.spins = spb;
    // candidates: bucket b's (sets per CTA, bond residency) and each
    // bucket's warps; the launch takes the larger warp count, and the
    // other bucket's surplus warps sit out its sweeps.  The current plan
    // first, so that ties keep it.
    float best_ms = -1.0f;
    std::array<int, 4> best = {B.res_sets, B.res_js, A.res_threads, B.res_threads};
    std::vector<std::array<int, 4>> cands = {best};
    for (const auto& c : h->pair_cands)
      for (const int ta : {512, 576})
        for (const int tb : {512, 576, 640}) {
          const std::array<int, 4> cand = {c[0], c[1], ta, tb};
          if (cand != best) cands.push_back(cand);
        }
    for (const auto& c : cands) {
      const int t = std::max(c[2], c[3]);
      void* fn = pair_kernel(h->V, h->prec, h->pair_special, c[1]);
      cudaFuncAttributes fa;
      HSG_CUDA(cudaFuncGetAttributes(&fa, fn));
      if (t > fa.maxThreadsPerBlock) continue;
      int occ = 0;
      HSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, h->pair_smem));
      if (occ < 1) continue;
      set_b(c[0], c[1]);
      PersistentParams qb = persistent_params(h, B, pb.steps);
      qb.spins = spb;
      qb.perm = perm;
      qb.temp_of = temp_of;
      qb.E = E;
      qb.accepted = acc;
      PersistentParams qa = pa;
      qa.warps = c[2] / 32;
      qb.warps = c[3] / 32;
      float ms = 0.0f;
      HSG_TRY(time_ms(h, e0, e1, 2, [&]() { return launch_pair(h, qa, qb, t, h->stream); }, &ms));
      if (best_ms < 0.0f || ms < 0.98f * best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    set_b(best[0], best[1]);
    A.res_threads = best[2];
    B.res_threads = best[3];
    h->pair_threads = std::max(best[2], best[3]);
    tune_store(key, {(best[0] << 2) | best[1], best[2], best[3]});
    return HSG_OK;
  };
  if (st == HSG_OK) st = run();
  cudaStreamSynchronize(h->stream);
  cudaFree(spa);
  cudaFree(spb);
  cudaFree(perm);
  cudaFree(temp_of);
  cudaFree(E);
  cudaFree(acc);
  return st;
}

}  // namespace

extern "C" {

hsg_status hsg_autotune(hsg_t h) {
  NvtxRange nvtx_range("hsg_autotune");
  if (!h) return fail(HSG_EINVAL, "handle is NULL");
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_TRY(status_check(h));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HSG_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaGetLastError();
    return fail(HSG_ECUDA, "cudaEventCreate failed");
  }
  uint64_t* sink = h->launch_sink;
  uint64_t scratch_launches = 0;
  h->launch_sink = &scratch_launches;  // tuning launches are not the run's
  hsg_status st = HSG_OK;
  for (Bucket& b : h->buckets) {
    if (st == HSG_OK && b.fused) st = tune_fused(h, b, e0, e1);
    if (st == HSG_OK && h->persistent && !h->res_pair) st = tune_persistent(h, b, e0, e1);
  }
  if (st == HSG_OK && h->res_pair) st = tune_pair(h, e0, e1);
  h->launch_sink = sink;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the captured step graphs hold the old launch shapes
  for (int a = 0; a < 2; ++a)
    for (int m = 0; m < 2; ++m)
      if (h->g_step[a][m]) {
        cudaGraphExecDestroy(h->g_step[a][m]);
        h->g_step[a][m] = nullptr;
      }
  return st;
}

hsg_status hsg_get_launch_count(hsg_t h, uint64_t* out) {
  if (!h || !out) return fail(HSG_EINVAL, "NULL argument");
  *out = h->launches;
  return HSG_OK;
}

hsg_status hsg_set_counters(hsg_t h, const uint64_t in[3]) {
  if (!h || !in) return fail(HSG_EINVAL, "NULL argument");
  const uint32_t dev[2] = {static_cast<uint32_t>(in[0]), static_cast<uint32_t>(in[1])};
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  HSG_CUDA(cudaMemcpy(h->d_counters, dev, sizeof(dev), cudaMemcpyHostToDevice));
  for (int j = 0; j < 3; ++j) h->counters[j] = in[j];
  return HSG_OK;
}

// Checkpoint format: magic, version, a fingerprint of the configuration,
// host counters, then each device array in a fixed order.
static const uint64_t kMagic = 0x31475348u;  // "HSG1"

static void fingerprint(const hsg_ctx* h, std::vector<int64_t>& f) {
  f.clear();
  f.push_back(h->S);
  f.push_back(h->n_rep);
  f.push_back(h->NT);
  f.push_back(h->V);
  f.push_back(h->prec);
  int32_t d_bits;
  std::memcpy(&d_bits, &h->bimodal_D, sizeof d_bits);
  f.push_back(d_bits);
  for (int L : h->Ls) f.push_back(L);
}

namespace {
struct DevArray {
  void* ptr;
  size_t bytes;
};
std::vector<DevArray> checkpoint_arrays(hsg_ctx* h) {
  std::vector<DevArray> a;
  for (Bucket& b : h->buckets) {
    a.push_back({b.d_spins[b.cur], sizeof(float) * static_cast<size_t>(b.S_b) * h->R * 3 * b.N});
    a.push_back({b.d_J, static_cast<size_t>(b.S_b) * 3 * b.N * bond_bytes(h->prec)});
  }
  const size_t S = h->S, NT = h->NT;
  a.push_back({h->d_perm, sizeof(int) * S * h->n_rep * NT});
  a.push_back({h->d_temp_of, sizeof(int) * S * h->R});
  a.push_back({h->d_E, sizeof(double) * S * h->R});
  a.push_back({h->d_obs, sizeof(double) * S * NT * HSG_NOBS});
  a.push_back({h->d_counts, sizeof(long long) * S * NT});
  a.push_back({h->d_pt_acc, sizeof(long long) * S * h->n_rep * acc_stride(h)});
  a.push_back({h->d_counters, sizeof(uint32_t) * 2});
  return a;
}
}  // namespace

hsg_status hsg_save(hsg_t h, const char* path) {
  if (!h || !path) return fail(HSG_EINVAL, "NULL argument");
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(HSG_EIO, std::string("cannot open ") + path);
  std::vector<int64_t> fp;
  fingerprint(h, fp);
  const uint64_t hdr[3] = {kMagic, HSG_VERSION, fp.size()};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(fp.data(), sizeof(int64_t), fp.size(), f) == fp.size() &&
            std::fwrite(h->counters, sizeof(h->counters), 1, f) == 1;
  const int ev = h->energy_valid ? 1 : 0;
  ok = ok && std::fwrite(&ev, sizeof(ev), 1, f) == 1;
  for (const DevArray& d : checkpoint_arrays(h)) {
    if (!ok) break;
    std::vector<char> buf(d.bytes);
    if (cudaMemcpy(buf.data(), d.ptr, d.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      cudaGetLastError();
      return fail(HSG_ECUDA, "device read during checkpoint failed");
    }
    ok = std::fwrite(buf.data(), 1, d.bytes, f) == d.bytes;
  }
  if (std::fclose(f) != 0) ok = false;
  if (!ok) return fail(HSG_EIO, std::string("write failed: ") + path);
  return HSG_OK;
}

hsg_status hsg_load(hsg_t h, const char* path) {
  if (!h || !path) return fail(HSG_EINVAL, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(HSG_EIO, std::string("cannot open ") + path);
  std::vector<int64_t> fp, fp_file;
  fingerprint(h, fp);
  uint64_t hdr[3];
  uint64_t counters[3];
  int ev = 0;
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kMagic && hdr[1] == HSG_VERSION &&
            hdr[2] == fp.size();
  if (ok) {
    fp_file.resize(fp.size());
    ok = std::fread(fp_file.data(), sizeof(int64_t), fp.size(), f) == fp.size() && fp_file == fp;
  }
  if (!ok) {
    std::fclose(f);
    return fail(HSG_EINVAL, "checkpoint does not match this context's configuration");
  }
  ok = std::fread(counters, sizeof(counters), 1, f) == 1 && std::fread(&ev, sizeof(ev), 1, f) == 1;
  std::vector<DevArray> arrays = checkpoint_arrays(h);
  std::vector<std::vector<char>> bufs;
  for (const DevArray& d : arrays) {
    if (!ok) break;
    bufs.emplace_back(d.bytes);
    ok = std::fread(bufs.back().data(), 1, d.bytes, f) == d.bytes;
  }
  std::fclose(f);
  if (!ok) return fail(HSG_EIO, std::string("truncated checkpoint: ") + path);
  HSG_CUDA(cudaStreamSynchronize(h->stream));
  for (size_t j = 0; j < arrays.size(); ++j)
    HSG_CUDA(cudaMemcpy(arrays[j].ptr, bufs[j].data(), arrays[j].bytes, cudaMemcpyHostToDevice));
  for (int j = 0; j < 3; ++j) h->counters[j] = counters[j];
  h->energy_valid = ev != 0;
  return HSG_OK;
}

hsg_status hsg_philox4x32_10(const uint32_t* in, long n, uint32_t* out) {
  if (n < 0 || (n > 0 && (!in || !out))) return fail(HSG_EINVAL, "bad arguments");
  if (n == 0) return HSG_OK;
  uint32_t *d_in = nullptr, *d_out = nullptr;
  HSG_TRY(dalloc(&d_in, 6 * static_cast<size_t>(n)));
  if (dalloc(&d_out, 4 * static_cast<size_t>(n)) != HSG_OK) {
    cudaFree(d_in);
    return HSG_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(d_in, in, sizeof(uint32_t) * 6 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_philox_eval<<<static_cast<unsigned>((n + 255) / 256), 256>>>(d_in, n, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(HSG_ECUDA, std::string("philox evaluation failed: ") + cudaGetErrorString(e));
  return HSG_OK;
}

}  // extern "C"
