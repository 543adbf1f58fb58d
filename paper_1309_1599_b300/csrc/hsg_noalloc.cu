// hsg_energy_noalloc: lattice energies from caller-owned device buffers, with
// no device memory allocated by the library at any point.
//
// Why it exists: some callers cannot let a library call cudaMalloc/cudaFree.
// Examples are hosts that hand out all device memory from a fixed arena they
// plan up front, and latency-critical loops that must never stop in the
// driver's allocator (cudaMalloc and cudaFree can synchronise the device).
// The context API (hsg_lattice_create) allocates everything it owns, so such
// callers cannot use it.  This entry point takes the spins, couplings and
// output as device pointers and keeps its one piece of working memory -- the
// per-block partial sums of the energy reduction -- in a fixed, file-scope
// device array that every GPU loading the library holds until the process
// exits.
//
// Every caller buffer is checked before anything runs (device memory of the
// current device, inside one allocation large enough, aligned), so a wrong
// pointer is refused with HSG_EINVAL instead of faulting a shared GPU.
//
// Sharing rules: all calls on a device use the same array, and it keeps what
// the last call left in it.  Every entry a call reads is written earlier in
// that same call, so nothing needs clearing between calls; but two calls whose
// work overlaps on the GPU (different streams, or different host threads
// without ordering) race on the array and give wrong energies.  Order such
// calls on one stream, or synchronise between them.
#include <cuda.h>  // driver API types only: the two driver calls are looked up at run time
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/hsg.h"
#include "kernels.cuh"

using namespace hsg;

namespace {

// Capacity of the working array in doubles: one partial sum per
// (lattice, block of kSweepThreads white sites).  2 MiB per device.
constexpr long long kScratchDoubles = HSG_NOALLOC_SCRATCH_DOUBLES;

static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

// The array's device address per CUDA context (a context destroyed and
// created again, e.g. after cudaDeviceReset, has a new id and may hold the
// array elsewhere): a fixed table of (context id, address), no heap.
constexpr int kMaxContexts = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  double* ptr;
};
std::mutex g_mu;
ScratchEntry g_scratch[kMaxContexts] = {};
int g_scratch_next = 0;

// Driver calls, looked up through the runtime so that the library needs no
// link dependency on the driver library.
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);
using PfnMemGetAddressRange = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
struct DriverCalls {
  PfnCtxGetCurrent ctx_get_current = nullptr;
  PfnCtxGetId ctx_get_id = nullptr;
  PfnMemGetAddressRange mem_get_address_range = nullptr;
};

}  // namespace

// Records the message that hsg_last_error() returns (defined in hsg.cu).
void hsg_record_error(const std::string& msg);

namespace {

hsg_status noalloc_fail(hsg_status st, const std::string& msg) {
  hsg_record_error(msg);
  return st;
}

hsg_status driver_calls(const DriverCalls** out) {
  static DriverCalls calls;
  static bool looked_up = false;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!looked_up) {
    struct {
      const char* name;
      void** fn;
    } want[] = {{"cuCtxGetCurrent", reinterpret_cast<void**>(&calls.ctx_get_current)},
                {"cuCtxGetId", reinterpret_cast<void**>(&calls.ctx_get_id)},
                {"cuMemGetAddressRange", reinterpret_cast<void**>(&calls.mem_get_address_range)}};
    for (auto& w : want) {
      cudaDriverEntryPointQueryResult q;
      const cudaError_t e = cudaGetDriverEntryPointByVersion(w.name, w.fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || *w.fn == nullptr) {
        cudaGetLastError();
        return noalloc_fail(HSG_ECUDA, std::string("driver entry point ") + w.name + " not found");
      }
    }
    looked_up = true;
  }
  *out = &calls;
  return HSG_OK;
}

// Device address of the working array in the current context.  Host code
// cannot use the symbol itself (it names a host-side stand-in), so the
// address is looked up with the context current, the first time the context
// calls, and remembered by context id.  The lookup is refused while `stream`
// is being captured into a graph.
hsg_status scratch_for_current_context(const DriverCalls* drv, cudaStream_t stream, double** out) {
  CUcontext ctx = nullptr;
  if (drv->ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr)
    return noalloc_fail(HSG_ECUDA, "no current CUDA context on this thread (use the device first)");
  unsigned long long id = 0;
  if (drv->ctx_get_id(ctx, &id) != CUDA_SUCCESS) return noalloc_fail(HSG_ECUDA, "cuCtxGetId failed");
  std::lock_guard<std::mutex> lock(g_mu);
  for (const ScratchEntry& en : g_scratch)
    if (en.ptr != nullptr && en.ctx_id == id) {
      *out = en.ptr;
      return HSG_OK;
    }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(HSG_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  }
  if (cs != cudaStreamCaptureStatusNone)
    return noalloc_fail(HSG_ESTATE, "the first call in a CUDA context looks up the working array's address, "
                                    "which is not done during stream capture: make one call outside capture first");
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_energy_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return noalloc_fail(HSG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  g_scratch[g_scratch_next] = {id, static_cast<double*>(p)};
  g_scratch_next = (g_scratch_next + 1) % kMaxContexts;
  *out = static_cast<double*>(p);
  return HSG_OK;
}

// A caller's buffer: `bytes` from p must lie in one allocation of device (or
// managed) memory that the current device can use, p aligned to `align`.
hsg_status check_buffer(const DriverCalls* drv, const void* p, size_t bytes, size_t align, int dev,
                        const char* name) {
  if (reinterpret_cast<uintptr_t>(p) % align != 0)
    return noalloc_fail(HSG_EINVAL, std::string(name) + " is not aligned to " + std::to_string(align) + " bytes");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(HSG_EINVAL, std::string(name) + " is not a CUDA pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return noalloc_fail(HSG_EINVAL, std::string(name) + " is not device memory");
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return noalloc_fail(HSG_EINVAL, std::string(name) + " is on device " + std::to_string(a.device) +
                                        ", the current device is " + std::to_string(dev));
  CUdeviceptr base = 0;
  size_t size = 0;
  if (drv->mem_get_address_range(&base, &size, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS)
    return noalloc_fail(HSG_EINVAL, std::string(name) + ": no device allocation holds this address");
  const size_t avail = static_cast<size_t>(base + size - reinterpret_cast<CUdeviceptr>(p));
  if (bytes > avail)
    return noalloc_fail(HSG_EINVAL, std::string(name) + " needs " + std::to_string(bytes) +
                                        " bytes, its allocation holds " + std::to_string(avail) +
                                        " from that address");
  return HSG_OK;
}

// Sum of each lattice's partials in a fixed order (one warp per lattice).
__global__ void k_energy_finalize_flat(const double* __restrict__ partial, int chunks, int n_lat,
                                       double* __restrict__ E) {
  const int lat = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (lat >= n_lat) return;
  double acc = 0.0;
  for (int c = lane; c < chunks; c += 32) acc += partial[static_cast<size_t>(lat) * chunks + c];
  acc = warp_sum(acc);
  if (lane == 0) E[lat] = acc;
}

}  // namespace

extern "C" hsg_status hsg_energy_noalloc(const float* spins, const float* J6, int L, int n_samples,
                                         int lattices_per_sample, double* E_out, void* stream) {
  if (!spins || !J6 || !E_out) return noalloc_fail(HSG_EINVAL, "NULL device pointer");
  if (L < 4 || L > 512 || (L & 1)) return noalloc_fail(HSG_EINVAL, "L must be even and in [4, 512]");
  if (n_samples < 1 || lattices_per_sample < 1)
    return noalloc_fail(HSG_EINVAL, "n_samples and lattices_per_sample must be >= 1");
  const int N = L * L * L;
  const int chunks = (N / 2 + kSweepThreads - 1) / kSweepThreads;
  const long long n_lat = static_cast<long long>(n_samples) * lattices_per_sample;
  if (n_lat * chunks > kScratchDoubles)
    return noalloc_fail(HSG_EINVAL, "request needs " + std::to_string(n_lat * chunks) +
                                        " partial sums; the fixed working array holds " +
                                        std::to_string(kScratchDoubles) +
                                        " (lattices x ceil(L^3/512) must not exceed it)");
  if (n_lat * 32 > 0x7fffffffLL) return noalloc_fail(HSG_EINVAL, "too many lattices");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DriverCalls* drv = nullptr;
  hsg_status st = driver_calls(&drv);
  if (st != HSG_OK) return st;
  int dev = -1;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e0));
  // the kernels read spins as floats and couplings as float pairs, and write
  // doubles: every buffer must be device memory of the current device, large
  // enough and aligned, or nothing is launched
  const size_t lat_floats = 3 * static_cast<size_t>(N);
  if ((st = check_buffer(drv, spins, n_lat * lat_floats * sizeof(float), 4, dev, "spins")) != HSG_OK) return st;
  if ((st = check_buffer(drv, J6, static_cast<size_t>(n_samples) * lat_floats * 6 * sizeof(float), 8, dev, "J6")) !=
      HSG_OK)
    return st;
  if ((st = check_buffer(drv, E_out, n_lat * sizeof(double), 8, dev, "E_out")) != HSG_OK) return st;
  double* scratch = nullptr;
  if ((st = scratch_for_current_context(drv, s, &scratch)) != HSG_OK) return st;

  SweepParams p;
  p.b.spins = const_cast<float*>(spins);  // read only in the energy pass
  p.b.J = J6;
  p.b.sample_ids = nullptr;               // not read by the energy pass
  p.b.L = L;
  p.b.N = N;
  p.b.S_b = n_samples;
  p.b.G = lattices_per_sample;
  p.b.D = 0.0f;                           // FP32 couplings: unused
  p.colour = 1;
  p.chunks = chunks;
  p.R = lattices_per_sample;
  p.temp_of = nullptr;
  p.beta_f = nullptr;
  p.key = make_uint2(0u, 0u);
  p.counters = nullptr;
  p.e_partial = scratch;
  const unsigned grid = static_cast<unsigned>(n_lat * chunks);
  k_sweep_half<kEnergyOnly, 1, kPrecF32><<<grid, kSweepThreads, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("energy pass: ") + cudaGetErrorString(e));
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((n_lat * 32 + threads - 1) / threads);
  k_energy_finalize_flat<<<blocks, threads, 0, s>>>(scratch, chunks, static_cast<int>(n_lat), E_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("energy sum: ") + cudaGetErrorString(e));
  return HSG_OK;
}
