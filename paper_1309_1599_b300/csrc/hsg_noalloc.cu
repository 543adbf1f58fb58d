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
// Sharing rules: all calls on a device use the same array, and it keeps what
// the last call left in it.  Every entry a call reads is written earlier in
// that same call, so nothing needs clearing between calls; but two calls whose
// work overlaps on the GPU (different streams, or different host threads
// without ordering) race on the array and give wrong energies.  Order such
// calls on one stream, or synchronise between them.
#include <cuda_runtime.h>

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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

// Records the message that hsg_last_error() returns (defined in hsg.cu).
void hsg_record_error(const std::string& msg);

namespace {

hsg_status noalloc_fail(hsg_status st, const std::string& msg) {
  hsg_record_error(msg);
  return st;
}

// Device address of the working array for the current device.  Host code
// cannot use the symbol itself (it names a host-side stand-in), so the
// address is looked up once per device with that device current.
hsg_status scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(HSG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HSG_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || p == nullptr)
      return noalloc_fail(HSG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
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
  double* scratch = nullptr;
  hsg_status st = scratch_for_current_device(&scratch);
  if (st != HSG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

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
