// Whole-sample host <-> device transfers: staged records in natural site
// order to and from the device layout (parity-split rows, V interleaved
// lattices per element), and the packing of couplings to their storage
// format.  Off the Monte Carlo path: used by the setters and getters only.
#pragma once
#include <cuda_fp16.h>

#include "kernels.cuh"

namespace hsg {

// Host spins of consecutive slots [count][N][3] (natural site order), staged
// on the device in chunks <-> the device layout of one sample.  Element q of
// a chunk is site (q0 + q) % N of slot (q0 + q) / N; spins_s is the sample's
// first lattice group ([G][3][N][V]).
static __global__ void k_scatter_spins_many(const float* __restrict__ stage, float* __restrict__ spins_s, int L,
                                            int V, long long q0, long long n) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const long long N = static_cast<long long>(L) * L * L;
  const long long qq = q0 + q;
  const int slot = static_cast<int>(qq / N), i = static_cast<int>(qq - slot * N);
  const int d = site_of<true>(i % L, i / L, L);
  const size_t plane = static_cast<size_t>(N) * V;
  float* base = spins_s + static_cast<size_t>(slot / V) * 3 * plane + static_cast<size_t>(d) * V + slot % V;
  for (int c = 0; c < 3; ++c) base[c * plane] = stage[3 * q + c];
}

static __global__ void k_gather_spins_many(const float* __restrict__ spins_s, float* __restrict__ stage, int L,
                                           int V, long long q0, long long n) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const long long N = static_cast<long long>(L) * L * L;
  const long long qq = q0 + q;
  const int slot = static_cast<int>(qq / N), i = static_cast<int>(qq - slot * N);
  const int d = site_of<true>(i % L, i / L, L);
  const size_t plane = static_cast<size_t>(N) * V;
  const float* base = spins_s + static_cast<size_t>(slot / V) * 3 * plane + static_cast<size_t>(d) * V + slot % V;
  for (int c = 0; c < 3; ++c) stage[3 * q + c] = base[c * plane];
}

// Couplings J6 [n][3][6] (FP32, natural sites i0 .. i0+n-1) staged on the
// device -> the storage format of one sample ([3][N] bonds in storage site
// order): FP32 as given, FP16 rounded to nearest even (the host's rounding)
// with two zero halves of padding.
template <int PREC>
static __global__ void k_pack_couplings(const float* __restrict__ stage, void* __restrict__ J, int L, long long i0,
                                        long long n) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const long long N = static_cast<long long>(L) * L * L;
  const long long i = i0 + t / 3;
  const int mu = static_cast<int>(t % 3);
  const size_t d = static_cast<size_t>(mu) * N + site_of<true>(static_cast<int>(i % L), static_cast<int>(i / L), L);
  const float* in = stage + 6 * t;
  if constexpr (PREC == kPrecF32) {
    float* out = static_cast<float*>(J) + 6 * d;
    for (int e = 0; e < 6; ++e) out[e] = in[e];
  } else {
    __half hv[8];
    for (int e = 0; e < 6; ++e) hv[e] = __float2half_rn(in[e]);
    hv[6] = __float2half_rn(0.0f);
    hv[7] = __float2half_rn(0.0f);
    static_cast<uint4*>(J)[d] = *reinterpret_cast<const uint4*>(hv);
  }
}

}  // namespace hsg
