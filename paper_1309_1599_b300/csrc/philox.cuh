// Device Philox4x32-10 and the uniform mappings of the hsg interface.
//
// Written from the generator's published definition (J. K. Salmon,
// M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): ten rounds, each mapping the counter (c0,c1,c2,c3) under
// key (k0,k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)), with the key advanced by the Weyl increments between rounds.
// It stands in for the Parisi-Rapuano + congruential generator of the paper
// (App. A.4.1): being counter based it needs no per-thread state, so any
// sweep can be replayed or resumed bit for bit.
#pragma once
#include <cstdint>

namespace hsg {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Stream tags (fourth counter word) of the interface.
constexpr uint32_t kTagHeatBath = 1u;
constexpr uint32_t kTagTempering = 2u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += kPhiloxW0;
      k.y += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// (k + 1/2) 2^-23 for the top 23 bits k of w: an odd multiple of 2^-24 in
// (0,1), exact in binary32 (as is 1 - r).
__device__ __forceinline__ float uniform23(uint32_t w) {
  return (static_cast<float>(w >> 9) + 0.5f) * 0x1p-23f;
}

// 52-bit uniform in (0,1) from two words, exact in binary64.
__device__ __forceinline__ double uniform52(uint32_t w0, uint32_t w1) {
  const uint64_t v = (static_cast<uint64_t>(w0 >> 6) << 26) | static_cast<uint64_t>(w1 >> 6);
  return (static_cast<double>(v) + 0.5) * 0x1p-52;
}

}  // namespace hsg
