// Shared-memory-resident Monte Carlo of small lattices: one launch runs K
// whole Monte Carlo steps (Sec. III: heat-bath sweep, overrelaxation sweeps,
// energies, one parallel-tempering sweep) for every replica set of every
// sample, with the spins of a replica set held in shared memory from the
// first step to the last.
//
// A CTA owns one replica set: the N_T lattices of one replica index of one
// sample (all temperatures), V lattices interleaved per element exactly as in
// global memory, so the set is one contiguous block copied in at the start
// and out at the end.  Parallel tempering only exchanges temperatures inside
// a replica set (App. A.1), so each CTA runs its own PT sweep after its own
// energies; no CTA ever waits for another.  Samples of different L (buckets)
// run in the same launch; a CTA finds its bucket from its index.
//
// The arithmetic is that of the streaming kernels: the same site order, the
// same field summation (forward and backward partial sums), the same
// single-spin updates and the same Philox counters (the sweep counters
// advance by one per step), so the spins agree bit for bit with the
// streaming path as long as the PT decisions agree (their energies are
// summed in a different order, so a decision within rounding of its
// threshold may differ).
#pragma once
#include "kernels.cuh"

namespace hsg {

constexpr int kPersistentThreads = 512;
constexpr int kMaxBuckets = 8;
constexpr int kMaxTempsResident = 64;
constexpr int kMaxStepsPerLaunch = 256;

struct PersistentBucket {
  float* spins;            // bucket spins [S_b][G][3][N][V]
  const void* J;           // bucket couplings
  const int* sample_ids;   // [S_b]
  int L, N, S_b, G;
  int cta_begin;           // first CTA of this bucket (CTAs = S_b * n_rep)
};

struct PersistentParams {
  PersistentBucket b[kMaxBuckets];
  int n_buckets;
  int R, n_rep, NT, n_or, steps;
  const double* beta;      // [NT]
  double* E;               // [S][R]
  int* perm;               // [S][n_rep][NT] temperature -> slot
  int* temp_of;            // [S][R]
  long long* accepted;     // [S][n_rep][max(NT-1,1)]
  uint2 key;
  const uint32_t* counters;  // [0] heat-bath sweeps, [1] PT sweeps (at launch)
};

template <int V>
__device__ __forceinline__ void lds_plane(const float* base, size_t plane, int i, float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      const float2 t = reinterpret_cast<const float2*>(base + c * plane)[i];
      s[c][0] = t.x;
      s[c][1] = t.y;
    } else {
      s[c][0] = base[c * plane + i];
    }
  }
}

template <int V>
__device__ __forceinline__ void sts_plane(float* base, size_t plane, int i, const float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      reinterpret_cast<float2*>(base + c * plane)[i] = make_float2(s[c][0], s[c][1]);
    } else {
      base[c * plane + i] = s[c][0];
    }
  }
}

// One colour half-sweep (KIND: heat-bath or overrelaxation) of the resident
// replica set, sp: [G_set][3][N][V] in shared memory.  The (site, group)
// pairs of the colour are spread over the threads, consecutive threads on
// consecutive sites of one group.
template <int KIND, int V, int PREC>
__device__ __forceinline__ void resident_half_sweep(float* sp, const void* Jb, int L, int N, int G_set, int colour,
                                                    const float* beta_lat, uint32_t lat_base, uint32_t t,
                                                    uint2 key) {
  const int half = L >> 1;
  const int LL = L * L;
  const int n_col = N >> 1;
  const size_t plane = static_cast<size_t>(N) * V;
  for (int w = threadIdx.x; w < G_set * n_col; w += blockDim.x) {
    const int g = w / n_col;
    const int ic = w - g * n_col;
    const int row = ic / half;
    const int k = ic - row * half;
    const int y = row % L;
    const int z = row / L;
    const int x = 2 * k + ((colour + y + z) & 1);
    const int i_nat = x + L * row;
    const int i = site_of<true>(x, row, L);
    const int ixm = site_of<true>((x == 0) ? L - 1 : x - 1, row, L);
    const int ixp = site_of<true>((x == L - 1) ? 0 : x + 1, row, L);
    const int iym = (y == 0) ? i + (L - 1) * L : i - L;
    const int iyp = (y == L - 1) ? i - (L - 1) * L : i + L;
    const int izm = (z == 0) ? i + (L - 1) * LL : i - LL;
    const int izp = (z == L - 1) ? i - (L - 1) * LL : i + LL;
    float* base = sp + static_cast<size_t>(g) * 3 * plane;
    float h[3][V], hf[3][V], hb[3][V], j[6], s[3][V];
    zero3<V>(hf);
    zero3<V>(hb);
    load_bond<PREC>(Jb, i, j);                          lds_plane<V>(base, plane, ixp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jb, N + i, j);                      lds_plane<V>(base, plane, iyp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + i, j);   lds_plane<V>(base, plane, izp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jb, ixm, j);                        lds_plane<V>(base, plane, ixm, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(Jb, N + iym, j);                    lds_plane<V>(base, plane, iym, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + izm, j); lds_plane<V>(base, plane, izm, s); add_bond<V>(j, s, hb);
    combine_field<V>(hf, hb, h);
    float o[3][V];
    if constexpr (KIND == kHB) {
      const uint32_t lat0 = lat_base + static_cast<uint32_t>(g * V);
      const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(i_nat), lat0 >> 1, t, kTagHeatBath), key);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const uint32_t lat = lat0 + v;
        heat_bath_draw(h[0][v], h[1][v], h[2][v], beta_lat[g * V + v], (lat & 1u) ? r.z : r.x,
                       (lat & 1u) ? r.w : r.y, o[0][v], o[1][v], o[2][v]);
      }
      sts_plane<V>(base, plane, i, o);
    } else {
      lds_plane<V>(base, plane, i, o);
      overrelax_v<V>(h, o);
      sts_plane<V>(base, plane, i, o);
    }
  }
}

// Energies of the resident lattices, E = -sum over white sites of s.h
// (every bond has one white end): per group, per-thread FP32 terms summed in
// FP64, warp sums, then a fixed-order sum over warps.
template <int V, int PREC>
__device__ __forceinline__ void resident_energies(const float* sp, const void* Jb, int L, int N, int G_set,
                                                  double* s_E, double (*s_red)[V]) {
  const int half = L >> 1;
  const int LL = L * L;
  const size_t plane = static_cast<size_t>(N) * V;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int g = 0; g < G_set; ++g) {
    const float* base = sp + static_cast<size_t>(g) * 3 * plane;
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0;
    for (int ic = threadIdx.x; ic < (N >> 1); ic += blockDim.x) {
      const int row = ic / half;
      const int k = ic - row * half;
      const int y = row % L;
      const int z = row / L;
      const int x = 2 * k + ((1 + y + z) & 1);
      const int i = site_of<true>(x, row, L);
      const int ixm = site_of<true>((x == 0) ? L - 1 : x - 1, row, L);
      const int ixp = site_of<true>((x == L - 1) ? 0 : x + 1, row, L);
      const int iym = (y == 0) ? i + (L - 1) * L : i - L;
      const int iyp = (y == L - 1) ? i - (L - 1) * L : i + L;
      const int izm = (z == 0) ? i + (L - 1) * LL : i - LL;
      const int izp = (z == L - 1) ? i - (L - 1) * LL : i + LL;
      float h[3][V], hf[3][V], hb[3][V], j[6], s[3][V], o[3][V];
      zero3<V>(hf);
      zero3<V>(hb);
      load_bond<PREC>(Jb, i, j);                          lds_plane<V>(base, plane, ixp, s); add_bond<V>(j, s, hf);
      load_bond<PREC>(Jb, N + i, j);                      lds_plane<V>(base, plane, iyp, s); add_bond<V>(j, s, hf);
      load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + i, j);   lds_plane<V>(base, plane, izp, s); add_bond<V>(j, s, hf);
      load_bond<PREC>(Jb, ixm, j);                        lds_plane<V>(base, plane, ixm, s); add_bond<V>(j, s, hb);
      load_bond<PREC>(Jb, N + iym, j);                    lds_plane<V>(base, plane, iym, s); add_bond<V>(j, s, hb);
      load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + izm, j); lds_plane<V>(base, plane, izm, s); add_bond<V>(j, s, hb);
      combine_field<V>(hf, hb, h);
      lds_plane<V>(base, plane, i, o);
#pragma unroll
      for (int v = 0; v < V; ++v)
        acc[v] -= static_cast<double>(fmaf(o[0][v], h[0][v], fmaf(o[1][v], h[1][v], o[2][v] * h[2][v])));
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const double d = warp_sum(acc[v]);
      if (lane == 0) s_red[warp][v] = d;
    }
    __syncthreads();
    if (threadIdx.x < V) {
      double e = 0.0;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) e += s_red[w][threadIdx.x];
      s_E[g * V + threadIdx.x] = e;
    }
    __syncthreads();
  }
}

template <int V, int PREC>
__global__ void __launch_bounds__(kPersistentThreads) k_persistent(PersistentParams p) {
  extern __shared__ __align__(16) float sp[];
  __shared__ double s_E[kMaxTempsResident];
  __shared__ float s_beta_lat[kMaxTempsResident];   // beta of each local lattice
  __shared__ int s_perm[kMaxTempsResident];         // temperature -> local lattice
  __shared__ int s_acc[kMaxTempsResident];
  __shared__ double s_red[kPersistentThreads / 32][V];

  int bi = 0;
  while (bi + 1 < p.n_buckets && static_cast<int>(blockIdx.x) >= p.b[bi + 1].cta_begin) ++bi;
  const PersistentBucket& B = p.b[bi];
  const int local = blockIdx.x - B.cta_begin;
  const int sb = local / p.n_rep, r = local - sb * p.n_rep;
  const int sg = B.sample_ids[sb];
  const int NT = p.NT, L = B.L, N = B.N;
  const int G_set = NT / V;                               // groups of this replica set
  const size_t set_floats = static_cast<size_t>(NT) * 3 * N;
  float* gsp = B.spins + (static_cast<size_t>(sb) * B.G + static_cast<size_t>(r) * G_set) * 3 * N * V;
  const void* Jb = (PREC == kPrecF16)
                       ? static_cast<const void*>(static_cast<const uint4*>(B.J) + static_cast<size_t>(sb) * 3 * N)
                       : static_cast<const void*>(static_cast<const float*>(B.J) + static_cast<size_t>(sb) * 3 * N * 6);
  const uint32_t lat_base = static_cast<uint32_t>(sg) * p.R + static_cast<uint32_t>(r * NT);
  const uint32_t gset = static_cast<uint32_t>(sg) * p.n_rep + r;
  const uint32_t t_hb0 = p.counters[0], t_pt0 = p.counters[1];

  // replica set -> shared memory (contiguous, 16-byte aligned)
  {
    const float4* src = reinterpret_cast<const float4*>(gsp);
    float4* dst = reinterpret_cast<float4*>(sp);
    for (size_t q = threadIdx.x; q < set_floats / 4; q += blockDim.x) dst[q] = src[q];
  }
  if (threadIdx.x < NT) {
    const int k = threadIdx.x;
    const int slot = p.perm[(static_cast<size_t>(sg) * p.n_rep + r) * NT + k];
    s_perm[k] = slot - r * NT;
    s_beta_lat[slot - r * NT] = static_cast<float>(p.beta[k]);
    s_acc[k] = 0;
  }
  __syncthreads();

  for (int step = 0; step < p.steps; ++step) {
    const uint32_t t = t_hb0 + static_cast<uint32_t>(step);
    for (int c = 0; c < 2; ++c) {
      resident_half_sweep<kHB, V, PREC>(sp, Jb, L, N, G_set, c, s_beta_lat, lat_base, t, p.key);
      __syncthreads();
    }
    for (int o = 0; o < p.n_or; ++o) {
      for (int c = 0; c < 2; ++c) {
        resident_half_sweep<kOR, V, PREC>(sp, Jb, L, N, G_set, c, s_beta_lat, lat_base, t, p.key);
        __syncthreads();
      }
    }
    resident_energies<V, PREC>(sp, Jb, L, N, G_set, s_E, s_red);
    // parallel tempering within the replica set (App. A.1)
    if (threadIdx.x == 0 && NT > 1) {
      const uint32_t tp = t_pt0 + static_cast<uint32_t>(step);
      for (int k = 0; k + 1 < NT; ++k) {
        const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(k), gset, tp, kTagTempering), p.key);
        const double u = uniform52(w.x, w.y);
        const int a = s_perm[k], b = s_perm[k + 1];
        const double delta = (p.beta[k] - p.beta[k + 1]) * (s_E[a] - s_E[b]);
        if (delta >= 0.0 || u < exp(delta)) {
          s_perm[k] = b;
          s_perm[k + 1] = a;
          s_acc[k] += 1;
        }
      }
      for (int k = 0; k < NT; ++k) s_beta_lat[s_perm[k]] = static_cast<float>(p.beta[k]);
    }
    __syncthreads();
  }

  // shared memory -> replica set; energies, labels and acceptances out
  {
    const float4* src = reinterpret_cast<const float4*>(sp);
    float4* dst = reinterpret_cast<float4*>(gsp);
    for (size_t q = threadIdx.x; q < set_floats / 4; q += blockDim.x) dst[q] = src[q];
  }
  if (threadIdx.x < NT) {
    const int k = threadIdx.x;
    const size_t pbase = (static_cast<size_t>(sg) * p.n_rep + r) * NT;
    p.perm[pbase + k] = s_perm[k] + r * NT;
    p.temp_of[static_cast<size_t>(sg) * p.R + r * NT + s_perm[k]] = k;
    p.E[static_cast<size_t>(sg) * p.R + r * NT + k] = s_E[k];
    if (k + 1 < NT || NT == 1) {
      const int stride = NT > 1 ? NT - 1 : 1;
      p.accepted[(static_cast<size_t>(sg) * p.n_rep + r) * stride + k] += s_acc[k];
    }
  }
}

}  // namespace hsg
