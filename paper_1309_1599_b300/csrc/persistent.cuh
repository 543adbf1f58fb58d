// Shared-memory-resident Monte Carlo of small lattices: one launch runs K
// whole Monte Carlo steps (Sec. III: heat-bath sweep, overrelaxation sweeps,
// energies, one parallel-tempering sweep) for every replica set of the
// samples of one L (k_persistent), or of two lattice sizes at once
// (k_persistent_pair), with the spins held in shared memory from the first
// step to the last.
//
// A CTA owns one replica set -- the N_T lattices of one replica index of one
// sample (all temperatures) -- or several whole replica sets of one sample.
// Parallel tempering only exchanges temperatures inside a replica set
// (App. A.1), so each CTA runs the PT sweeps of its own sets after their
// energies; no CTA ever waits for another.  Where a whole set does not fit
// (L = 16 to 24), a CTA holds G_sub of its lattice groups for one step: the
// launch writes their energies and the caller runs the PT sweep.
//
// Shared-memory layout.  Global memory keeps each row's sites split by x
// parity (the streaming kernels' order).  In shared memory the sites are split
// by colour instead: colour c holds its N/2 sites in (row, x>>1) order, so
// the sites a warp updates and each of their six neighbours are consecutive
// words and the accesses are free of bank conflicts:
//   spins  [G_set][3][2 colours][N/2][V] floats
//   bonds  [3 directions][2 colours][N/2] x 6 entries, the bond (x, x+mu)
//          stored at its lower site x, when they fit beside the spins:
//          JS = 1 in the stored format (FP16: 12 B, FP32: 24 B, bimodal:
//          1 B), JS = 2 converted to FP32 once at the start (24 B); JS = 0:
//          read from global memory.
//
// Work split.  The warps are divided among work items of GP lattice groups
// each (wpg warps per item, or one warp looping over several items when
// there are more items than warps).  A thread updates one site of every
// group of its item at a time: with GP = 2 (two lattices per element and an
// even number of groups) each bond is read and converted once for four
// lattices, and the per-group arithmetic is unchanged.  The energies
// (E = -sum over white sites of s.h, every bond having one white end) are
// accumulated in the last white half-sweep of the step, where the white
// sites' fields are computed anyway, and reduced per group in a fixed order.
//
// The arithmetic is that of the streaming kernels: the same field summation
// (forward and backward partial sums), the same single-spin updates and the
// same Philox counters (the sweep counters advance by one per step), so the
// spins agree bit for bit with the streaming path as long as the PT
// decisions agree (their energies are summed in a different order, so a
// decision within rounding of its threshold may differ).
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace hsg {

constexpr int kPersistentMaxThreads = 1024;

// Launch bounds of the L specialisations: L = 12 runs one CTA per SM (its
// spins alone take 166 KB at 8 temperatures) and may use up to 102
// registers a thread at 640 threads; L = 8 runs two CTAs of 512 threads, and
// so does L = 16 (one 98 KB lattice group per CTA).
template <int LT>
constexpr int persistent_max_threads() {
  return LT == 12 ? 640 : (LT == 8 || LT == 16) ? 512 : kPersistentMaxThreads;
}
template <int LT>
constexpr int persistent_min_blocks() { return (LT == 8 || LT == 16) ? 2 : 1; }
constexpr int kMaxTempsResident = 64;
// Block limit of the two-bucket launch: the larger of its buckets' limits.
constexpr int kPairMaxThreads = 640;
constexpr int kMaxStepsPerLaunch = 256;

struct PersistentParams {
  float* spins;            // bucket spins [S_b][G][3][N][V]
  const void* J;           // bucket couplings (global storage order)
  const int* sample_ids;   // [S_b]
  int L, N, G;
  int R, n_rep, NT, n_or, steps;
  const double* beta;      // [NT]
  double* E;               // [S][R]
  int* perm;               // [S][n_rep][NT] temperature -> slot
  int* temp_of;            // [S][R]
  long long* accepted;     // [S][n_rep][max(NT-1,1)]
  uint2 key;
  const uint32_t* counters;  // [0] heat-bath sweeps, [1] PT sweeps (at launch)
  float D;                 // bimodal couplings: magnitude of the anisotropy
  int G_sub;               // lattice groups per CTA: sets * N_T/V (whole replica
                           // sets) or a divisor of N_T/V (part of one set)
  int sets;                // whole replica sets per CTA (a divisor of n_rep, with
                           // sets * N_T <= kMaxTempsResident), 1 for parts of a set
  int pt;                  // 1: PT in the kernel (whole sets); 0: one step per
                           // launch, energies out, the PT sweep by the caller
  int warps;               // warps that sweep (<= the block's); the others only
                           // copy in and out and join the barriers
};

// The CTA-wide tables of a resident CTA, indexed by local lattice (the
// lattices a CTA holds, numbered from its first slot) or, for the labels and
// acceptances, by set * N_T + temperature.
struct PersistentShared {
  double* E;          // [kMaxTempsResident] energy of each local lattice
  double* part;       // [2 kMaxTempsResident] per (group, warp of the group, lattice)
  float* beta_lat;    // [kMaxTempsResident] beta of each local lattice
  int* perm;          // [kMaxTempsResident] (set, temperature) -> local lattice
  int* acc;           // [kMaxTempsResident] accepted swaps per (set, pair)
};


template <int V>
__device__ __forceinline__ void lds_plane(const float* base, int plane, int i, float (&s)[3][V]) {
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
__device__ __forceinline__ void sts_plane(float* base, int plane, int i, const float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      reinterpret_cast<float2*>(base + c * plane)[i] = make_float2(s[c][0], s[c][1]);
    } else {
      base[c * plane + i] = s[c][0];
    }
  }
}

// One bond from the resident layout: the same floats as load_bond() gives for
// the same stored entries.
template <int PREC>
__device__ __forceinline__ void lds_bond(const void* Js, int idx, float (&j)[6], float D) {
  if constexpr (PREC == kPrecBimodal) {
    decode_bimodal(static_cast<const uint8_t*>(Js)[idx], D, j);
  } else if constexpr (PREC == kPrecF16) {
    const uint32_t* p = static_cast<const uint32_t*>(Js) + 3 * idx;
    __half2 h0, h1, h2;
    *reinterpret_cast<uint32_t*>(&h0) = p[0];
    *reinterpret_cast<uint32_t*>(&h1) = p[1];
    *reinterpret_cast<uint32_t*>(&h2) = p[2];
    const float2 a = __half22float2(h0), b = __half22float2(h1), c = __half22float2(h2);
    j[0] = a.x; j[1] = a.y; j[2] = b.x; j[3] = b.y; j[4] = c.x; j[5] = c.y;
  } else {
    const float2* p = reinterpret_cast<const float2*>(static_cast<const float*>(Js) + 6 * idx);
    const float2 a = p[0], b = p[1], c = p[2];
    j[0] = a.x; j[1] = a.y; j[2] = b.x; j[3] = b.y; j[4] = c.x; j[5] = c.y;
  }
}

// Geometry of site number ic of colour c: its neighbours' indices in the
// other colour of the colour-split layout (its own index is ic), its natural
// index x + L (y + L z), and, for bonds read from global memory, the
// parity-split storage indices of the site and of its -x, -y, -z neighbours.
struct ResidentSite {
  int jxp, jxm, jyp, jym, jzp, jzm;  // neighbours, colour-split index
  int i_nat;
  int gi, gxm, gym, gzm;             // global storage index (site, -x, -y, -z)
};

template <bool GLOBAL_J>
__device__ __forceinline__ ResidentSite resident_site(int ic, int colour, const int L) {
  const int half = L >> 1;
  const int row = ic / half;
  const int k = ic - row * half;
  const int y = row % L;
  const int z = row / L;
  const int p = (colour + y + z) & 1;                  // x parity of the site
  const int x = 2 * k + p;
  ResidentSite r;
  const int rb = row * half;
  r.jxp = rb + (p ? ((k + 1 == half) ? 0 : k + 1) : k);
  r.jxm = rb + (p ? k : ((k == 0) ? half - 1 : k - 1));
  const int hy = half, hz = half * L;
  r.jyp = (y == L - 1) ? ic - (L - 1) * hy : ic + hy;
  r.jym = (y == 0) ? ic + (L - 1) * hy : ic - hy;
  r.jzp = (z == L - 1) ? ic - (L - 1) * hz : ic + hz;
  r.jzm = (z == 0) ? ic + (L - 1) * hz : ic - hz;
  r.i_nat = x + L * row;
  if constexpr (GLOBAL_J) {
    const int LL = L * L;
    r.gi = site_of<true>(x, row, L);
    r.gxm = site_of<true>((x == 0) ? L - 1 : x - 1, row, L);
    r.gym = (y == 0) ? r.gi + (L - 1) * L : r.gi - L;
    r.gzm = (z == 0) ? r.gi + (L - 1) * LL : r.gi - LL;
  }
  return r;
}

// Local field (Eq. 3) at site ic of colour c of one resident lattice group:
// forward bonds (+x, +y, +z, stored at the site) into hf, backward bonds
// (-x, -y, -z, stored at the neighbour) into hb, in the streaming kernels'
// order.  sg: the group's spins, colour-split.  Js / Jg: resident or global
// bonds.
template <int V, int PREC, int JS>
__device__ __forceinline__ void resident_field(const float* sg, const void* Js, const void* Jg, float D,
                                               const int N, int colour, int ic, const ResidentSite& r,
                                               float (&h)[3][V]) {
  constexpr int BP = JS == 2 ? kPrecF32 : PREC;        // precision of the resident bonds
  const int hN = N >> 1;
  const int plane = N * V;
  const float* so = sg + (colour ^ 1) * hN * V;          // neighbours' colour
  const int c_own = colour * hN, c_nb = (colour ^ 1) * hN;
  float hf[3][V], hb[3][V], j[6], s[3][V];
  zero3<V>(hf);
  zero3<V>(hb);
  if constexpr (JS != 0) {
    lds_bond<BP>(Js, c_own + ic, j, D);           lds_plane<V>(so, plane, r.jxp, s); add_bond<V>(j, s, hf);
    lds_bond<BP>(Js, N + c_own + ic, j, D);       lds_plane<V>(so, plane, r.jyp, s); add_bond<V>(j, s, hf);
    lds_bond<BP>(Js, 2 * N + c_own + ic, j, D);   lds_plane<V>(so, plane, r.jzp, s); add_bond<V>(j, s, hf);
    lds_bond<BP>(Js, c_nb + r.jxm, j, D);         lds_plane<V>(so, plane, r.jxm, s); add_bond<V>(j, s, hb);
    lds_bond<BP>(Js, N + c_nb + r.jym, j, D);     lds_plane<V>(so, plane, r.jym, s); add_bond<V>(j, s, hb);
    lds_bond<BP>(Js, 2 * N + c_nb + r.jzm, j, D); lds_plane<V>(so, plane, r.jzm, s); add_bond<V>(j, s, hb);
  } else {
    const size_t n = static_cast<size_t>(N);
    load_bond<PREC>(Jg, r.gi, j, D);                lds_plane<V>(so, plane, r.jxp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jg, n + r.gi, j, D);            lds_plane<V>(so, plane, r.jyp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jg, 2 * n + r.gi, j, D);        lds_plane<V>(so, plane, r.jzp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(Jg, r.gxm, j, D);               lds_plane<V>(so, plane, r.jxm, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(Jg, n + r.gym, j, D);           lds_plane<V>(so, plane, r.jym, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(Jg, 2 * n + r.gzm, j, D);       lds_plane<V>(so, plane, r.jzm, s); add_bond<V>(j, s, hb);
  }
  combine_field<V>(hf, hb, h);
}

// resident_field for GP lattice groups at once (same site, same colour):
// each bond is read (and converted) once and applied to every group, each
// group's field summed in resident_field's order.  sgs[q]: group q's spins.
template <int V, int PREC, int JS, int GP>
__device__ __forceinline__ void resident_field_gp(float* const (&sgs)[GP], const void* Js, const void* Jg, float D,
                                                  const int N, int colour, int ic, const ResidentSite& r,
                                                  float (&h)[GP][3][V]) {
  if constexpr (GP == 1) {
    float h1[3][V];
    resident_field<V, PREC, JS>(sgs[0], Js, Jg, D, N, colour, ic, r, h1);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v) h[0][c][v] = h1[c][v];
  } else {
    constexpr int BP = JS == 2 ? kPrecF32 : PREC;
    const int hN = N >> 1;
    const int plane = N * V;
    const int off_nb = (colour ^ 1) * hN * V;            // neighbours' colour
    const int c_own = colour * hN, c_nb = (colour ^ 1) * hN;
    float hf[GP][3][V], hb[GP][3][V], j[6], s[3][V];
#pragma unroll
    for (int q = 0; q < GP; ++q) {
      zero3<V>(hf[q]);
      zero3<V>(hb[q]);
    }
    auto apply = [&](int nb, float (&acc)[GP][3][V]) {
#pragma unroll
      for (int q = 0; q < GP; ++q) {
        lds_plane<V>(sgs[q] + off_nb, plane, nb, s);
        add_bond<V>(j, s, acc[q]);
      }
    };
    if constexpr (JS != 0) {
      lds_bond<BP>(Js, c_own + ic, j, D);           apply(r.jxp, hf);
      lds_bond<BP>(Js, N + c_own + ic, j, D);       apply(r.jyp, hf);
      lds_bond<BP>(Js, 2 * N + c_own + ic, j, D);   apply(r.jzp, hf);
      lds_bond<BP>(Js, c_nb + r.jxm, j, D);         apply(r.jxm, hb);
      lds_bond<BP>(Js, N + c_nb + r.jym, j, D);     apply(r.jym, hb);
      lds_bond<BP>(Js, 2 * N + c_nb + r.jzm, j, D); apply(r.jzm, hb);
    } else {
      const size_t n = static_cast<size_t>(N);
      load_bond<PREC>(Jg, r.gi, j, D);              apply(r.jxp, hf);
      load_bond<PREC>(Jg, n + r.gi, j, D);          apply(r.jyp, hf);
      load_bond<PREC>(Jg, 2 * n + r.gi, j, D);      apply(r.jzp, hf);
      load_bond<PREC>(Jg, r.gxm, j, D);             apply(r.jxm, hb);
      load_bond<PREC>(Jg, n + r.gym, j, D);         apply(r.jym, hb);
      load_bond<PREC>(Jg, 2 * n + r.gzm, j, D);     apply(r.jzm, hb);
    }
#pragma unroll
    for (int q = 0; q < GP; ++q) combine_field<V>(hf[q], hb[q], h[q]);
  }
}

// Warp layout of a CTA over the G_set lattice groups of its replica set.
struct ResidentWarps {
  int wpg;    // warps per group
  int gpp;    // groups in flight at once
  int g0;     // this warp's first group (>= gpp: idle in the sweeps)
  int sub;    // this warp's index within its group
};

__device__ __forceinline__ ResidentWarps resident_warps(int G_set, int W) {
  const int warp = threadIdx.x >> 5;
  ResidentWarps rw;
  rw.wpg = W >= G_set ? W / G_set : 1;
  rw.gpp = W / rw.wpg;
  rw.g0 = warp < W ? warp / rw.wpg : rw.gpp;  // warps beyond W sit out the sweeps
  rw.sub = warp - (warp < W ? rw.g0 : 0) * rw.wpg;
  return rw;
}

// One colour half-sweep (KIND: heat-bath or overrelaxation) of the resident
// replica set.  The warps take items of GP groups (groups gi*GP .. gi*GP+GP-1)
// and, within an item, sites.  With ENERGY (the last white half-sweep of a
// step), each warp also sums -s.h over its sites of each group it updates
// (FP32 terms in FP64) into s_part[(g * wpg + sub) * V + v].
template <int KIND, bool ENERGY, int V, int PREC, int JS, int LT, int GP>
__device__ __forceinline__ void resident_half_sweep(float* sp, const void* Js, const void* Jg, float D,
                                                    const int Lrt,
                                                    const ResidentWarps& rw, int G_set, int colour,
                                                    const float* beta_lat, uint32_t lat_base, uint32_t t,
                                                    uint2 key, double* s_part) {
  const int L = LT > 0 ? LT : Lrt;
  const int N = L * L * L;
  const int hN = N >> 1;
  const int plane = N * V;
  const int lane = threadIdx.x & 31;
  const int G_items = G_set / GP;
  if (rw.g0 >= rw.gpp) return;
  for (int gi = rw.g0; gi < G_items; gi += rw.gpp) {
    float* sgs[GP];
#pragma unroll
    for (int q = 0; q < GP; ++q) sgs[q] = sp + (gi * GP + q) * 3 * plane;
    double acc[GP][V];
#pragma unroll
    for (int q = 0; q < GP; ++q)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[q][v] = 0.0;
    for (int ic = rw.sub * 32 + lane; ic < hN; ic += rw.wpg * 32) {
      const ResidentSite r = resident_site<JS == 0>(ic, colour, L);
      float h[GP][3][V];
      resident_field_gp<V, PREC, JS, GP>(sgs, Js, Jg, D, N, colour, ic, r, h);
#pragma unroll
      for (int q = 0; q < GP; ++q) {
        const int g = gi * GP + q;
        float* own = sgs[q] + colour * hN * V;
        float o[3][V];
        if constexpr (KIND == kHB) {
          const uint32_t lat0 = lat_base + static_cast<uint32_t>(g * V);
          const uint4 u =
              philox4x32_10(make_uint4(static_cast<uint32_t>(r.i_nat), lat0 >> 1, t, kTagHeatBath), key);
          float bq[V];
#pragma unroll
          for (int v = 0; v < V; ++v) bq[v] = beta_lat[g * V + v];
          heat_bath_site<V>(h[q], bq, u, lat0, o);
        } else {
          lds_plane<V>(own, plane, ic, o);
          overrelax_v<V>(h[q], o);
        }
        sts_plane<V>(own, plane, ic, o);
        if constexpr (ENERGY) {
#pragma unroll
          for (int v = 0; v < V; ++v)
            acc[q][v] -= static_cast<double>(
                fmaf(o[0][v], h[q][0][v], fmaf(o[1][v], h[q][1][v], o[2][v] * h[q][2][v])));
        }
      }
    }
    if constexpr (ENERGY) {
#pragma unroll
      for (int q = 0; q < GP; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const double d = warp_sum(acc[q][v]);
          if (lane == 0) s_part[((gi * GP + q) * rw.wpg + rw.sub) * V + v] = d;
        }
    }
  }
}

// Position in the colour-split layout of global storage index i (row-wise
// parity split): colour * N/2 + row * L/2 + (x >> 1).
__device__ __forceinline__ int colour_split_index(int i, int L, int N) {
  const int half = L >> 1;
  const int row = i / L;
  const int rem = i - row * L;
  const int px = rem >= half ? 1 : 0;                  // x parity block
  const int k = rem - px * half;
  const int y = row % L, z = row / L;
  const int c = (px + y + z) & 1;
  return c * (N >> 1) + row * half + k;
}

// K whole steps of the replica sets one CTA holds, for one L: the body of
// the resident kernels.  cta: the CTA's index among those of its bucket.
// V: lattices per element; PREC: stored coupling precision; JS: bond
// residency (see above); LT: L as a compile-time constant, or 0 for the
// runtime p.L; GP: lattice groups per work item (2: each bond read and
// converted once for two groups).
template <int V, int PREC, int JS, int LT, int GP>
__device__ __forceinline__ void persistent_body(const PersistentParams& p, const int cta, float* sp,
                                                const PersistentShared& sh) {
  double* s_E = sh.E;
  double* s_part = sh.part;
  float* s_beta_lat = sh.beta_lat;
  int* s_perm = sh.perm;
  int* s_acc = sh.acc;
  const int NT = p.NT;
  const int sets = p.sets;                                // whole replica sets held (1: a set or part of one)
  const int G_sub = p.G_sub;                              // groups held by this CTA
  const bool whole = p.pt != 0;                           // whole replica sets, PT here
  const int NT_loc = G_sub * V;                           // lattices held by this CTA
  int sb, r0, part;
  if (sets > 1) {                                         // several whole sets of one sample
    const int cps = p.n_rep / sets;
    sb = cta / cps;
    r0 = (cta - sb * cps) * sets;
    part = 0;
  } else {                                                // one set, or part n of one
    const int n_sub = NT / V / G_sub;                     // CTAs per replica set
    const int sr = cta / n_sub;
    part = cta - sr * n_sub;
    sb = sr / p.n_rep;
    r0 = sr - sb * p.n_rep;
  }
  const int sg = p.sample_ids[sb];
  const int L = LT > 0 ? LT : p.L;
  const int N = L * L * L;
  float* gsp = p.spins + (static_cast<size_t>(sb) * p.G + static_cast<size_t>(r0) * (NT / V) +
                          static_cast<size_t>(part) * G_sub) * 3 * N * V;
  const void* Jg = sample_bonds<PREC>(p.J, sb, N);
  void* Js = sp + static_cast<size_t>(NT_loc) * 3 * N;    // after the spins (16-byte aligned)
  const int loc0 = r0 * NT + part * NT_loc;               // first local lattice's slot
  const uint32_t lat_base = static_cast<uint32_t>(sg) * p.R + static_cast<uint32_t>(loc0);
  const uint32_t t_hb0 = p.counters[0], t_pt0 = p.counters[1];
  const int G_set = G_sub;                                // groups swept by this CTA
  const ResidentWarps rw = resident_warps(G_set / GP, min(p.warps, static_cast<int>(blockDim.x >> 5)));

  // replica set -> shared memory, parity-split rows -> colour split; one
  // element = the V interleaved lattices of a site
  using VecT = typename std::conditional<V == 2, float2, float>::type;
  {
    const VecT* src = reinterpret_cast<const VecT*>(gsp);
    VecT* dst = reinterpret_cast<VecT*>(sp);
    for (int q = threadIdx.x; q < G_set * 3 * N; q += blockDim.x) {
      const int gc = q / N, i = q - gc * N;
      dst[gc * N + colour_split_index(i, L, N)] = src[q];
    }
  }
  if constexpr (JS != 0) {
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
      const int d = q / N, i = q - d * N;
      const int o = d * N + colour_split_index(i, L, N);
      if constexpr (JS == 2) {
        float j[6];
        load_bond<PREC>(Jg, q, j, p.D);
        float2* d2 = reinterpret_cast<float2*>(static_cast<float*>(Js) + 6 * o);
        d2[0] = make_float2(j[0], j[1]);
        d2[1] = make_float2(j[2], j[3]);
        d2[2] = make_float2(j[4], j[5]);
      } else if constexpr (PREC == kPrecBimodal) {
        static_cast<uint8_t*>(Js)[o] = static_cast<const uint8_t*>(Jg)[q];
      } else if constexpr (PREC == kPrecF16) {
        const uint4 u = static_cast<const uint4*>(Jg)[q];
        uint32_t* w = static_cast<uint32_t*>(Js) + 3 * o;
        w[0] = u.x;
        w[1] = u.y;
        w[2] = u.z;
      } else {
        const float2* s2 = reinterpret_cast<const float2*>(static_cast<const float*>(Jg) + 6 * static_cast<size_t>(q));
        float2* d2 = reinterpret_cast<float2*>(static_cast<float*>(Js) + 6 * o);
        d2[0] = s2[0];
        d2[1] = s2[1];
        d2[2] = s2[2];
      }
    }
  }
  // labels of the sets held: (set j, temperature k) -> local lattice
  for (int q = threadIdx.x; q < sets * NT; q += blockDim.x) {
    const int j = q / NT, k = q - j * NT;
    const int slot = p.perm[(static_cast<size_t>(sg) * p.n_rep + r0 + j) * NT + k];
    const int li = slot - loc0;
    s_perm[q] = li;
    if (li >= 0 && li < NT_loc) s_beta_lat[li] = static_cast<float>(p.beta[k]);
    s_acc[q] = 0;
  }
  __syncthreads();

  for (int step = 0; step < p.steps; ++step) {
    const uint32_t t = t_hb0 + static_cast<uint32_t>(step);
    resident_half_sweep<kHB, false, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 0, s_beta_lat, lat_base, t,
                                                     p.key, s_part);
    __syncthreads();
    if (p.n_or == 0) {
      resident_half_sweep<kHB, true, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 1, s_beta_lat, lat_base, t,
                                                      p.key, s_part);
    } else {
      resident_half_sweep<kHB, false, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 1, s_beta_lat, lat_base, t,
                                                       p.key, s_part);
      __syncthreads();
      for (int o = 0; o < p.n_or; ++o) {
        resident_half_sweep<kOR, false, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 0, s_beta_lat, lat_base,
                                                         t, p.key, s_part);
        __syncthreads();
        if (o + 1 < p.n_or) {
          resident_half_sweep<kOR, false, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 1, s_beta_lat, lat_base,
                                                           t, p.key, s_part);
          __syncthreads();
        } else {
          resident_half_sweep<kOR, true, V, PREC, JS, LT, GP>(sp, Js, Jg, p.D, L, rw, G_set, 1, s_beta_lat, lat_base,
                                                          t, p.key, s_part);
        }
      }
    }
    __syncthreads();
    // energies of the local lattices, fixed-order sums of the warp partials
    if (threadIdx.x < NT_loc) {
      const int g = threadIdx.x / V, v = threadIdx.x - g * V;
      double e = 0.0;
      for (int w = 0; w < rw.wpg; ++w) e += s_part[(g * rw.wpg + w) * V + v];
      s_E[threadIdx.x] = e;
    }
    __syncthreads();
    // parallel tempering within each replica set (App. A.1) this CTA holds
    // whole, one thread per set
    if (whole && threadIdx.x < sets && NT > 1) {
      const int j = threadIdx.x;
      const uint32_t gset = static_cast<uint32_t>(sg) * p.n_rep + static_cast<uint32_t>(r0 + j);
      int* pm = s_perm + j * NT;
      int* ac = s_acc + j * NT;
      const uint32_t tp = t_pt0 + static_cast<uint32_t>(step);
      for (int k = 0; k + 1 < NT; ++k) {
        const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(k), gset, tp, kTagTempering), p.key);
        const double u = uniform52(w.x, w.y);
        const int a = pm[k], b = pm[k + 1];
        const double delta = (p.beta[k] - p.beta[k + 1]) * (s_E[a] - s_E[b]);
        if (delta >= 0.0 || u < exp(delta)) {
          pm[k] = b;
          pm[k + 1] = a;
          ac[k] += 1;
        }
      }
      for (int k = 0; k < NT; ++k) s_beta_lat[pm[k]] = static_cast<float>(p.beta[k]);
    }
    __syncthreads();
  }

  // shared memory -> replica set; energies, labels and acceptances out
  {
    const VecT* src = reinterpret_cast<const VecT*>(sp);
    VecT* dst = reinterpret_cast<VecT*>(gsp);
    for (int q = threadIdx.x; q < G_set * 3 * N; q += blockDim.x) {
      const int gc = q / N, i = q - gc * N;
      dst[q] = src[gc * N + colour_split_index(i, L, N)];
    }
  }
  if (threadIdx.x < NT_loc) p.E[static_cast<size_t>(sg) * p.R + loc0 + threadIdx.x] = s_E[threadIdx.x];
  if (whole) {  // labels and acceptances of the sets held (parts of a set: PT follows)
    for (int q = threadIdx.x; q < sets * NT; q += blockDim.x) {
      const int j = q / NT, k = q - j * NT;
      const size_t pbase = (static_cast<size_t>(sg) * p.n_rep + r0 + j) * NT;
      const int li = s_perm[q];
      p.perm[pbase + k] = li + loc0;
      p.temp_of[static_cast<size_t>(sg) * p.R + loc0 + li] = k;
      if (k + 1 < NT || NT == 1) {
        const int stride = NT > 1 ? NT - 1 : 1;
        p.accepted[(static_cast<size_t>(sg) * p.n_rep + r0 + j) * stride + k] += s_acc[q];
      }
    }
  }
}

#define HSG_PERSISTENT_SHARED                                                    \
  extern __shared__ __align__(16) float sp[];                                     \
  __shared__ double s_E[kMaxTempsResident];                                       \
  __shared__ double s_part[kMaxTempsResident * 2];                                \
  __shared__ float s_beta_lat[kMaxTempsResident];                                 \
  __shared__ int s_perm[kMaxTempsResident];                                       \
  __shared__ int s_acc[kMaxTempsResident];                                        \
  const PersistentShared sh{s_E, s_part, s_beta_lat, s_perm, s_acc}

// Resident steps of one bucket (one L): CTA b holds the sets numbered b.
template <int V, int PREC, int JS, int LT, int GP = 1>
__global__ void __launch_bounds__(persistent_max_threads<LT>(), persistent_min_blocks<LT>())
    k_persistent(PersistentParams p) {
  HSG_PERSISTENT_SHARED;
  persistent_body<V, PREC, JS, LT, GP>(p, blockIdx.x, sp, sh);
}

// Resident steps of two buckets of different L in one launch: the first
// ctas_a CTAs run bucket a, the others bucket b, all with the launch's block
// size and shared memory (the larger of the two buckets' needs), so the
// CTAs of both sizes share the GPU and neither bucket's last wave runs alone.
template <int V, int PREC, int JSA, int LA, int GPA, int JSB, int LB, int GPB>
__global__ void __launch_bounds__(kPairMaxThreads, 1)
    k_persistent_pair(PersistentParams a, PersistentParams b, int ctas_a) {
  HSG_PERSISTENT_SHARED;
  if (static_cast<int>(blockIdx.x) < ctas_a)
    persistent_body<V, PREC, JSA, LA, GPA>(a, blockIdx.x, sp, sh);
  else
    persistent_body<V, PREC, JSB, LB, GPB>(b, blockIdx.x - ctas_a, sp, sh);
}

}  // namespace hsg
