// Fused checkerboard sweep: one pass over the lattice updates every black
// site and then every white site (App. A.1: black half with the old white
// spins, white half with the new black spins), reading each spin once from
// HBM and writing it once.
//
// A CTA owns one lattice group (V lattices of one sample; or GP groups, each
// thread updating its sites in all of them) and a band of `band_rows` rows y
// (all x), and marches through the planes z.  At step z it
// updates the black sites of plane z and then the white sites of plane z-1:
// black(z) needs the white spins of planes z-1, z, z+1 before they change,
// white(z-1) needs the black spins of planes z-2, z-1, z after they changed.
//   * Planes are staged in shared memory by 1-D bulk TMA copies
//     (cp.async.bulk, mbarrier completion) into a ring of 4 slots, issued two
//     planes ahead.  A slot holds the band plus two halo rows on each side.
//   * Each thread owns one x-pair (2k, 2k+1) of one row: at every plane it
//     holds one black and one white site.  The z-neighbours of its sites are
//     its own sites at the neighbouring planes, kept in registers; shared
//     memory serves only the in-plane neighbours (rows are stored
//     parity-split, so these reads are contiguous across a warp).
//   * Spins are read from one buffer and written to the other (ping-pong), so
//     the halo rows of neighbouring bands and the periodic wrap in z are read
//     unmodified.  The march covers planes 0..L+1; black(0) and black(1) are
//     recomputed at the end (same inputs, same random numbers) for white(0).
//   * Halo rows: the black sites of the rows just outside the band are
//     updated too (not stored), because the band's white sites need them.
//     With band_rows == L a CTA holds whole planes and rows wrap in y.
//   * The field is summed in the same order as in k_sweep_half (+x, -x, +y,
//     -y, +z, -z), so both kernels give the same spins bit for bit.
//   * Waits on the TMA barriers are bounded (clock64); on expiry the kernel
//     writes HSG_ETIMEOUT to *status, waits (bounded) for its copies in
//     flight and returns; no thread ever spins without limit.
#pragma once
#include "kernels.cuh"

namespace hsg {

constexpr int kFusedMaxThreads = 576;
constexpr int kFusedSlots = 4;
constexpr int kStatusTimeout = 4;                 // value of HSG_ETIMEOUT
constexpr long long kCleanupWait = 2000000000LL;  // cycles, per outstanding copy

struct FusedParams {
  const float* in;        // spins before the sweep, bucket layout
  float* out;             // spins after the sweep
  const void* J;
  const int* sample_ids;  // [S_b] global sample index
  int L, N, G, R;
  int band_rows;          // rows written per CTA; == L for whole planes
  int n_bands;            // L / band_rows
  const int* temp_of;     // [S][R]
  const float* beta_f;    // [N_T]
  uint2 key;
  const uint32_t* counters;
  double* e_partial;      // [S_b*R][n_bands] or null
  int* status;            // device status word
  long long timeout;      // clock64 cycles for one wait
  int probe_timeout;      // nonzero: first wait on a barrier nobody completes
  float D;                // bimodal couplings: magnitude of the anisotropy
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long timeout) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > timeout) return false;
  }
  return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int V>
__device__ __forceinline__ void lds_site(const float* p, float (&s)[3][V], int comp_stride) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      const float2 t = *reinterpret_cast<const float2*>(p + c * comp_stride);
      s[c][0] = t.x;
      s[c][1] = t.y;
    } else {
      s[c][0] = p[c * comp_stride];
    }
  }
}

template <int V>
__device__ __forceinline__ void sts_site(float* p, const float (&s)[3][V], int comp_stride) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      *reinterpret_cast<float2*>(p + c * comp_stride) = make_float2(s[c][0], s[c][1]);
    } else {
      p[c * comp_stride] = s[c][0];
    }
  }
}

template <int V>
__device__ __forceinline__ void stg_site(float* p, const float (&s)[3][V], size_t comp_stride) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      *reinterpret_cast<float2*>(p + c * comp_stride) = make_float2(s[c][0], s[c][1]);
    } else {
      p[c * comp_stride] = s[c][0];
    }
  }
}

template <int V>
__device__ __forceinline__ void copy3(float (&d)[3][V], const float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) d[c][v] = s[c][v];
}

// Local field h = sum over the six bonds of J s_neighbour (J symmetric) of
// one site in each of GP lattice groups, accumulated as in k_sweep_half
// (forward bonds x+1, y+1, z+1 and backward bonds x-1, y-1, z-1 in two
// partial sums).  Each bond is loaded and converted once and serves all GP
// groups; every lattice's sums are those of a single group, so the result
// does not depend on GP.  Jb points at the sample's couplings; pos, pos_xm,
// pos_ym, pos_zm are the storage positions of the site and of its neighbours
// at x-1, y-1, z-1 (whose +x, +y, +z bonds are this site's -x, -y, -z
// bonds).  jz_up / jz_dn: the +z / -z bond, already loaded by the caller (or
// null: load it here).
template <int GP, int V, int PREC>
__device__ __forceinline__ void site_field(const void* Jb, float D, int N, int pos, int pos_xm, int pos_ym,
                                           int pos_zm, const float (&xp)[GP][3][V], const float (&xm)[GP][3][V],
                                           const float (&yu)[GP][3][V], const float (&yd)[GP][3][V],
                                           const float (&zu)[GP][3][V], const float (&zd)[GP][3][V],
                                           float (&h)[GP][3][V], const float* jz_up = nullptr,
                                           const float* jz_dn = nullptr) {
  float hf[GP][3][V], hb[GP][3][V], j[6];
#pragma unroll
  for (int g = 0; g < GP; ++g) {
    zero3<V>(hf[g]);
    zero3<V>(hb[g]);
  }
  load_bond<PREC>(Jb, pos, j, D);
#pragma unroll
  for (int g = 0; g < GP; ++g) add_bond<V>(j, xp[g], hf[g]);
  load_bond<PREC>(Jb, N + pos, j, D);
#pragma unroll
  for (int g = 0; g < GP; ++g) add_bond<V>(j, yu[g], hf[g]);
  if (jz_up) {
#pragma unroll
    for (int e = 0; e < 6; ++e) j[e] = jz_up[e];
  } else {
    load_bond<PREC>(Jb, 2 * N + pos, j, D);
  }
#pragma unroll
  for (int g = 0; g < GP; ++g) add_bond<V>(j, zu[g], hf[g]);
  load_bond<PREC>(Jb, pos_xm, j, D);
#pragma unroll
  for (int g = 0; g < GP; ++g) add_bond<V>(j, xm[g], hb[g]);
  load_bond<PREC>(Jb, N + pos_ym, j, D);
#pragma unroll
  for (int g = 0; g < GP; ++g) add_bond<V>(j, yd[g], hb[g]);
  if (jz_dn) {
#pragma unroll
    for (int e = 0; e < 6; ++e) j[e] = jz_dn[e];
  } else {
    load_bond<PREC>(Jb, 2 * N + pos_zm, j, D);
  }
#pragma unroll
  for (int g = 0; g < GP; ++g) {
    add_bond<V>(j, zd[g], hb[g]);
    combine_field<V>(hf[g], hb[g], h[g]);
  }
}

// A site's V lattices as a set of one group (same storage), for site_field.
template <int V>
__device__ __forceinline__ float (&one_group(float (&s)[3][V]))[1][3][V] {
  return *reinterpret_cast<float(*)[1][3][V]>(&s);
}

template <int KIND, int V>
__device__ __forceinline__ void update_site(const float (&h)[3][V], float (&s)[3][V], const float (&beta)[V],
                                            uint32_t i_nat, uint32_t lat0, uint32_t t, uint2 key) {
  if constexpr (KIND == kHB) {
    const uint4 w = philox4x32_10(make_uint4(i_nat, lat0 >> 1, t, kTagHeatBath), key);
    heat_bath_site<V>(h, beta, w, lat0, s);
  } else {
    overrelax_v<V>(h, s);
  }
}

// The site of every one of the GP groups: group g's planes follow group
// g-1's in a slot (gstride floats apart) and in global memory.
template <int GP, int V>
__device__ __forceinline__ void lds_sites(const float* p, float (&s)[GP][3][V], int comp_stride, int gstride) {
#pragma unroll
  for (int g = 0; g < GP; ++g) lds_site<V>(p + g * gstride, s[g], comp_stride);
}

// Registers per thread of the fused sweep: 96 holds one group's working set
// with two CTAs per SM; two groups per thread run one CTA per SM (their ring
// takes twice the shared memory) and get the registers that frees.
template <int GP>
constexpr int fused_max_regs() {
  return GP == 1 ? 96 : 168;
}

// LT, BT: the lattice size and band height as compile-time constants (the
// common tilings), or 0 to take them from p at run time.  With constants the
// ring-slot strides and plane parities fold into immediate offsets once the
// march over z is unrolled by the ring period.  GP: lattice groups (of V
// lattices of one sample) per CTA; a thread updates its sites in all GP
// groups, so each bond load and conversion serves GP * V lattices.
template <int KIND, int V, int PREC, int LT = 0, int BT = 0, int GP = 1>
__global__ void __maxnreg__(fused_max_regs<GP>()) k_sweep_fused(FusedParams p) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t bars[kFusedSlots + 1];  // [kFusedSlots]: never completed
  __shared__ double s_red[GP * V][kFusedMaxThreads / 32];
  __shared__ int s_failed;

  const int L = LT > 0 ? LT : p.L, half = L >> 1, N = L * L * L;
  const int band_rows = BT > 0 ? BT : p.band_rows;
  const int n_bands = L / band_rows;
  const bool full = (band_rows == L);
  const int slot_rows = full ? L : band_rows + 4;
  const int row_f = L * V;                        // floats per staged row
  const int comp_f = slot_rows * row_f;           // floats per component in a slot
  const int grp_f = 3 * comp_f;                   // floats per group in a slot
  const int slot_f = GP * grp_f;
  const int gs = blockIdx.x / n_bands;            // set of GP groups
  const int band = blockIdx.x - gs * n_bands;
  const int GS = p.G / GP;                        // sets per sample
  const int sb = gs / GS, g0 = (gs - sb * GS) * GP;
  const int y0 = band * band_rows;
  const int tid = threadIdx.x;
  const int rows_t = full ? L : band_rows + 2;
  const bool active = tid < rows_t * half;
  const int rt = active ? tid / half : 0;
  const int k = active ? tid - rt * half : 0;
  const int r = full ? rt : rt + 1;               // row within a slot
  const int y = full ? rt : (y0 - 2 + r + L) % L; // lattice row
  const bool owner = active && (full || (r >= 2 && r < band_rows + 2));
  const int r_up = full ? (r + 1 == L ? 0 : r + 1) : r + 1;
  const int r_dn = full ? (r == 0 ? L - 1 : r - 1) : r - 1;
  const int k_up = (k + 1 == half) ? 0 : k + 1;
  const int k_dn = (k == 0) ? half - 1 : k - 1;
  const int y_dn = (y == 0) ? L - 1 : y - 1;
  const size_t plane_g = static_cast<size_t>(N) * V;   // component stride in global memory
  const size_t gbase = static_cast<size_t>(gs) * GP * 3 * plane_g;
  const float* in_g = p.in + gbase;
  float* out_g = p.out + gbase;
  // couplings of this sample (element size depends on the storage precision)
  const void* Jb = sample_bonds<PREC>(p.J, sb, N);
  const bool want_energy = (p.e_partial != nullptr);
  const int LL = L * L;
  const int yrow = y * L, ydrow = y_dn * L;

  float beta[GP][V];
  uint32_t lat0[GP], t_hb = 0;
  if constexpr (KIND == kHB) {
    const int sg = p.sample_ids[sb];
    t_hb = p.counters[0];
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      lat0[g] = static_cast<uint32_t>(sg) * p.R + static_cast<uint32_t>((g0 + g) * V);
#pragma unroll
      for (int v = 0; v < V; ++v)
        beta[g][v] = p.beta_f[p.temp_of[static_cast<size_t>(sg) * p.R + (g0 + g) * V + v]];
    }
  } else {
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      lat0[g] = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) beta[g][v] = 0.0f;
    }
  }

  const uint32_t slot_bytes = static_cast<uint32_t>(slot_f) * 4u;
  const int ystart = full ? 0 : (y0 - 2 + L) % L;
  // Virtual plane vp (from -1 to L+2) lives in slot (vp+1) & 3.
  auto issue = [&](int vp) {
    const int pl = (vp + L) % L;
    const int s = (vp + 1) & 3;
    float* dst = smem + s * slot_f;
    mbar_expect_tx(&bars[s], slot_bytes);
    for (int c = 0; c < 3 * GP; ++c) {  // component c % 3 of group c / 3
      int done = 0;
      while (done < slot_rows) {
        const int yy = (ystart + done) % L;
        const int n = min(slot_rows - done, L - yy);
        const float* src = in_g + c * plane_g + (static_cast<size_t>(pl) * L + yy) * row_f;
        bulk_copy_g2s(dst + c * comp_f + done * row_f, src, static_cast<uint32_t>(n * row_f * 4), &bars[s]);
        done += n;
      }
    }
  };
  auto parity_of = [](int vp) -> uint32_t { return static_cast<uint32_t>(((vp + 1) >> 2) & 1); };
  // Site (row rr, x-parity a, pair kk) of group 0 in the slot holding virtual
  // plane vp.
  auto at = [&](int vp, int rr, int a, int kk) -> float* {
    return smem + ((vp + 1) & 3) * slot_f + rr * row_f + (a * half + kk) * V;
  };

  if (tid == 0) {
    for (int s = 0; s <= kFusedSlots; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_failed = 0;
  }
  __syncthreads();
  int issued = -2;  // highest virtual plane issued (meaningful in thread 0)
  if (tid == 0) {
    for (int vp = -1; vp <= 2; ++vp) issue(vp);
    issued = 2;
  }

  // Registers hold only the new black spins of this thread's column at the
  // two previous planes (their slots are refilled before they are needed
  // again) and of the current plane; everything else is read from the
  // resident slots: planes z-1, z (in-plane neighbours, old white spins,
  // new black spins) and z+1.
  float Bm2[GP][3][V], Bm1[GP][3][V], B0[GP][3][V];
#pragma unroll
  for (int g = 0; g < GP; ++g) {
    zero3<V>(Bm2[g]);
    zero3<V>(Bm1[g]);
  }
  double e_acc[GP][V];
#pragma unroll
  for (int g = 0; g < GP; ++g)
#pragma unroll
    for (int v = 0; v < V; ++v) e_acc[g][v] = 0.0;

  int first_unwaited = -1;  // lowest virtual plane not yet known complete
  bool ok = true;
  if (p.probe_timeout) ok = mbar_wait_bounded(&bars[kFusedSlots], 0, p.timeout);
  ok = ok && mbar_wait_bounded(&bars[0], parity_of(-1), p.timeout);
  ok = ok && mbar_wait_bounded(&bars[1], parity_of(0), p.timeout);
  bool failed = __syncthreads_or(!ok) != 0;
  if (!failed) first_unwaited = 1;

#pragma unroll(LT > 0 ? 4 : 1)
  for (int z = 0; !failed && z <= L + 1; ++z) {
    // A thread whose wait expires flags the CTA; everyone sees the flag after
    // this step's barrier (the step's results are then discarded).
    if (!mbar_wait_bounded(&bars[(z + 2) & 3], parity_of(z + 1), p.timeout)) s_failed = 1;
    const int pz = z % L;
    if (active) {
      // black site of plane z: x-parity ab, from the old white spins; its
      // column's white sites at z-1 and z+1 have the same x-parity
      const int ab = (y + pz) & 1;
      const int pz_dn = (pz == 0) ? L - 1 : pz - 1;
      const bool do_white = (z >= 2 && owner);
      const int q = (z + L - 1) % L;  // plane of the white update
      const int q_dn = (q == 0) ? L - 1 : q - 1;
      const int aw = ab;              // white site of plane z-1 in this column
      const int plq = q * LL;
      float xp[GP][3][V], xm[GP][3][V], yu[GP][3][V], yd[GP][3][V], zu[GP][3][V], zd[GP][3][V], h[GP][3][V];
      lds_sites<GP, V>(at(z, r, ab, k), B0, comp_f, grp_f);
      lds_sites<GP, V>(at(z, r, ab ^ 1, ab ? k_up : k), xp, comp_f, grp_f);
      lds_sites<GP, V>(at(z, r, ab ^ 1, ab ? k : k_dn), xm, comp_f, grp_f);
      lds_sites<GP, V>(at(z, r_up, ab, k), yu, comp_f, grp_f);
      lds_sites<GP, V>(at(z, r_dn, ab, k), yd, comp_f, grp_f);
      lds_sites<GP, V>(at(z + 1, r, ab, k), zu, comp_f, grp_f);
      lds_sites<GP, V>(at(z - 1, r, ab, k), zd, comp_f, grp_f);
      // the z bond between this column's sites at planes z-1 and z: the
      // black site's -z bond and the +z bond of the white site updated below
      float jz[6];
      load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + pz_dn * LL + yrow + ab * half + k, jz, p.D);
      {
        const int pl = pz * LL;
        site_field<GP, V, PREC>(Jb, p.D, N, pl + yrow + ab * half + k, pl + yrow + (ab ? k : half + k_dn),
                                pl + ydrow + ab * half + k, pz_dn * LL + yrow + ab * half + k, xp, xm, yu, yd,
                                zu, zd, h, nullptr, jz);
      }
      const uint32_t i_nat = static_cast<uint32_t>(2 * k + ab + L * (y + L * pz));
#pragma unroll
      for (int g = 0; g < GP; ++g) {
        update_site<KIND, V>(h[g], B0[g], beta[g], i_nat, lat0[g], t_hb, p.key);
        sts_site<V>(at(z, r, ab, k) + g * grp_f, B0[g], comp_f);
      }

      // white site of plane z-1 from the new black spins
      if (do_white) {
        float w[GP][3][V];
        lds_sites<GP, V>(at(z - 1, r, aw, k), w, comp_f, grp_f);
        lds_sites<GP, V>(at(z - 1, r, aw ^ 1, aw ? k_up : k), xp, comp_f, grp_f);
        lds_sites<GP, V>(at(z - 1, r, aw ^ 1, aw ? k : k_dn), xm, comp_f, grp_f);
        lds_sites<GP, V>(at(z - 1, r_up, aw, k), yu, comp_f, grp_f);
        lds_sites<GP, V>(at(z - 1, r_dn, aw, k), yd, comp_f, grp_f);
        site_field<GP, V, PREC>(Jb, p.D, N, plq + yrow + aw * half + k, plq + yrow + (aw ? k : half + k_dn),
                                plq + ydrow + aw * half + k, q_dn * LL + yrow + aw * half + k, xp, xm, yu, yd,
                                B0, Bm2, h, jz, nullptr);
        const uint32_t iw_nat = static_cast<uint32_t>(2 * k + aw + L * (y + L * q));
        float* dst = out_g + static_cast<size_t>(plq + yrow) * V;
#pragma unroll
        for (int g = 0; g < GP; ++g) {
          update_site<KIND, V>(h[g], w[g], beta[g], iw_nat, lat0[g], t_hb, p.key);
          if (want_energy) {
#pragma unroll
            for (int v = 0; v < V; ++v)
              e_acc[g][v] += static_cast<double>(
                  fmaf(w[g][0][v], h[g][0][v], fmaf(w[g][1][v], h[g][1][v], w[g][2][v] * h[g][2][v])));
          }
          stg_site<V>(dst + g * 3 * plane_g + ((aw ^ 1) * half + k) * V, Bm1[g], plane_g);
          stg_site<V>(dst + g * 3 * plane_g + (aw * half + k) * V, w[g], plane_g);
        }
      }
    }
    // Generic-proxy accesses of the slot being refilled must precede the
    // asynchronous copy that overwrites it.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_failed) {
      failed = true;
      break;
    }
    first_unwaited = z + 2;
    if (tid == 0 && z + 3 <= L + 2) {
      issue(z + 3);
      issued = z + 3;
    }
#pragma unroll
    for (int g = 0; g < GP; ++g) {
      copy3<V>(Bm2[g], Bm1[g]);
      copy3<V>(Bm1[g], B0[g]);
    }
  }

  if (failed) {
    // Record the expiry and wait (bounded) for this CTA's copies in flight
    // before its shared memory is released.
    if (tid == 0) {
      atomicExch(p.status, kStatusTimeout);
      for (int vp = first_unwaited; vp <= issued; ++vp)
        mbar_wait_bounded(&bars[(vp + 1) & 3], parity_of(vp), kCleanupWait);
    }
    return;
  }

  if (p.e_partial != nullptr) {
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int g = 0; g < GP; ++g)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double d = warp_sum(-e_acc[g][v]);
        if (lane == 0) s_red[g * V + v][warp] = d;
      }
    __syncthreads();
    if (tid < GP * V) {
      double acc = 0.0;
      const int nw = (blockDim.x + 31) >> 5;
      for (int w = 0; w < nw; ++w) acc += s_red[tid][w];
      const size_t lat_local = static_cast<size_t>(sb) * p.R + g0 * V + tid;
      p.e_partial[lat_local * n_bands + band] = acc;
    }
  }
}

}  // namespace hsg
