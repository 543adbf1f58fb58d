// Measurement kernels (Sec. II.B): the overlap and chiral-overlap sums of
// every replica pair at every temperature, with their Fourier components
// and the Schwinger-Dyson residual, accumulated in FP64.
#pragma once
#include "kernels.cuh"

namespace hsg {

constexpr int kMeasureThreads = 256;
constexpr int kNQ = 30;  // raw measurement sums per pair, see k_measure
// Sites per thread summed in FP32 before the sums are added to the FP64
// accumulators: every per-site term is at most 1 in magnitude, so a batch's
// FP32 rounding stays below 2e-6 of its terms; 32 rather than 8 sites per
// flush took the L = 64 measurement from 2.83 to 2.28 ms (the FP64 adds and
// the shared-memory accumulator traffic quartered), 64 was slower again.
constexpr int kMeasureBatch = 32;

// ---------------------------------------------------------------------------
// Measurement (Sec. II.B).  One block per (sample, temperature k, replica
// pair, chunk of sites).  Per site: q = s^a.s^b, the chiralities
// zeta_mu = s_{x+mu}.(s_x x s_{x-mu}) of both replicas, kappa_mu = zeta^a
// zeta^b, the Fourier sums at k = 0 and k_nu = 2 pi e_nu / L, and the
// Schwinger-Dyson terms 2T s.h - h^2 + (s.h)^2 of both lattices.
// Raw sums (kNQ = 30): [0] q, [1+2nu,2+2nu] q cos, q sin, [7+mu] kappa_mu,
// [10+2(3mu+nu), 11+...] kappa_mu cos, sin, [28] SD_a, [29] SD_b.
// FP32 within batches of kMeasureBatch sites, FP64 across batches and threads.
// ---------------------------------------------------------------------------
struct MeasureParams {
  BucketView b;
  int R, n_rep, NT, P, chunks;
  const int* perm;      // [S][n_rep][NT]
  const double* beta;   // [NT]
  const float* phase;   // [L][2]: cos, sin of 2 pi x / L
  double* partial;      // [S_b][NT][P][chunks][kNQ]
};

template <int V>
__device__ __forceinline__ void load_one(const float* base, size_t plane, int i, float (&s)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) s[c] = __ldg(base + c * plane + static_cast<size_t>(i) * V);
}

__device__ __forceinline__ float triple(const float (&up)[3], const float (&a)[3], const float (&dn)[3]) {
  const float cx = a[1] * dn[2] - a[2] * dn[1];
  const float cy = a[2] * dn[0] - a[0] * dn[2];
  const float cz = a[0] * dn[1] - a[1] * dn[0];
  return fmaf(up[0], cx, fmaf(up[1], cy, up[2] * cz));
}

__device__ __forceinline__ void add_bond1(const float (&j)[6], const float (&s)[3], float (&h)[3]) {
  h[0] = fmaf(j[0], s[0], fmaf(j[3], s[1], fmaf(j[4], s[2], h[0])));
  h[1] = fmaf(j[3], s[0], fmaf(j[1], s[1], fmaf(j[5], s[2], h[1])));
  h[2] = fmaf(j[4], s[0], fmaf(j[5], s[1], fmaf(j[2], s[2], h[2])));
}

// The raw sums of one site i of the replica pair (base_a, base_b), added to
// part[kNQ].
template <int V, int PREC>
__device__ __forceinline__ void measure_site(const void* J, float D, size_t jb, const float* sh_phase,
                                             const float* base_a, const float* base_b, size_t plane, int L, int N,
                                             int i, bool do_sd, float T, float (&part)[kNQ]) {
  const int row = i / L, jr = i - row * L;
  const int half = L >> 1;
  const int x = (jr < half) ? 2 * jr : 2 * (jr - half) + 1;
  const int y = row % L, z = row / L;
  const int LL = L * L;
  const int nb[6] = {site_of<true>((x == L - 1) ? 0 : x + 1, row, L),
                     site_of<true>((x == 0) ? L - 1 : x - 1, row, L),
                     (y == L - 1) ? i - (L - 1) * L : i + L, (y == 0) ? i + (L - 1) * L : i - L,
                     (z == L - 1) ? i - (L - 1) * LL : i + LL, (z == 0) ? i + (L - 1) * LL : i - LL};
  float sa[3], sbv[3];
  load_one<V>(base_a, plane, i, sa);
  load_one<V>(base_b, plane, i, sbv);
  float ha[3] = {0.f, 0.f, 0.f}, hb[3] = {0.f, 0.f, 0.f};
  float za[3], zb[3];
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    float ua[3], da[3], ub[3], db[3];
    load_one<V>(base_a, plane, nb[2 * mu], ua);
    load_one<V>(base_a, plane, nb[2 * mu + 1], da);
    load_one<V>(base_b, plane, nb[2 * mu], ub);
    load_one<V>(base_b, plane, nb[2 * mu + 1], db);
    za[mu] = triple(ua, sa, da);
    zb[mu] = triple(ub, sbv, db);
    if (do_sd) {
      float j[6];
      load_bond<PREC>(J, jb + static_cast<size_t>(mu) * N + i, j, D);
      add_bond1(j, ua, ha);
      add_bond1(j, ub, hb);
      load_bond<PREC>(J, jb + static_cast<size_t>(mu) * N + nb[2 * mu + 1], j, D);
      add_bond1(j, da, ha);
      add_bond1(j, db, hb);
    }
  }
  const float q = fmaf(sa[0], sbv[0], fmaf(sa[1], sbv[1], sa[2] * sbv[2]));
  const float c[3] = {sh_phase[2 * x], sh_phase[2 * y], sh_phase[2 * z]};
  const float s[3] = {sh_phase[2 * x + 1], sh_phase[2 * y + 1], sh_phase[2 * z + 1]};
  part[0] += q;
#pragma unroll
  for (int nu = 0; nu < 3; ++nu) {
    part[1 + 2 * nu] = fmaf(q, c[nu], part[1 + 2 * nu]);
    part[2 + 2 * nu] = fmaf(q, s[nu], part[2 + 2 * nu]);
  }
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const float kap = za[mu] * zb[mu];
    part[7 + mu] += kap;
#pragma unroll
    for (int nu = 0; nu < 3; ++nu) {
      part[10 + 2 * (3 * mu + nu)] = fmaf(kap, c[nu], part[10 + 2 * (3 * mu + nu)]);
      part[11 + 2 * (3 * mu + nu)] = fmaf(kap, s[nu], part[11 + 2 * (3 * mu + nu)]);
    }
  }
  if (do_sd) {
    const float sha = fmaf(sa[0], ha[0], fmaf(sa[1], ha[1], sa[2] * ha[2]));
    const float hha = fmaf(ha[0], ha[0], fmaf(ha[1], ha[1], ha[2] * ha[2]));
    const float shb = fmaf(sbv[0], hb[0], fmaf(sbv[1], hb[1], sbv[2] * hb[2]));
    const float hhb = fmaf(hb[0], hb[0], fmaf(hb[1], hb[1], hb[2] * hb[2]));
    part[28] += 2.0f * T * sha - (hha - sha * sha);
    part[29] += 2.0f * T * shb - (hhb - shb * shb);
  }
}

// Replica pair of measurement unit `unit` = (sample, temperature k, pair pp).
struct MeasureUnit {
  const float* base_a;
  const float* base_b;
  size_t jb;
  bool do_sd;
  float T;
};

template <int V>
__device__ __forceinline__ MeasureUnit measure_unit(const MeasureParams& p, int unit) {
  const BucketView& b = p.b;
  const int N = b.N;
  const int pp = unit % p.P;
  const int k = (unit / p.P) % p.NT;
  const int sb = unit / (p.P * p.NT);
  const int sg = b.sample_ids[sb];
  const int slot_a = p.perm[(static_cast<size_t>(sg) * p.n_rep + 2 * pp) * p.NT + k];
  const bool has_b = 2 * pp + 1 < p.n_rep;
  const int slot_b = has_b ? p.perm[(static_cast<size_t>(sg) * p.n_rep + 2 * pp + 1) * p.NT + k] : slot_a;
  const size_t plane = static_cast<size_t>(N) * V;
  MeasureUnit m;
  m.base_a = b.spins + (static_cast<size_t>(sb) * b.G + slot_a / V) * 3 * plane + slot_a % V;
  m.base_b = b.spins + (static_cast<size_t>(sb) * b.G + slot_b / V) * 3 * plane + slot_b % V;
  m.jb = static_cast<size_t>(sb) * 3 * N;
  const double beta = p.beta[k];
  m.do_sd = beta > 0.0;
  m.T = m.do_sd ? static_cast<float>(1.0 / beta) : 0.0f;
  return m;
}

// Dynamic shared memory of k_measure and k_measure_warp: the per-thread FP64
// accumulators [kNQ][kMeasureThreads], then the phase table [L][2].
constexpr size_t measure_block_smem(int L) {
  return sizeof(double) * kNQ * kMeasureThreads + 2 * sizeof(float) * static_cast<size_t>(L);
}

// One block per (unit, chunk of sites).  FP32 within batches of
// kMeasureBatch sites, FP64 across batches (each thread's accumulators live in shared memory, so
// that two blocks fit per SM) and threads.
template <int V, int PREC>
__global__ void __launch_bounds__(kMeasureThreads, 2) k_measure(MeasureParams p) {
  extern __shared__ __align__(16) double m_acc[];                 // [kNQ][kMeasureThreads]
  float* sh_phase = reinterpret_cast<float*>(m_acc + kNQ * kMeasureThreads);  // [L][2]
  __shared__ double red[kMeasureThreads / 32][kNQ];
  const BucketView& b = p.b;
  const int L = b.L, N = b.N;
  for (int t = threadIdx.x; t < 2 * L; t += blockDim.x) sh_phase[t] = p.phase[t];
  double* acc = m_acc + threadIdx.x;                               // stride kMeasureThreads
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q * kMeasureThreads] = 0.0;
  __syncthreads();

  const int unit = blockIdx.x / p.chunks;
  const int chunk = blockIdx.x - unit * p.chunks;
  const MeasureUnit m = measure_unit<V>(p, unit);
  const size_t plane = static_cast<size_t>(N) * V;

  float part[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) part[q] = 0.0f;

  const int per_chunk = (N + p.chunks - 1) / p.chunks;
  const int start = chunk * per_chunk;
  const int end = min(N, start + per_chunk);
  int batch = 0;
  for (int i = start + threadIdx.x; i < end; i += blockDim.x) {
    measure_site<V, PREC>(b.J, b.D, m.jb, sh_phase, m.base_a, m.base_b, plane, L, N, i, m.do_sd, m.T, part);
    if (++batch == kMeasureBatch) {
#pragma unroll
      for (int qq = 0; qq < kNQ; ++qq) {
        acc[qq * kMeasureThreads] += static_cast<double>(part[qq]);
        part[qq] = 0.0f;
      }
      batch = 0;
    }
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int qq = 0; qq < kNQ; ++qq) {
    const double d = warp_sum(acc[qq * kMeasureThreads] + static_cast<double>(part[qq]));
    if (lane == 0) red[warp][qq] = d;
  }
  __syncthreads();
  if (threadIdx.x < kNQ) {
    double sum = 0.0;
    for (int w = 0; w < kMeasureThreads / 32; ++w) sum += red[w][threadIdx.x];
    p.partial[(static_cast<size_t>(unit) * p.chunks + chunk) * kNQ + threadIdx.x] = sum;
  }
}

// Small lattices: one warp per unit over all its sites (p.chunks == 1), so
// the reduction is a warp sum only.  Same per-site terms and batching as
// k_measure, and, as there, each thread's FP64 accumulators live in shared
// memory so that two blocks fit per SM.
template <int V, int PREC>
__global__ void __launch_bounds__(kMeasureThreads, 2) k_measure_warp(MeasureParams p, int n_units) {
  extern __shared__ __align__(16) double m_acc[];                 // [kNQ][kMeasureThreads]
  float* sh_phase = reinterpret_cast<float*>(m_acc + kNQ * kMeasureThreads);  // [L][2]
  const BucketView& b = p.b;
  const int L = b.L, N = b.N;
  for (int t = threadIdx.x; t < 2 * L; t += blockDim.x) sh_phase[t] = p.phase[t];
  double* acc = m_acc + threadIdx.x;                               // stride kMeasureThreads
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q * kMeasureThreads] = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int unit = blockIdx.x * (kMeasureThreads / 32) + warp;
  if (unit >= n_units) return;
  const MeasureUnit m = measure_unit<V>(p, unit);
  const size_t plane = static_cast<size_t>(N) * V;

  float part[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) part[q] = 0.0f;
  int batch = 0;
  for (int i = lane; i < N; i += 32) {
    measure_site<V, PREC>(b.J, b.D, m.jb, sh_phase, m.base_a, m.base_b, plane, L, N, i, m.do_sd, m.T, part);
    if (++batch == kMeasureBatch) {
#pragma unroll
      for (int qq = 0; qq < kNQ; ++qq) {
        acc[qq * kMeasureThreads] += static_cast<double>(part[qq]);
        part[qq] = 0.0f;
      }
      batch = 0;
    }
  }
  double mine = 0.0;
#pragma unroll
  for (int qq = 0; qq < kNQ; ++qq) {
    const double d = warp_sum(acc[qq * kMeasureThreads] + static_cast<double>(part[qq]));
    if (lane == qq) mine = d;
  }
  if (lane < kNQ) p.partial[static_cast<size_t>(unit) * kNQ + lane] = mine;
}

// Turns the raw sums of one bucket into the accumulated observables:
// one thread per (sample, temperature).
static __global__ void k_measure_finalize(const double* __restrict__ partial, const int* __restrict__ sample_ids,
                                   int S_b, int NT, int P, int chunks, int n_rep, int R, int N,
                                   const int* __restrict__ perm, const double* __restrict__ E,
                                   double* __restrict__ obs, long long* __restrict__ counts) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= S_b * NT) return;
  const int sb = u / NT, k = u - sb * NT;
  const int sg = sample_ids[sb];
  const double invN = 1.0 / N;
  double* o = obs + (static_cast<size_t>(sg) * NT + k) * 9;
  for (int pp = 0; pp < P; ++pp) {
    double Q[kNQ];
    for (int q = 0; q < kNQ; ++q) Q[q] = 0.0;
    const size_t unit = (static_cast<size_t>(sb) * NT + k) * P + pp;
    for (int c = 0; c < chunks; ++c)
      for (int q = 0; q < kNQ; ++q) Q[q] += partial[(unit * chunks + c) * kNQ + q];
    const bool has_b = 2 * pp + 1 < n_rep;
    if (has_b) {
      const double q0 = Q[0] * invN;
      double q2k = 0.0;
      for (int nu = 0; nu < 3; ++nu) {
        const double re = Q[1 + 2 * nu] * invN, im = Q[2 + 2 * nu] * invN;
        q2k += re * re + im * im;
      }
      double c2 = 0.0, c4 = 0.0, c2k = 0.0;
      for (int mu = 0; mu < 3; ++mu) {
        const double c0 = Q[7 + mu] * invN;
        c2 += c0 * c0;
        c4 += c0 * c0 * c0 * c0;
        for (int nu = 0; nu < 3; ++nu) {
          const double re = Q[10 + 2 * (3 * mu + nu)] * invN, im = Q[11 + 2 * (3 * mu + nu)] * invN;
          c2k += re * re + im * im;
        }
      }
      o[2] += q0 * q0;
      o[3] += q0 * q0 * q0 * q0;
      o[4] += q2k / 3.0;
      o[5] += c2 / 3.0;
      o[6] += c4 / 3.0;
      o[7] += c2k / 9.0;
      o[8] += (Q[28] + Q[29]) * invN;
    } else {
      o[8] += Q[28] * invN;
    }
  }
  for (int r = 0; r < n_rep; ++r) {
    const int slot = perm[(static_cast<size_t>(sg) * n_rep + r) * NT + k];
    const double e = E[static_cast<size_t>(sg) * R + slot] * invN;
    o[0] += e;
    o[1] += e * e;
  }
  counts[static_cast<size_t>(sg) * NT + k] += 1;
}

}  // namespace hsg
