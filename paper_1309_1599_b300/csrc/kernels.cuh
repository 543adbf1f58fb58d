// Device kernels of libhsg: checkerboard heat-bath / overrelaxation sweeps with
// the fused energy, parallel tempering and the overlap/chirality measurement.
//
// Device layout of one bucket (samples of equal L; N = L^3 sites, V lattices
// interleaved per element, G = R/V lattice groups per sample):
//   spins   float [S_b][G][3][N][V]   component planes, lattice lane innermost
//   J f32   float [S_b][3][N][6]      bond (x, x+e_mu) at [mu][site]: xx,yy,zz,xy,xz,yz
//   J f16   half  [S_b][3][N][8]      same six entries + two zero pads (16 B/bond)
// Storage order of the sites ("parity-split rows"): row = y + L*z, and within
// a row the L/2 sites of even x come first, then the L/2 sites of odd x:
//   site(x, y, z) = (y + L*z)*L + (x & 1)*(L/2) + (x >> 1).
// Black sites have x+y+z even.  Random-number counters always use the
// natural index x + L*(y + L*z), so they do not depend on the storage order.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "philox.cuh"

namespace hsg {

enum : int { kHB = 0, kOR = 1, kEnergyOnly = 2 };
// Coupling storage: FP32 (6 floats), FP16 (6 halves + 2 pads, one 16-B
// load) or bimodal (one byte: the signs of J = +-1 and of the six D = +-D).
enum : int { kPrecF32 = 0, kPrecF16 = 1, kPrecBimodal = 2 };
constexpr int kSweepThreads = 256;

struct BucketView {
  float* spins;
  const void* J;
  const int* sample_ids;  // [S_b] global sample index
  int L, N, S_b, G;
  float D;                // bimodal couplings: magnitude of the anisotropy
};

struct SweepParams {
  BucketView b;
  int colour;              // 0 black, 1 white
  int chunks;              // blocks per lattice group
  int R;                   // lattices per sample
  const int* temp_of;      // [S][R] temperature index of each slot
  const float* beta_f;     // [N_T]
  uint2 key;               // Philox key
  const uint32_t* counters;  // [0] heat-bath sweep counter, [1] PT counter
  double* e_partial;       // [S_b*R][chunks] energy partials, or null
};

// ---------------------------------------------------------------------------
// Loads
// ---------------------------------------------------------------------------
// One bimodal bond (Sec. II.A): bit 0 is the sign of the isotropic coupling
// J = +-1, bits 1..6 the signs of D^xx, D^yy, D^zz, D^xy, D^xz, D^yz = +-D
// (a set bit means negative); the six stored entries of J I + D follow.
__device__ __forceinline__ void decode_bimodal(uint32_t bits, float D, float (&j)[6]) {
  const float eps = __int_as_float(0x3f800000 | ((bits & 1u) << 31));
  const uint32_t d = __float_as_uint(D);
  float dd[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) dd[k] = __uint_as_float(d ^ (((bits >> (k + 1)) & 1u) << 31));
  j[0] = eps + dd[0];
  j[1] = eps + dd[1];
  j[2] = eps + dd[2];
  j[3] = dd[3];
  j[4] = dd[4];
  j[5] = dd[5];
}

// The couplings of bucket sample sb (3 N bonds), in the storage format.
template <int PREC>
__device__ __forceinline__ const void* sample_bonds(const void* J, int sb, int N) {
  const size_t off = static_cast<size_t>(sb) * 3 * N;
  if constexpr (PREC == kPrecF32) return static_cast<const float*>(J) + off * 6;
  else if constexpr (PREC == kPrecF16) return static_cast<const uint4*>(J) + off;
  else return static_cast<const uint8_t*>(J) + off;
}

// Bond number `bond` of J as six FP32 entries (xx, yy, zz, xy, xz, yz).  D is
// used by the bimodal format only.
template <int PREC>
__device__ __forceinline__ void load_bond(const void* J, size_t bond, float (&j)[6], float D) {
  if constexpr (PREC == kPrecBimodal) {
    decode_bimodal(__ldg(static_cast<const uint8_t*>(J) + bond), D, j);
  } else if constexpr (PREC == kPrecF32) {
    const float2* p = reinterpret_cast<const float2*>(static_cast<const float*>(J) + bond * 6);
    const float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    j[0] = a.x; j[1] = a.y; j[2] = b.x; j[3] = b.y; j[4] = c.x; j[5] = c.y;
  } else {
    const uint4 u = __ldg(static_cast<const uint4*>(J) + bond);
    __half2 h0, h1, h2;
    *reinterpret_cast<uint32_t*>(&h0) = u.x;
    *reinterpret_cast<uint32_t*>(&h1) = u.y;
    *reinterpret_cast<uint32_t*>(&h2) = u.z;
    const float2 a = __half22float2(h0), b = __half22float2(h1), c = __half22float2(h2);
    j[0] = a.x; j[1] = a.y; j[2] = b.x; j[3] = b.y; j[4] = c.x; j[5] = c.y;
  }
}

template <int V>
__device__ __forceinline__ void load_spin(const float* base, size_t plane, int i, float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(base + c * plane) + i);
      s[c][0] = t.x;
      s[c][1] = t.y;
    } else {
      s[c][0] = __ldg(base + c * plane + i);
    }
  }
}

template <int V>
__device__ __forceinline__ void store_spin(float* base, size_t plane, int i, const float (&s)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (V == 2) {
      reinterpret_cast<float2*>(base + c * plane)[i] = make_float2(s[c][0], s[c][1]);
    } else {
      base[c * plane + i] = s[c][0];
    }
  }
}

// h += J s for the symmetric J = [[xx,xy,xz],[xy,yy,yz],[xz,yz,zz]].  With
// two interleaved lattices the pair (lattice 0, lattice 1) is one packed
// FP32x2 fused multiply-add per matrix element (same rounding per lane as
// fmaf, so results do not depend on V).
template <int V>
__device__ __forceinline__ void add_bond(const float (&j)[6], const float (&s)[3][V], float (&h)[3][V]) {
  if constexpr (V == 2) {
    const float2 s0 = make_float2(s[0][0], s[0][1]), s1 = make_float2(s[1][0], s[1][1]),
                 s2 = make_float2(s[2][0], s[2][1]);
    float2 h0 = make_float2(h[0][0], h[0][1]), h1 = make_float2(h[1][0], h[1][1]),
           h2 = make_float2(h[2][0], h[2][1]);
    h0 = __ffma2_rn(make_float2(j[0], j[0]), s0,
                    __ffma2_rn(make_float2(j[3], j[3]), s1, __ffma2_rn(make_float2(j[4], j[4]), s2, h0)));
    h1 = __ffma2_rn(make_float2(j[3], j[3]), s0,
                    __ffma2_rn(make_float2(j[1], j[1]), s1, __ffma2_rn(make_float2(j[5], j[5]), s2, h1)));
    h2 = __ffma2_rn(make_float2(j[4], j[4]), s0,
                    __ffma2_rn(make_float2(j[5], j[5]), s1, __ffma2_rn(make_float2(j[2], j[2]), s2, h2)));
    h[0][0] = h0.x; h[0][1] = h0.y;
    h[1][0] = h1.x; h[1][1] = h1.y;
    h[2][0] = h2.x; h[2][1] = h2.y;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      h[0][v] = fmaf(j[0], s[0][v], fmaf(j[3], s[1][v], fmaf(j[4], s[2][v], h[0][v])));
      h[1][v] = fmaf(j[3], s[0][v], fmaf(j[1], s[1][v], fmaf(j[5], s[2][v], h[1][v])));
      h[2][v] = fmaf(j[4], s[0][v], fmaf(j[5], s[1][v], fmaf(j[2], s[2][v], h[2][v])));
    }
  }
}

// ---------------------------------------------------------------------------
// Single-spin updates (App. A.1)
// ---------------------------------------------------------------------------
// Heat-bath: s ~ exp(beta s.h) on the sphere.  u = cos(angle to h) by the
// inverse CDF written for w = 1 - u (w = -log1p(r0 expm1(-2 kappa))/kappa,
// kappa = beta|h|, continuous limit 2 r0 for kappa < 1e-30); azimuth 2 pi r1
// in the orthonormal frame of Duff et al. (JCGT 6(1), 2017); axis e_z if h=0.
__device__ __forceinline__ void heat_bath_draw(float hx, float hy, float hz, float beta,
                                               uint32_t w0, uint32_t w1,
                                               float& sx, float& sy, float& sz) {
  const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
  const float inv = (hh > 0.0f) ? rsqrtf(hh) : 0.0f;   // 1/|h| (2 ulp)
  const float hn = hh * inv;
  const float kappa = beta * hn;
  const float r0 = uniform23(w0);
  const float r1 = uniform23(w1);
  // w = -log(1 - y)/kappa with y = r0 (1 - e^{-2 kappa}).  In binary32 the
  // single expression log1p(r0 expm1(-2 kappa)) loses all accuracy when y is
  // close to 1 (expm1 rounds to -1 and 1 - y cancels), so the two regimes are
  // evaluated separately: log1p(-y) for y < 1/2, and for y >= 1/2 the
  // logarithm of 1 - y = (1 - r0) + r0 e^{-2 kappa}, a sum of two positive
  // terms in which 1 - r0 is exact.  For kappa > 1/2, 1 - e^{-2 kappa} >= 0.63
  // cannot cancel, so the fast exponential serves both terms; expm1 is kept
  // for small kappa, where 1 - e^{-2 kappa} is small.  For y >= 1/2 the
  // argument of the logarithm lies in (0, 1/2], where the fast logarithm's
  // relative error (about 2^-21) leaves w accurate to ~5e-7 relative.  For
  // y < 1/2 w must stay accurate near the pole, where sin(theta) ~ sqrt(2w)
  // would amplify an absolute error: log1p for kappa <= 1/2, and for
  // kappa > 1/2 a series below y = 1/16 and the fast logarithm above.
  float w;
  if (kappa < 1e-30f) {
    w = 2.0f * r0;
  } else {
    float lg;
    if (kappa > 0.5f) {
      const float e2k = __expf(-2.0f * kappa);
      const float y = fmaf(-r0, e2k, r0);
      // Without branches: one fast logarithm serves y >= 1/16, of 1 - y for
      // y < 1/2 (1 - y rounds by at most 2^-25 there, and the logarithm's
      // absolute error of 2^-21.4 leaves w within 7.2e-7 for kappa > 1/2,
      // while sin(theta) >= 0.92) or of the sum above for y >= 1/2; below
      // y = 1/16 the Mercator series of log(1 - y) to y^7 is used
      // (truncation error below 1e-9 relative).
      const float arg = (y < 0.5f) ? 1.0f - y : fmaf(r0, e2k, 1.0f - r0);
      const float lf = __logf(arg);
      const float ps =
          y * fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, fmaf(y, 1.0f / 7.0f, 1.0f / 6.0f), 0.2f), 0.25f),
                                         1.0f / 3.0f), 0.5f), 1.0f);
      lg = (y < 0.0625f) ? -ps : lf;
    } else {
      const float em = expm1f(-2.0f * kappa);
      const float e2k = em + 1.0f;
      const float y = -r0 * em;
      lg = (y < 0.5f) ? log1pf(-y) : __logf(fmaf(r0, e2k, 1.0f - r0));
    }
    w = __fdividef(-lg, kappa);
  }
  w = fminf(fmaxf(w, 0.0f), 2.0f);
  // 1 + u = 2 - w.  Near the antipole (u -> -1) it is small and cancels in
  // 2 - w, which sin(theta) = sqrt(w (2 - w)) would magnify; for w > 1.99
  // (sin(theta) < 0.14) it is evaluated directly as 2 - w = log1p((1 - r0)
  // (e^{2 kappa} - 1)) / kappa, with 1 - r0 exact.  There (1 - r0)
  // (e^{2 kappa} - 1) < e^{0.01 kappa} - 1 stays below 1/2, and w > 1.99 needs
  // 1 - r0 < e^{-1.99 kappa}, so kappa < 8.4 (1 - r0 >= 2^-24) and
  // e^{2 kappa} is finite; the kappa bound below is a second guard.
  float wc = 2.0f - w;
  if (w > 1.99f && kappa >= 1e-30f && kappa < 40.0f) {
    wc = __fdividef(log1pf((1.0f - r0) * expm1f(2.0f * kappa)), kappa);
    w = 2.0f - wc;
  }
  const float u = 1.0f - w;
  const float w2 = fmaxf(w * wc, 0.0f);
  const float st = (w2 > 0.0f) ? w2 * rsqrtf(w2) : 0.0f;   // sin(theta), 2 ulp
  // azimuth phi = 2 pi r1: evaluated as phi - pi in (-pi, pi), where the
  // fast sine and cosine are accurate to 2^-21.4, then reflected
  float sp, cp;
  __sincosf(6.283185307179586f * (r1 - 0.5f), &sp, &cp);
  sp = -sp;
  cp = -cp;
  float nx = 0.0f, ny = 0.0f, nz = 1.0f;
  if (hh > 0.0f) {
    nx = hx * inv;
    ny = hy * inv;
    nz = hz * inv;
  }
  const float sgn = copysignf(1.0f, nz);
  const float p = __fdividef(-1.0f, sgn + nz);   // |sgn + nz| in [1, 2]
  const float q = nx * ny * p;
  const float e1x = fmaf(sgn * nx * nx, p, 1.0f), e1y = sgn * q, e1z = -sgn * nx;
  const float e2x = q, e2y = fmaf(ny * ny, p, sgn), e2z = -ny;
  const float ax = fmaf(cp, e1x, sp * e2x), ay = fmaf(cp, e1y, sp * e2y), az = fmaf(cp, e1z, sp * e2z);
  sx = fmaf(u, nx, st * ax);
  sy = fmaf(u, ny, st * ay);
  sz = fmaf(u, nz, st * az);
}

// Heat-bath draws of the two lattices of one site: the operations of
// heat_bath_draw lane for lane, with the multiply-add arithmetic of the common
// case (kappa > 1/2 in both lanes, no antipole correction) as FP32x2
// instructions, which round each lane as the scalar ones do.  Any other case
// is drawn by heat_bath_draw itself, so the draws equal it bit for bit.
__device__ __forceinline__ void heat_bath_draw2(const float (&h)[3][2], const float (&beta)[2], uint32_t w0a,
                                                uint32_t w1a, uint32_t w0b, uint32_t w1b, float (&s)[3][2]) {
  const float2 hx = make_float2(h[0][0], h[0][1]), hy = make_float2(h[1][0], h[1][1]),
               hz = make_float2(h[2][0], h[2][1]);
  const float2 hh = __ffma2_rn(hx, hx, __ffma2_rn(hy, hy, __fmul2_rn(hz, hz)));
  const float2 inv = make_float2((hh.x > 0.0f) ? rsqrtf(hh.x) : 0.0f, (hh.y > 0.0f) ? rsqrtf(hh.y) : 0.0f);
  const float2 kappa = __fmul2_rn(make_float2(beta[0], beta[1]), __fmul2_rn(hh, inv));
  const float2 r0 = make_float2(uniform23(w0a), uniform23(w0b));
  const float2 e2k = make_float2(__expf(-2.0f * kappa.x), __expf(-2.0f * kappa.y));
  const float2 nr0 = make_float2(-r0.x, -r0.y);
  const float2 one = make_float2(1.0f, 1.0f);
  const float2 y = __ffma2_rn(nr0, e2k, r0);
  const float2 a_lo = __fadd2_rn(one, make_float2(-y.x, -y.y));
  const float2 a_hi = __ffma2_rn(r0, e2k, __fadd2_rn(one, nr0));
  const float lfx = __logf((y.x < 0.5f) ? a_lo.x : a_hi.x), lfy = __logf((y.y < 0.5f) ? a_lo.y : a_hi.y);
  const float2 c7 = make_float2(1.0f / 7.0f, 1.0f / 7.0f), c6 = make_float2(1.0f / 6.0f, 1.0f / 6.0f),
               c5 = make_float2(0.2f, 0.2f), c4 = make_float2(0.25f, 0.25f),
               c3 = make_float2(1.0f / 3.0f, 1.0f / 3.0f), c2 = make_float2(0.5f, 0.5f);
  const float2 ps = __fmul2_rn(
      y, __ffma2_rn(y, __ffma2_rn(y, __ffma2_rn(y, __ffma2_rn(y, __ffma2_rn(y, __ffma2_rn(y, c7, c6), c5), c4), c3),
                                  c2), one));
  const float lgx = (y.x < 0.0625f) ? -ps.x : lfx, lgy = (y.y < 0.0625f) ? -ps.y : lfy;
  float2 w = make_float2(__fdividef(-lgx, kappa.x), __fdividef(-lgy, kappa.y));
  w.x = fminf(fmaxf(w.x, 0.0f), 2.0f);
  w.y = fminf(fmaxf(w.y, 0.0f), 2.0f);
  if (!(kappa.x > 0.5f && kappa.y > 0.5f) || w.x > 1.99f || w.y > 1.99f) {
    heat_bath_draw(h[0][0], h[1][0], h[2][0], beta[0], w0a, w1a, s[0][0], s[1][0], s[2][0]);
    heat_bath_draw(h[0][1], h[1][1], h[2][1], beta[1], w0b, w1b, s[0][1], s[1][1], s[2][1]);
    return;
  }
  const float2 nw = make_float2(-w.x, -w.y);
  const float2 wc = __fadd2_rn(make_float2(2.0f, 2.0f), nw);
  const float2 u = __fadd2_rn(one, nw);
  const float2 ww = __fmul2_rn(w, wc);
  const float2 w2 = make_float2(fmaxf(ww.x, 0.0f), fmaxf(ww.y, 0.0f));
  const float2 sq = __fmul2_rn(w2, make_float2(rsqrtf(w2.x), rsqrtf(w2.y)));
  const float2 st = make_float2((w2.x > 0.0f) ? sq.x : 0.0f, (w2.y > 0.0f) ? sq.y : 0.0f);
  const float2 r1 = make_float2(uniform23(w1a), uniform23(w1b));
  const float2 phi = __fmul2_rn(make_float2(6.283185307179586f, 6.283185307179586f),
                                __fadd2_rn(r1, make_float2(-0.5f, -0.5f)));
  float2 sp, cp;
  __sincosf(phi.x, &sp.x, &cp.x);
  __sincosf(phi.y, &sp.y, &cp.y);
  sp = make_float2(-sp.x, -sp.y);
  cp = make_float2(-cp.x, -cp.y);
  const float2 px = __fmul2_rn(hx, inv), py = __fmul2_rn(hy, inv), pz = __fmul2_rn(hz, inv);
  const float2 nx = make_float2((hh.x > 0.0f) ? px.x : 0.0f, (hh.y > 0.0f) ? px.y : 0.0f);
  const float2 ny = make_float2((hh.x > 0.0f) ? py.x : 0.0f, (hh.y > 0.0f) ? py.y : 0.0f);
  const float2 nz = make_float2((hh.x > 0.0f) ? pz.x : 1.0f, (hh.y > 0.0f) ? pz.y : 1.0f);
  const float2 sgn = make_float2(copysignf(1.0f, nz.x), copysignf(1.0f, nz.y));
  const float2 sn = __fadd2_rn(sgn, nz);
  const float2 p = make_float2(__fdividef(-1.0f, sn.x), __fdividef(-1.0f, sn.y));
  const float2 q = __fmul2_rn(__fmul2_rn(nx, ny), p);
  const float2 e1x = __ffma2_rn(__fmul2_rn(__fmul2_rn(sgn, nx), nx), p, one);
  const float2 e1y = __fmul2_rn(sgn, q);
  const float2 e1z = __fmul2_rn(make_float2(-sgn.x, -sgn.y), nx);
  const float2 e2x = q;
  const float2 e2y = __ffma2_rn(__fmul2_rn(ny, ny), p, sgn);
  const float2 e2z = make_float2(-ny.x, -ny.y);
  const float2 ax = __ffma2_rn(cp, e1x, __fmul2_rn(sp, e2x));
  const float2 ay = __ffma2_rn(cp, e1y, __fmul2_rn(sp, e2y));
  const float2 az = __ffma2_rn(cp, e1z, __fmul2_rn(sp, e2z));
  const float2 sx = __ffma2_rn(u, nx, __fmul2_rn(st, ax));
  const float2 sy = __ffma2_rn(u, ny, __fmul2_rn(st, ay));
  const float2 sz = __ffma2_rn(u, nz, __fmul2_rn(st, az));
  s[0][0] = sx.x; s[0][1] = sx.y;
  s[1][0] = sy.x; s[1][1] = sy.y;
  s[2][0] = sz.x; s[2][1] = sz.y;
}

// The heat-bath draws of the V lattices lat0 .. lat0+V-1 of one site from one
// Philox block w: a lattice takes the words (x, y) if its index is even and
// (z, w) if it is odd.
template <int V>
__device__ __forceinline__ void heat_bath_site(const float (&h)[3][V], const float (&beta)[V], uint4 w,
                                               uint32_t lat0, float (&s)[3][V]) {
  if constexpr (V == 2) {
    const bool odd = (lat0 & 1u) != 0;
    heat_bath_draw2(h, beta, odd ? w.z : w.x, odd ? w.w : w.y, odd ? w.x : w.z, odd ? w.y : w.w, s);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const uint32_t lat = lat0 + v;
      heat_bath_draw(h[0][v], h[1][v], h[2][v], beta[v], (lat & 1u) ? w.z : w.x, (lat & 1u) ? w.w : w.y,
                     s[0][v], s[1][v], s[2][v]);
    }
  }
}

// Overrelaxation: reflection of s about h, s' = 2h(h.s)/h^2 - s.
__device__ __forceinline__ void overrelax(float hx, float hy, float hz, float& sx, float& sy, float& sz) {
  const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
  if (hh > 0.0f) {
    const float hs = fmaf(hx, sx, fmaf(hy, sy, hz * sz));
    const float f = __fdividef(2.0f * hs, hh);  // |h|^2 is O(1..100): well inside its range
    sx = fmaf(f, hx, -sx);
    sy = fmaf(f, hy, -sy);
    sz = fmaf(f, hz, -sz);
  }
}

// Overrelaxation of V lattices at once (the two interleaved lattices share
// packed FP32x2 arithmetic; each lane rounds exactly like overrelax()).
template <int V>
__device__ __forceinline__ void overrelax_v(const float (&h)[3][V], float (&s)[3][V]) {
  if constexpr (V == 2) {
    const float2 hx = make_float2(h[0][0], h[0][1]), hy = make_float2(h[1][0], h[1][1]),
                 hz = make_float2(h[2][0], h[2][1]);
    const float2 sx = make_float2(s[0][0], s[0][1]), sy = make_float2(s[1][0], s[1][1]),
                 sz = make_float2(s[2][0], s[2][1]);
    const float2 hh = __ffma2_rn(hx, hx, __ffma2_rn(hy, hy, __fmul2_rn(hz, hz)));
    const float2 hs = __ffma2_rn(hx, sx, __ffma2_rn(hy, sy, __fmul2_rn(hz, sz)));
    const float2 f = make_float2(__fdividef(2.0f * hs.x, hh.x), __fdividef(2.0f * hs.y, hh.y));
    const float2 nx = __ffma2_rn(f, hx, make_float2(-sx.x, -sx.y));
    const float2 ny = __ffma2_rn(f, hy, make_float2(-sy.x, -sy.y));
    const float2 nz = __ffma2_rn(f, hz, make_float2(-sz.x, -sz.y));
    if (hh.x > 0.0f) {
      s[0][0] = nx.x; s[1][0] = ny.x; s[2][0] = nz.x;
    }
    if (hh.y > 0.0f) {
      s[0][1] = nx.y; s[1][1] = ny.y; s[2][1] = nz.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) overrelax(h[0][v], h[1][v], h[2][v], s[0][v], s[1][v], s[2][v]);
  }
}

// Storage index of site (x, row) with row = y + L*z: parity-split when SPLIT,
// natural order x + L*row otherwise.
template <bool SPLIT>
__device__ __forceinline__ int site_of(int x, int row, int L) {
  if constexpr (SPLIT) return row * L + (x & 1) * (L >> 1) + (x >> 1);
  return row * L + x;
}

// The field of a site is accumulated in two partial sums -- the bonds to
// x+1, y+1, z+1 (in that order) and to x-1, y-1, z-1 -- added at the end.
// Two independent chains of FMAs halve the dependent latency; every sweep
// kernel uses this same order, so their results agree bit for bit.
template <int V>
__device__ __forceinline__ void zero3(float (&h)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) h[c][v] = 0.0f;
}

template <int V>
__device__ __forceinline__ void combine_field(const float (&hf)[3][V], const float (&hb)[3][V], float (&h)[3][V]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) h[c][v] = hf[c][v] + hb[c][v];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// One colour half-sweep of every lattice of a bucket.  Thread = one site of
// the colour x V lattices of one group; the six neighbours are of the other
// colour and are only read.  With e_partial set, each block also writes
// -sum s.h over its sites (per lattice) -- on the white half this is the
// lattice energy, since every bond has exactly one white end and
// overrelaxation keeps s.h.
// ---------------------------------------------------------------------------
template <int KIND, int V, int PREC, bool SPLIT = false>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_half(SweepParams p) {
  const BucketView& b = p.b;
  const int gi = blockIdx.x / p.chunks;  // lattice group within the bucket
  const int chunk = blockIdx.x - gi * p.chunks;
  const int ic = chunk * kSweepThreads + threadIdx.x;
  const int L = b.L, N = b.N, half = L >> 1;
  const bool active = ic < (N >> 1);
  const int sb = gi / b.G, g = gi - sb * b.G;
  float e_acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) e_acc[v] = 0.0f;

  if (active) {
    const int row = ic / half;
    const int k = ic - row * half;
    const int y = row % L;
    const int z = row / L;
    const int x = 2 * k + ((p.colour + y + z) & 1);
    const int i_nat = x + L * row;
    const int i = site_of<SPLIT>(x, row, L);
    const int LL = L * L;
    const int ixm = site_of<SPLIT>((x == 0) ? L - 1 : x - 1, row, L);
    const int ixp = site_of<SPLIT>((x == L - 1) ? 0 : x + 1, row, L);
    const int iym = (y == 0) ? i + (L - 1) * L : i - L;
    const int iyp = (y == L - 1) ? i - (L - 1) * L : i + L;
    const int izm = (z == 0) ? i + (L - 1) * LL : i - LL;
    const int izp = (z == L - 1) ? i - (L - 1) * LL : i + LL;

    float* base = b.spins + static_cast<size_t>(gi) * 3 * N * V;
    const size_t plane = static_cast<size_t>(N) * V;
    const size_t jb = static_cast<size_t>(sb) * 3 * N;

    float h[3][V], hf[3][V], hb[3][V];
    zero3<V>(hf);
    zero3<V>(hb);
    float j[6];
    float s[3][V];
    load_bond<PREC>(b.J, jb + i, j, b.D);              load_spin<V>(base, plane, ixp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(b.J, jb + N + i, j, b.D);          load_spin<V>(base, plane, iyp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(b.J, jb + 2 * size_t(N) + i, j, b.D);   load_spin<V>(base, plane, izp, s); add_bond<V>(j, s, hf);
    load_bond<PREC>(b.J, jb + ixm, j, b.D);            load_spin<V>(base, plane, ixm, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(b.J, jb + N + iym, j, b.D);        load_spin<V>(base, plane, iym, s); add_bond<V>(j, s, hb);
    load_bond<PREC>(b.J, jb + 2 * size_t(N) + izm, j, b.D); load_spin<V>(base, plane, izm, s); add_bond<V>(j, s, hb);
    combine_field<V>(hf, hb, h);

    if constexpr (KIND == kHB) {
      const uint32_t t = p.counters[0];
      const int sg = b.sample_ids[sb];
      const uint32_t lat0 = static_cast<uint32_t>(sg) * p.R + static_cast<uint32_t>(g * V);
      const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(i_nat), lat0 >> 1, t, kTagHeatBath), p.key);
      float out[3][V], beta[V];
#pragma unroll
      for (int v = 0; v < V; ++v) beta[v] = p.beta_f[p.temp_of[static_cast<size_t>(sg) * p.R + g * V + v]];
      heat_bath_site<V>(h, beta, w, lat0, out);
      store_spin<V>(base, plane, i, out);
    } else {
      float o[3][V];
      load_spin<V>(base, plane, i, o);
      if constexpr (KIND == kOR) {
        overrelax_v<V>(h, o);
        store_spin<V>(base, plane, i, o);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) e_acc[v] = fmaf(o[0][v], h[0][v], fmaf(o[1][v], h[1][v], o[2][v] * h[2][v]));
    }
  }

  if (p.e_partial != nullptr) {
    __shared__ double red[V][kSweepThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const double d = warp_sum(-static_cast<double>(e_acc[v]));
      if (lane == 0) red[v][warp] = d;
    }
    __syncthreads();
    if (threadIdx.x < V) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kSweepThreads / 32; ++w) acc += red[threadIdx.x][w];
      const size_t lat_local = static_cast<size_t>(sb) * p.R + g * V + threadIdx.x;
      p.e_partial[lat_local * p.chunks + chunk] = acc;
    }
  }
}

// E[sample*R + slot] = sum of the chunk partials of that lattice, one warp per
// lattice, fixed summation order.
static __global__ void k_energy_finalize(const double* __restrict__ partial, int chunks, int n_lat,
                                  const int* __restrict__ sample_ids, int R, double* __restrict__ E) {
  const int lat = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (lat >= n_lat) return;
  double acc = 0.0;
  for (int c = lane; c < chunks; c += 32) acc += partial[static_cast<size_t>(lat) * chunks + c];
  acc = warp_sum(acc);
  if (lane == 0) {
    const int sb = lat / R, slot = lat - sb * R;
    E[static_cast<size_t>(sample_ids[sb]) * R + slot] = acc;
  }
}

// ---------------------------------------------------------------------------
// Parallel tempering (App. A.1): one thread per replica set.
// ---------------------------------------------------------------------------
static __global__ void k_pt_sweep(int n_sets, int n_rep, int NT, int R, const double* __restrict__ beta,
                           const double* __restrict__ E, int* __restrict__ perm,
                           int* __restrict__ temp_of, long long* __restrict__ accepted, uint2 key,
                           const uint32_t* __restrict__ counters) {
  const int gset = blockIdx.x * blockDim.x + threadIdx.x;
  if (gset >= n_sets) return;
  const int s = gset / n_rep;
  int* pm = perm + static_cast<size_t>(gset) * NT;
  const double* Es = E + static_cast<size_t>(s) * R;
  const uint32_t t = counters[1];
  const int acc_stride = NT > 1 ? NT - 1 : 1;
  for (int k = 0; k + 1 < NT; ++k) {
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(gset), t,
                                             kTagTempering), key);
    const double r = uniform52(w.x, w.y);
    const int a = pm[k], c = pm[k + 1];
    const double delta = (beta[k] - beta[k + 1]) * (Es[a] - Es[c]);
    if (delta >= 0.0 || r < exp(delta)) {
      pm[k] = c;
      pm[k + 1] = a;
      accepted[static_cast<size_t>(gset) * acc_stride + k] += 1;
    }
  }
  for (int k = 0; k < NT; ++k) temp_of[static_cast<size_t>(s) * R + pm[k]] = k;
}

// The same parallel-tempering sweep with one warp per replica set, for up to
// kPtWarpMaxTemps temperatures: the lanes stage the set's labels, the
// energies of the lattices they point at and the random numbers of every
// pair in shared memory, lane 0 runs the sequential sweep over the pairs in
// k_pt_sweep's order and arithmetic (so the decisions are the same bit for
// bit), and the lanes write the labels and acceptances back.  The sweep no
// longer waits on a global load per pair.
constexpr int kPtWarpMaxTemps = 256;

static __global__ void __launch_bounds__(32) k_pt_sweep_warp(int n_rep, int NT, int R,
                                                             const double* __restrict__ beta,
                                                             const double* __restrict__ E, int* __restrict__ perm,
                                                             int* __restrict__ temp_of,
                                                             long long* __restrict__ accepted, uint2 key,
                                                             const uint32_t* __restrict__ counters) {
  __shared__ int s_lab[kPtWarpMaxTemps];
  __shared__ double s_en[kPtWarpMaxTemps], s_beta[kPtWarpMaxTemps], s_r[kPtWarpMaxTemps];
  __shared__ unsigned char s_acc[kPtWarpMaxTemps];
  const int gset = blockIdx.x;
  const int lane = threadIdx.x;
  const int s = gset / n_rep;
  int* pm = perm + static_cast<size_t>(gset) * NT;
  const double* Es = E + static_cast<size_t>(s) * R;
  const uint32_t t = counters[1];
  for (int k = lane; k < NT; k += 32) {
    const int a = pm[k];
    s_lab[k] = a;
    s_en[k] = Es[a];
    s_beta[k] = beta[k];
    s_acc[k] = 0;
    if (k + 1 < NT) {
      const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(k), static_cast<uint32_t>(gset), t,
                                               kTagTempering), key);
      s_r[k] = uniform52(w.x, w.y);
    }
  }
  __syncwarp();
  if (lane == 0) {
    for (int k = 0; k + 1 < NT; ++k) {
      const double delta = (s_beta[k] - s_beta[k + 1]) * (s_en[k] - s_en[k + 1]);
      if (delta >= 0.0 || s_r[k] < exp(delta)) {
        const int a = s_lab[k];
        s_lab[k] = s_lab[k + 1];
        s_lab[k + 1] = a;
        const double e = s_en[k];
        s_en[k] = s_en[k + 1];
        s_en[k + 1] = e;
        s_acc[k] = 1;
      }
    }
  }
  __syncwarp();
  const int acc_stride = NT > 1 ? NT - 1 : 1;
  for (int k = lane; k < NT; k += 32) {
    pm[k] = s_lab[k];
    temp_of[static_cast<size_t>(s) * R + s_lab[k]] = k;
    if (s_acc[k]) accepted[static_cast<size_t>(gset) * acc_stride + k] += 1;
  }
}

static __global__ void k_bump_counters(uint32_t* counters, uint32_t d_hb, uint32_t d_pt) {
  counters[0] += d_hb;
  counters[1] += d_pt;
}

// Host spins [N][3] in natural site order (staged on the device) <-> one lane
// of the device layout (parity-split storage order).
static __global__ void k_scatter_spins(const float* __restrict__ stage, float* __restrict__ base, int L, int V, int v) {
  const int N = L * L * L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int d = site_of<true>(i % L, i / L, L);
  const size_t plane = static_cast<size_t>(N) * V;
  for (int c = 0; c < 3; ++c) base[c * plane + static_cast<size_t>(d) * V + v] = stage[3 * static_cast<size_t>(i) + c];
}

static __global__ void k_gather_spins(const float* __restrict__ base, float* __restrict__ stage, int L, int V, int v) {
  const int N = L * L * L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int d = site_of<true>(i % L, i / L, L);
  const size_t plane = static_cast<size_t>(N) * V;
  for (int c = 0; c < 3; ++c) stage[3 * static_cast<size_t>(i) + c] = base[c * plane + static_cast<size_t>(d) * V + v];
}

static __global__ void k_fill_spins(float* __restrict__ spins, size_t n_per_comp_block, size_t total) {
  // Sets every spin to (0,0,1): component 2 planes to 1, others to 0.
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const size_t comp = (idx / n_per_comp_block) % 3;
  spins[idx] = comp == 2 ? 1.0f : 0.0f;
}

static __global__ void k_philox_eval(const uint32_t* __restrict__ in, long n, uint32_t* __restrict__ out) {
  const long r = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t* q = in + 6 * r;
  const uint4 w = philox4x32_10(make_uint4(q[0], q[1], q[2], q[3]), make_uint2(q[4], q[5]));
  out[4 * r + 0] = w.x;
  out[4 * r + 1] = w.y;
  out[4 * r + 2] = w.z;
  out[4 * r + 3] = w.w;
}

}  // namespace hsg
