/*
 * hsg_oracle.c -- plain FP64 CPU oracle for equilibrium Monte Carlo of the
 * 3d Edwards-Anderson Heisenberg spin glass with random anisotropic couplings
 * (Baity-Jesi, Fernandez, Martin-Mayor, Sanz, arXiv:1309.1599).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library; the two agree
 * only through the interface definitions written out below (the Philox
 * counter layout and the uniform mapping), which each side implements on its
 * own.
 *
 * Conventions (all arrays plain C, row-major, caller-owned):
 *   site index      i = x + L*(y + L*z), 0 <= x,y,z < L, periodic boundaries
 *   colour          black if (x+y+z) even, white otherwise (L even)
 *   spins           s[i*3 + a], a = 0,1,2 (components x,y,z)
 *   couplings       J9[(i*3 + mu)*9 + a*3 + b] = J^{ab} of the bond
 *                   (i, i+e_mu), mu = 0,1,2 (+x,+y,+z), stored at the lower
 *                   site; the bond energy is -s_i^T J s_{i+e_mu}.  A general
 *                   (not necessarily symmetric) 3x3 matrix is accepted.
 *
 * Every floating-point operation is IEEE double; no blocking, fusion or
 * reordering beyond the definitions cited at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4xW-10 counter-based generator, written from its published          */
/* definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel  */
/* random numbers: as easy as 1, 2, 3", SC'11.  One round maps the counter    */
/* (c0,c1,c2,c3) with key (k0,k1) to                                          */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),        */
/* where hi/lo are the upper/lower W bits of the 2W-bit product, and the key  */
/* is bumped by the Weyl constants (W0,W1) modulo 2^W between rounds.         */
/* One body serves both word widths W = 32 and W = 64, so that checking the   */
/* 64-bit member against an independent implementation also checks the       */
/* rounds and key schedule of the 32-bit member the Monte Carlo uses.         */
/* The paper itself uses a Parisi-Rapuano + congruential generator (App.      */
/* A.4.1); a counter-based generator replaces it here.                        */
/* ------------------------------------------------------------------------ */
static void philox4xW_10(int W, const uint64_t ctr[4], const uint64_t key[2],
                         uint64_t out[4]) {
  uint64_t M0, M1, W0, W1, mask;
  if (W == 32) {
    M0 = 0xD2511F53ull;
    M1 = 0xCD9E8D57ull;
    W0 = 0x9E3779B9ull;
    W1 = 0xBB67AE85ull;
    mask = 0xFFFFFFFFull;
  } else {
    M0 = 0xD2E7470EE14C6C93ull;
    M1 = 0xCA5A826395121157ull;
    W0 = 0x9E3779B97F4A7C15ull;
    W1 = 0xBB67AE8584CAA73Bull;
    mask = ~0ull;
  }
  uint64_t c0 = ctr[0] & mask, c1 = ctr[1] & mask, c2 = ctr[2] & mask, c3 = ctr[3] & mask;
  uint64_t k0 = key[0] & mask, k1 = key[1] & mask;
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 = (k0 + W0) & mask;
      k1 = (k1 + W1) & mask;
    }
    unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> W) & mask, lo0 = (uint64_t)p0 & mask;
    uint64_t hi1 = (uint64_t)(p1 >> W) & mask, lo1 = (uint64_t)p1 & mask;
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint64_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]}, k[2] = {key[0], key[1]}, o[4];
  philox4xW_10(32, c, k, o);
  for (int j = 0; j < 4; ++j) out[j] = (uint32_t)o[j];
}

/* The 64-bit member is not used by the Monte Carlo; it exists so that the
 * shared body can be checked bit for bit against an independent library. */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                          uint64_t out[4]) {
  philox4xW_10(64, ctr, key, out);
}

/* Uniform in (0,1) from one 32-bit word: the top 23 bits k give
 * (k + 1/2) * 2^-23 = (2k+1) * 2^-24, an odd multiple of 2^-24 that is exact
 * in both binary32 and binary64 (so 1 - r is exact too). */
double oracle_uniform23(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * 0x1p-23;
}

/* Uniform in (0,1) with 52 random bits from two words, exact in binary64:
 * v = (w0 >> 6) * 2^26 + (w1 >> 6), r = (v + 1/2) * 2^-52. */
double oracle_uniform52(uint32_t w0, uint32_t w1) {
  uint64_t v = ((uint64_t)(w0 >> 6) << 26) | (uint64_t)(w1 >> 6);
  return ((double)v + 0.5) * 0x1p-52;
}

/* Stream tags in the fourth counter word. */
#define ORACLE_TAG_HB 1u
#define ORACLE_TAG_PT 2u

/* The two uniforms of a heat-bath draw at site i of lattice `lattice` during
 * heat-bath sweep number t.  Counter (i, lattice/2, t, HB); even lattices take
 * words 0,1, odd lattices words 2,3. */
void oracle_hb_words(uint64_t seed, uint32_t site, uint32_t lattice,
                     uint32_t t, uint32_t w[2]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {site, lattice >> 1, t, ORACLE_TAG_HB};
  uint32_t out[4];
  oracle_philox4x32_10(ctr, key, out);
  if (lattice & 1u) {
    w[0] = out[2];
    w[1] = out[3];
  } else {
    w[0] = out[0];
    w[1] = out[1];
  }
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry                                                          */
/* ------------------------------------------------------------------------ */
static long site_index(int L, int x, int y, int z) {
  return (long)x + (long)L * ((long)y + (long)L * (long)z);
}

/* Neighbour of site i one step along direction mu (0,1,2), sign +1 or -1. */
static long neighbour(int L, long i, int mu, int sign) {
  int x = (int)(i % L);
  int y = (int)((i / L) % L);
  int z = (int)(i / ((long)L * L));
  int c[3] = {x, y, z};
  c[mu] = (c[mu] + sign + L) % L;
  return site_index(L, c[0], c[1], c[2]);
}

static int site_colour(int L, long i) {
  int x = (int)(i % L);
  int y = (int)((i / L) % L);
  int z = (int)(i / ((long)L * L));
  return (x + y + z) & 1;
}

/* ------------------------------------------------------------------------ */
/* Local field.  Eq. (1): H = -sum_<xy> s_x^T J_xy s_y with J_xy = eps I + D. */
/* The conditional density of one spin (App. A.1) is exp(s_x . h_x / T)      */
/* with h_x = -dH/ds_x:                                                      */
/*   h_x = sum_mu [ J_{x,mu} s_{x+mu} + J_{x-mu,mu}^T s_{x-mu} ].            */
/* ------------------------------------------------------------------------ */
/* The same sum from the site's own data: Jup[mu] (row-major 3x3) is the
   bond (x, x+mu), Jdn[mu] the bond (x-mu, x), s_up[mu] and s_dn[mu] the
   spins at x+mu and x-mu. */
void oracle_site_field(const double *Jup, const double *Jdn, const double *s_up,
                       const double *s_dn, double h[3]) {
  h[0] = h[1] = h[2] = 0.0;
  for (int mu = 0; mu < 3; ++mu) {
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) {
        h[a] += Jup[mu * 9 + a * 3 + b] * s_up[mu * 3 + b];
        h[a] += Jdn[mu * 9 + b * 3 + a] * s_dn[mu * 3 + b];
      }
    }
  }
}

void oracle_local_field(int L, const double *J9, const double *s, long i,
                        double h[3]) {
  double Jup[27], Jdn[27], s_up[9], s_dn[9];
  for (int mu = 0; mu < 3; ++mu) {
    long up = neighbour(L, i, mu, +1);
    long dn = neighbour(L, i, mu, -1);
    for (int e = 0; e < 9; ++e) {
      Jup[mu * 9 + e] = J9[(i * 3 + mu) * 9 + e];   /* bond (i, i+mu) */
      Jdn[mu * 9 + e] = J9[(dn * 3 + mu) * 9 + e];  /* bond (i-mu, i) */
    }
    for (int b = 0; b < 3; ++b) {
      s_up[mu * 3 + b] = s[up * 3 + b];
      s_dn[mu * 3 + b] = s[dn * 3 + b];
    }
  }
  oracle_site_field(Jup, Jdn, s_up, s_dn, h);
}

/* Natural index of the neighbour of site i in direction mu (0, 1, 2 = x, y,
   z), forward (sign = +1) or backward (sign = -1), periodic. */
long oracle_neighbour(int L, long i, int mu, int sign) { return neighbour(L, i, mu, sign); }

/* Bimodal couplings (Sec. II.A): the isotropic coupling J = +-1 and the six
   independent entries D^{ab} (a >= b) of the symmetric anisotropy = +-D.
   One byte per bond: bit 0 is the sign of J, bits 1..6 the signs of
   D^xx, D^yy, D^zz, D^xy, D^xz, D^yz (a set bit means negative).  Writes the
   bond matrix J I + D as a general 3x3, row-major. */
void oracle_bimodal_j9(long n_bonds, const unsigned char *bits, double D, double *J9) {
  for (long k = 0; k < n_bonds; ++k) {
    unsigned v = bits[k];
    double iso = (v & 1u) ? -1.0 : 1.0;
    double d[6];
    for (int e = 0; e < 6; ++e) d[e] = ((v >> (e + 1)) & 1u) ? -D : D;
    double *M = J9 + k * 9;
    M[0] = iso + d[0]; M[1] = d[3];       M[2] = d[4];
    M[3] = d[3];       M[4] = iso + d[1]; M[5] = d[5];
    M[6] = d[4];       M[7] = d[5];       M[8] = iso + d[2];
  }
}

/* Energy, Eq. (1): each nearest-neighbour bond counted once. */
double oracle_energy(int L, const double *J9, const double *s) {
  long N = (long)L * L * L;
  double E = 0.0;
  for (long i = 0; i < N; ++i) {
    for (int mu = 0; mu < 3; ++mu) {
      long up = neighbour(L, i, mu, +1);
      const double *J = J9 + (i * 3 + mu) * 9;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) E -= s[i * 3 + a] * J[a * 3 + b] * s[up * 3 + b];
    }
  }
  return E;
}

/* ------------------------------------------------------------------------ */
/* Heat-bath draw (App. A.1): a new spin from the density                    */
/* P(s) ~ exp(beta s.h) on the unit sphere.  With u = cos(angle to h),        */
/* kappa = beta|h|, u has density ~ exp(kappa u) on [-1,1]; its inverse CDF,  */
/* written for w = 1 - u so that it neither overflows nor cancels, is         */
/*   w = -log1p(r0 * expm1(-2 kappa)) / kappa   (w = 2 r0 as kappa -> 0).     */
/* The azimuth is phi = 2 pi r1 around h, in the orthonormal frame (e1,e2)    */
/* of T. Duff et al., "Building an orthonormal basis, revisited", JCGT 6(1),  */
/* 2017.  If |h| = 0 the axis is taken as e_z.                                */
/* ------------------------------------------------------------------------ */
void oracle_hb_draw(const double h[3], double beta, uint32_t w0, uint32_t w1,
                    double s_new[3]) {
  double hh = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  double hn = sqrt(hh);
  double kappa = beta * hn;
  double r0 = oracle_uniform23(w0);
  double r1 = oracle_uniform23(w1);
  double w;
  if (kappa < 1e-30)
    w = 2.0 * r0;
  else
    w = -log1p(r0 * expm1(-2.0 * kappa)) / kappa;
  if (w < 0.0) w = 0.0;
  if (w > 2.0) w = 2.0;
  double u = 1.0 - w;
  double st2 = w * (2.0 - w);
  double st = sqrt(st2 > 0.0 ? st2 : 0.0);
  double phi = 2.0 * M_PI * r1;
  double cp = cos(phi), sp = sin(phi);

  double n[3];
  if (hn > 0.0) {
    n[0] = h[0] / hn;
    n[1] = h[1] / hn;
    n[2] = h[2] / hn;
  } else {
    n[0] = 0.0;
    n[1] = 0.0;
    n[2] = 1.0;
  }
  double sgn = copysign(1.0, n[2]);
  double p = -1.0 / (sgn + n[2]);
  double q = n[0] * n[1] * p;
  double e1[3] = {1.0 + sgn * n[0] * n[0] * p, sgn * q, -sgn * n[0]};
  double e2[3] = {q, sgn + n[1] * n[1] * p, -n[1]};
  for (int a = 0; a < 3; ++a) s_new[a] = u * n[a] + st * (cp * e1[a] + sp * e2[a]);
}

/* Overrelaxation (App. A.1): s' = 2 h (h.s)/h^2 - s, the reflection of s
 * about h.  Left unchanged if h = 0. */
void oracle_or_update(const double h[3], const double s[3], double s_new[3]) {
  double hh = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  if (hh == 0.0) {
    s_new[0] = s[0];
    s_new[1] = s[1];
    s_new[2] = s[2];
    return;
  }
  double hs = h[0] * s[0] + h[1] * s[1] + h[2] * s[2];
  double f = 2.0 * hs / hh;
  for (int a = 0; a < 3; ++a) s_new[a] = f * h[a] - s[a];
}

/* ------------------------------------------------------------------------ */
/* Checkerboard sweep of one lattice (App. A.1, sweep order): first every    */
/* black site, with the fields of the current white spins, then every white   */
/* site with the new black spins.  Within one colour no site is a neighbour  */
/* of another, so the result does not depend on the site order.              */
/* kind 0 = heat-bath (needs beta, seed, lattice id, heat-bath sweep index   */
/* t), kind 1 = overrelaxation.                                              */
/* ------------------------------------------------------------------------ */
void oracle_half_sweep(int L, const double *J9, double *s, int colour, int kind,
                       double beta, uint64_t seed, uint32_t lattice, uint32_t t) {
  long N = (long)L * L * L;
  for (long i = 0; i < N; ++i) {
    if (site_colour(L, i) != colour) continue;
    double h[3], s_new[3];
    oracle_local_field(L, J9, s, i, h);
    if (kind == 0) {
      uint32_t w[2];
      oracle_hb_words(seed, (uint32_t)i, lattice, t, w);
      oracle_hb_draw(h, beta, w[0], w[1], s_new);
    } else {
      oracle_or_update(h, s + i * 3, s_new);
    }
    s[i * 3 + 0] = s_new[0];
    s[i * 3 + 1] = s_new[1];
    s[i * 3 + 2] = s_new[2];
  }
}

void oracle_sweep(int L, const double *J9, double *s, int kind, double beta,
                  uint64_t seed, uint32_t lattice, uint32_t t) {
  oracle_half_sweep(L, J9, s, 0, kind, beta, seed, lattice, t);
  oracle_half_sweep(L, J9, s, 1, kind, beta, seed, lattice, t);
}

/* Sequential overrelaxation sweep (App. A.1): the sites are visited one at  */
/* a time in the natural order i = x + L (y + L z), each reflected about the  */
/* field of its neighbours' current values -- earlier sites already updated,  */
/* later ones not -- so the update travels through the lattice as a wave.     */
void oracle_sweep_sequential(int L, const double *J9, double *s) {
  long N = (long)L * L * L;
  for (long i = 0; i < N; ++i) {
    double h[3], s_new[3];
    oracle_local_field(L, J9, s, i, h);
    oracle_or_update(h, s + i * 3, s_new);
    s[i * 3 + 0] = s_new[0];
    s[i * 3 + 1] = s_new[1];
    s[i * 3 + 2] = s_new[2];
  }
}

/* ------------------------------------------------------------------------ */
/* Parallel tempering (App. A.1): for temperature pairs (i, i+1), taken in    */
/* order i = 0 .. n_temps-2, propose exchanging the configurations at beta_i */
/* and beta_{i+1}; Metropolis accepts with probability                       */
/* min(1, exp[(beta_i - beta_{i+1}) (E_i - E_{i+1})]).  The exchange is done */
/* on the temperature labels: perm[k] is the lattice slot at temperature k.  */
/* One uniform is drawn per pair whether or not it is needed: counter        */
/* (i, replica_set, t_pt, PT).                                               */
/* ------------------------------------------------------------------------ */
void oracle_pt_sweep(int n_temps, const double *beta, const double *E, int *perm,
                     uint64_t seed, uint32_t replica_set, uint32_t t_pt,
                     long long *accepted) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int i = 0; i + 1 < n_temps; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, replica_set, t_pt, ORACLE_TAG_PT};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    double r = oracle_uniform52(out[0], out[1]);
    int a = perm[i], b = perm[i + 1];
    double delta = (beta[i] - beta[i + 1]) * (E[a] - E[b]);
    if (delta >= 0.0 || r < exp(delta)) {
      perm[i] = b;
      perm[i + 1] = a;
      if (accepted) accepted[i] += 1;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. II.B).  For two replicas a, b at the same temperature:   */
/*   q_x = s^a_x . s^b_x,  q(k) = sum_x q_x exp(i k.x) / N,                   */
/*   zeta_{x,mu} = s_{x+mu} . (s_x x s_{x-mu}),  kappa_{x,mu} = zeta^a zeta^b, */
/*   q_CG^mu(k) = sum_x kappa_{x,mu} exp(i k.x) / N,                          */
/* at k = 0 and k = (2 pi / L) e_nu, nu = 0,1,2 (k_min and its permutations),  */
/* as a direct discrete Fourier sum.                                          */
/* Q0 = q(0); Qk[2nu], Qk[2nu+1] = Re, Im q(k_nu);                            */
/* C0[mu] = q_CG^mu(0); Ck[(mu*3+nu)*2 + 0/1] = Re, Im q_CG^mu(k_nu).         */
/* ------------------------------------------------------------------------ */
static double chirality(int L, const double *s, long i, int mu) {
  long up = neighbour(L, i, mu, +1);
  long dn = neighbour(L, i, mu, -1);
  const double *a = s + i * 3, *b = s + dn * 3, *c = s + up * 3;
  double cx = a[1] * b[2] - a[2] * b[1];
  double cy = a[2] * b[0] - a[0] * b[2];
  double cz = a[0] * b[1] - a[1] * b[0];
  return c[0] * cx + c[1] * cy + c[2] * cz;
}

void oracle_overlap_fourier(int L, const double *sa, const double *sb, double *Q0,
                            double Qk[6], double C0[3], double Ck[18]) {
  long N = (long)L * L * L;
  double q0 = 0.0, qk[6] = {0}, c0[3] = {0}, ck[18] = {0};
  for (long i = 0; i < N; ++i) {
    int xc[3] = {(int)(i % L), (int)((i / L) % L), (int)(i / ((long)L * L))};
    double q = sa[i * 3] * sb[i * 3] + sa[i * 3 + 1] * sb[i * 3 + 1] +
               sa[i * 3 + 2] * sb[i * 3 + 2];
    double kap[3];
    for (int mu = 0; mu < 3; ++mu) kap[mu] = chirality(L, sa, i, mu) * chirality(L, sb, i, mu);
    q0 += q;
    for (int mu = 0; mu < 3; ++mu) c0[mu] += kap[mu];
    for (int nu = 0; nu < 3; ++nu) {
      double ph = 2.0 * M_PI * (double)xc[nu] / (double)L;
      double cr = cos(ph), ci = sin(ph);
      qk[2 * nu] += q * cr;
      qk[2 * nu + 1] += q * ci;
      for (int mu = 0; mu < 3; ++mu) {
        ck[(mu * 3 + nu) * 2] += kap[mu] * cr;
        ck[(mu * 3 + nu) * 2 + 1] += kap[mu] * ci;
      }
    }
  }
  *Q0 = q0 / (double)N;
  for (int j = 0; j < 6; ++j) Qk[j] = qk[j] / (double)N;
  for (int j = 0; j < 3; ++j) C0[j] = c0[j] / (double)N;
  for (int j = 0; j < 18; ++j) Ck[j] = ck[j] / (double)N;
}

/* Per-pair measurement in the order used for accumulation:
 * out[0] = |q(0)|^2, out[1] = |q(0)|^4, out[2] = mean_nu |q(k_nu)|^2,
 * out[3] = mean_mu |q_CG^mu(0)|^2, out[4] = mean_mu |q_CG^mu(0)|^4,
 * out[5] = mean_{mu,nu} |q_CG^mu(k_nu)|^2  (the CG average over mu follows
 * Sec. II.B). */
void oracle_measure_pair(int L, const double *sa, const double *sb, double out[6]) {
  double Q0, Qk[6], C0[3], Ck[18];
  oracle_overlap_fourier(L, sa, sb, &Q0, Qk, C0, Ck);
  double q2 = Q0 * Q0;
  double q2k = 0.0;
  for (int nu = 0; nu < 3; ++nu) q2k += Qk[2 * nu] * Qk[2 * nu] + Qk[2 * nu + 1] * Qk[2 * nu + 1];
  double c2 = 0.0, c4 = 0.0, c2k = 0.0;
  for (int mu = 0; mu < 3; ++mu) {
    double m2 = C0[mu] * C0[mu];
    c2 += m2;
    c4 += m2 * m2;
    for (int nu = 0; nu < 3; ++nu) {
      double re = Ck[(mu * 3 + nu) * 2], im = Ck[(mu * 3 + nu) * 2 + 1];
      c2k += re * re + im * im;
    }
  }
  out[0] = q2;
  out[1] = q2 * q2;
  out[2] = q2k / 3.0;
  out[3] = c2 / 3.0;
  out[4] = c4 / 3.0;
  out[5] = c2k / 9.0;
}

/* Lattice average of the Schwinger-Dyson combination (App. A.4.3):
 * (1/N) sum_x [ 2T s_x.h_x - (h_x.h_x - (s_x.h_x)^2) ], zero in equilibrium. */
double oracle_sd_residual(int L, const double *J9, const double *s, double T) {
  long N = (long)L * L * L;
  double acc = 0.0;
  for (long i = 0; i < N; ++i) {
    double h[3];
    oracle_local_field(L, J9, s, i, h);
    double sh = s[i * 3] * h[0] + s[i * 3 + 1] * h[1] + s[i * 3 + 2] * h[2];
    double hh = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    acc += 2.0 * T * sh - (hh - sh * sh);
  }
  return acc / (double)N;
}

/* ------------------------------------------------------------------------ */
/* One sample's Monte Carlo run (Sec. III and App. A.1).  One step (MCS) is, */
/* in order: one heat-bath sweep of every lattice, n_or overrelaxation       */
/* sweeps of every lattice, the energies, one parallel-tempering sweep per   */
/* replica set (when n_temps > 1), and, every measure_every steps, the       */
/* observables.  The paper uses L overrelaxation sweeps per step; n_or is a  */
/* parameter here.                                                           */
/*                                                                           */
/* Lattices of the sample: slot = r*n_temps + j, r < n_replicas.             */
/* spins[slot*N*3 ...]; perm[r*n_temps + k] = slot at temperature k.         */
/* The heat-bath lattice id is lattice_base + slot, the parallel-tempering   */
/* replica-set id is replset_base + r.  hb_t and pt_t are the global sweep   */
/* counters; they advance by one per step.                                   */
/* obs[k*9 + j] accumulates, per measurement:                                */
/*   j = 0,1   sum over the n_replicas lattices at temperature k of e, e^2   */
/*             (e = E/N);                                                    */
/*   j = 2..7  sum over replica pairs (0,1),(2,3),... of the six per-pair     */
/*             values of oracle_measure_pair;                                */
/*   j = 8     sum over the lattices at k of the Schwinger-Dyson residual.    */
/* counts[k] counts measurements; accepted[r*(n_temps-1)+i] PT acceptances.  */
/* energies[slot] receives the last computed energies.                       */
/* ------------------------------------------------------------------------ */
int oracle_run(int L, const double *J9, int n_replicas, int n_temps,
               const double *beta, double *spins, int *perm, uint64_t seed,
               uint32_t lattice_base, uint32_t replset_base, uint32_t *hb_t,
               uint32_t *pt_t, long long *step_counter, int n_steps, int n_or,
               int measure_every, double *obs, long long *counts,
               long long *accepted, double *energies, int n_threads) {
  long N = (long)L * L * L;
  int R = n_replicas * n_temps;
  int *temp_of = (int *)malloc(sizeof(int) * (size_t)R);
  if (!temp_of) return -1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  for (int step = 0; step < n_steps; ++step) {
    for (int r = 0; r < n_replicas; ++r)
      for (int k = 0; k < n_temps; ++k) temp_of[perm[r * n_temps + k]] = k;
    uint32_t t = *hb_t;
#pragma omp parallel for schedule(dynamic, 1)
    for (int slot = 0; slot < R; ++slot) {
      double *s = spins + (long)slot * N * 3;
      double b = beta[temp_of[slot]];
      oracle_sweep(L, J9, s, 0, b, seed, lattice_base + (uint32_t)slot, t);
      for (int o = 0; o < n_or; ++o) oracle_sweep(L, J9, s, 1, b, seed, 0, 0);
      energies[slot] = oracle_energy(L, J9, s);
    }
    *hb_t += 1;
    if (n_temps > 1) {
      for (int r = 0; r < n_replicas; ++r)
        oracle_pt_sweep(n_temps, beta, energies, perm + r * n_temps, seed,
                        replset_base + (uint32_t)r, *pt_t,
                        accepted ? accepted + (long)r * (n_temps - 1) : NULL);
    }
    *pt_t += 1;
    *step_counter += 1;
    if (measure_every > 0 && (*step_counter % measure_every) == 0) {
#pragma omp parallel for schedule(dynamic, 1)
      for (int k = 0; k < n_temps; ++k) {
        double T = beta[k] > 0.0 ? 1.0 / beta[k] : INFINITY;
        double *o = obs + k * 9;
        for (int r = 0; r < n_replicas; ++r) {
          int slot = perm[r * n_temps + k];
          double e = energies[slot] / (double)N;
          o[0] += e;
          o[1] += e * e;
          if (beta[k] > 0.0)
            o[8] += oracle_sd_residual(L, J9, spins + (long)slot * N * 3, T);
        }
        for (int p = 0; p + 1 < n_replicas; p += 2) {
          int sa = perm[p * n_temps + k], sb = perm[(p + 1) * n_temps + k];
          double m[6];
          oracle_measure_pair(L, spins + (long)sa * N * 3, spins + (long)sb * N * 3, m);
          for (int j = 0; j < 6; ++j) o[2 + j] += m[j];
        }
        counts[k] += 1;
      }
    }
  }
  free(temp_of);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Batch helpers for the statistical pins (loops around the functions above) */
/* ------------------------------------------------------------------------ */

/* n heat-bath draws for one fixed field h: draw j uses the heat-bath words of
 * (site j, lattice, t).  out[j*3 + a]. */
void oracle_hb_draw_batch(const double h[3], double beta, uint64_t seed,
                          uint32_t lattice, uint32_t t, long n, double *out) {
  for (long j = 0; j < n; ++j) {
    uint32_t w[2];
    oracle_hb_words(seed, (uint32_t)j, lattice, t, w);
    oracle_hb_draw(h, beta, w[0], w[1], out + j * 3);
  }
}

/* Two spins coupled by one bond, energy -s1^T J s2, updated alternately by
 * heat-bath (s1 with field J s2, then s2 with field J^T s1).  Iteration j
 * draws s1 with words of (site 0, lattice, j) and s2 with (site 1, lattice, j).
 * Returns in sums[0], sums[1] the sums of x = s1^T J s2 and x^2 over the
 * iterations after n_skip. */
void oracle_two_site_chain(const double J[9], double beta, uint64_t seed,
                           uint32_t lattice, long n_skip, long n_iter,
                           double s1[3], double s2[3], double sums[2]) {
  sums[0] = sums[1] = 0.0;
  for (long j = 0; j < n_skip + n_iter; ++j) {
    uint32_t w[2];
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = J[a * 3] * s2[0] + J[a * 3 + 1] * s2[1] + J[a * 3 + 2] * s2[2];
    oracle_hb_words(seed, 0u, lattice, (uint32_t)j, w);
    oracle_hb_draw(h, beta, w[0], w[1], s1);
    for (int a = 0; a < 3; ++a) h[a] = J[a] * s1[0] + J[3 + a] * s1[1] + J[6 + a] * s1[2];
    oracle_hb_words(seed, 1u, lattice, (uint32_t)j, w);
    oracle_hb_draw(h, beta, w[0], w[1], s2);
    if (j >= n_skip) {
      double x = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) x += s1[a] * J[a * 3 + b] * s2[b];
      sums[0] += x;
      sums[1] += x * x;
    }
  }
}

/* Local fields of every site of one colour: h_out[i*3 + a] for sites of that
 * colour (other entries untouched). */
void oracle_fields(int L, const double *J9, const double *s, int colour, double *h_out) {
  long N = (long)L * L * L;
  for (long i = 0; i < N; ++i)
    if (site_colour(L, i) == colour) oracle_local_field(L, J9, s, i, h_out + i * 3);
}
