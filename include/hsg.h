/*
 * hsg.h -- C ABI of libhsg: equilibrium Monte Carlo of the 3d Edwards-Anderson
 * Heisenberg spin glass with random anisotropic couplings on one NVIDIA B300
 * (Baity-Jesi, Fernandez, Martin-Mayor, Sanz, arXiv:1309.1599).
 *
 * Model (Sec. II.A, Eq. (1)): unit 3-vector spins s_x on a periodic L^3 cubic
 * lattice, H = -sum_<x,y> s_x^T J_xy s_y, J_xy = eps_xy I + D_xy with D
 * symmetric, so every bond carries a symmetric 3x3 matrix of six entries.
 * A "sample" is one realisation of the couplings; it is simulated as
 * R = n_replicas * n_temps lattices ("slots") sharing those couplings.
 * Slot j of a sample is replica j / n_temps; at creation it sits at
 * temperature index j % n_temps.  Parallel tempering exchanges temperature
 * labels, never spins (App. A.1).
 *
 * Conventions for every call:
 *   - site index i = x + L*(y + L*z), 0 <= x,y,z < L; black sites have x+y+z
 *     even, white sites odd; a sweep updates all black sites, then all white.
 *   - Host arrays are owned by the caller and are read or written before the
 *     call returns.  All device memory is owned by the library.
 *   - Compute calls (sweeps, energies, PT, measurement, run_steps) are
 *     asynchronous: they are enqueued on the configured CUDA stream and return
 *     at once.  Calls that move data to or from the host synchronise that
 *     stream first.
 *   - Every call returns an hsg_status.  HSG_EINVAL leaves the state
 *     unchanged.  A CUDA failure returns HSG_ECUDA; a device-side wait that
 *     gave up returns HSG_ETIMEOUT.  hsg_last_error() describes the last
 *     failure of the calling thread.  Nothing aborts the process or traps the
 *     GPU.
 *   - Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed mod 2^32, seed >> 32); they replace the generator of App. A.4.
 *       heat-bath draw at site i of lattice l (l = sample*R + slot) in
 *       heat-bath sweep t: counter (i, l/2, t, 1); even l uses output words
 *       0,1, odd l words 2,3; uniform r = ((w >> 9) + 1/2) * 2^-23.
 *       parallel-tempering pair k of replica set g (g = sample*n_replicas + r)
 *       in PT sweep t: counter (k, g, t, 2); r = (((w0>>6)<<26 | w1>>6) + 1/2)
 *       * 2^-52.
 *     The library keeps the sweep counters t on the device; they start at 0.
 */
#ifndef HSG_H
#define HSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsg_ctx *hsg_t;

typedef enum {
  HSG_OK = 0,
  HSG_EINVAL = 1,   /* bad argument or configuration; nothing changed */
  HSG_ENOMEM = 2,   /* device or host allocation failed */
  HSG_ECUDA = 3,    /* a CUDA runtime call or kernel failed */
  HSG_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  HSG_ESTATE = 5,   /* call not valid in the current state */
  HSG_EIO = 6       /* checkpoint file could not be read or written */
} hsg_status;

/* Storage precision of the couplings on the device: FP32 or FP16, rounded
 * once (to nearest even) from the float32 host array, or bimodal (Sec. II.A:
 * J = +-1 and D^ab = +-D, one byte per bond holding the seven signs). */
enum { HSG_F32 = 0, HSG_F16 = 1, HSG_BIMODAL = 2 };

/* Device spin layout.
 *   HSG_LAYOUT_PLAIN    one lattice per thread; each lattice reads its own
 *                       couplings (the plain single-lattice form).
 *   HSG_LAYOUT_BATCHED  two lattices of the same sample interleaved per
 *                       element, updated by one thread against one coupling
 *                       read (requires R even). */
enum { HSG_LAYOUT_PLAIN = 0, HSG_LAYOUT_BATCHED = 1 };

/* Sweep kernel.
 *   HSG_SWEEP_AUTO      one fused pass per sweep (both colours, each spin read
 *                       and written once, planes staged in shared memory),
 *                       wherever the lattice size allows it (whole planes, or
 *                       bands of at least 8 rows that divide L); the two-pass
 *                       kernel otherwise, or where hsg_autotune finds it
 *                       faster.  Doubles the spin memory.
 *   HSG_SWEEP_TWO_PASS  always one kernel per colour half-sweep.
 * Both give the same spins bit for bit. */
enum { HSG_SWEEP_AUTO = 0, HSG_SWEEP_TWO_PASS = 1 };

/* Observables accumulated per (sample, temperature index) by hsg_measure
 * (Sec. II.B).  Per measurement, with e = E/N:
 *   [0] sum of e, [1] sum of e^2      over the n_replicas lattices at that T
 *   [2] |q(0)|^2, [3] |q(0)|^4, [4] mean_nu |q(k_nu)|^2,
 *   [5] mean_mu |qCG^mu(0)|^2, [6] mean_mu |qCG^mu(0)|^4,
 *   [7] mean_{mu,nu} |qCG^mu(k_nu)|^2  summed over replica pairs (0,1),(2,3),...
 *   [8] sum of the Schwinger-Dyson residual (1/N) sum_x [2T s.h - h^2 + (s.h)^2]
 *       over the lattices at that T (App. A.4.3; 0 where beta = 0)
 * where q(k) = sum_x s^a_x.s^b_x e^{ik.x}/N, k_nu = (2 pi/L) e_nu, and
 * qCG^mu(k) is the same sum of zeta^a_{x,mu} zeta^b_{x,mu}, zeta_{x,mu} =
 * s_{x+mu}.(s_x x s_{x-mu}).  counts[] holds the number of measurements. */
enum { HSG_NOBS = 9 };

typedef struct {
  int n_samples;          /* S >= 1 */
  const int *L;           /* [S] linear sizes, each even, 4 <= L <= 512 */
  int n_replicas;         /* >= 1 */
  int n_temps;            /* N_T >= 1 */
  const double *beta;     /* [N_T] inverse temperatures, >= 0, increasing */
  int coupling_prec;      /* HSG_F32, HSG_F16 or HSG_BIMODAL */
  int layout;             /* HSG_LAYOUT_PLAIN or HSG_LAYOUT_BATCHED */
  int n_or;               /* overrelaxation sweeps per step, >= 0 */
  int measure_every;      /* hsg_run_steps measures every this many steps (0: never) */
  uint64_t seed;          /* Philox key */
  void *stream;           /* cudaStream_t to use; NULL = the legacy default stream */
  long long timeout_cycles; /* bound (SM clock cycles) for each device-side wait,
                              0 = library default (4e9) */
  int sweep_kernel;       /* HSG_SWEEP_AUTO or HSG_SWEEP_TWO_PASS */
  int band_rows;          /* fused sweep: rows per CTA band, 0 = library choice;
                             otherwise L or a divisor of L >= 8 that fits the
                             block and shared-memory limits (HSG_EINVAL if not) */
  int persistent;         /* 1: hsg_run_steps keeps the lattices resident in
                             shared memory.  Where a replica set (the N_T
                             lattices of one replica of one sample) fits in
                             one CTA, whole steps, PT included, run in one
                             launch per lattice size and stretch of steps
                             between measurements; otherwise each CTA holds
                             part of a set for one step and the PT sweep
                             follows as its own kernel.  Needs N_T <= 64, N_T
                             a multiple of the layout's lattices per element,
                             and one lattice group, 12 V L^3 bytes (V = 1
                             plain, 2 batched), within 224 KiB for every L
                             (HSG_EINVAL otherwise).
                             2: as 1, with the samples of both lattice sizes
                             of a two-size context in one launch: CTAs of the
                             larger size hold one replica set each, CTAs of
                             the smaller size as many whole sets of one
                             sample as fit in the same shared memory.  Needs
                             every replica set held whole (HSG_EINVAL
                             otherwise); specialised for L = 12 with L = 8 in
                             the batched layout, generic (bonds read from
                             global memory) for other pairs; more than two
                             lattice sizes are refused (HSG_EINVAL).
                             0: streaming steps. */
  double bimodal_D;       /* HSG_BIMODAL: the magnitude D >= 0 of the
                             anisotropic couplings (the paper uses 0.5 and 1);
                             ignored by the other formats */
  int fused_groups;       /* fused sweep: lattice groups (of the layout's
                             lattices per element) that each thread updates
                             against one read of each coupling, for both the
                             heat-bath and the overrelaxation kernel; 0 =
                             library choice (1 until hsg_autotune picks per
                             kernel), 1, or 2 (batched layout with a multiple
                             of 4 lattices per sample; HSG_EINVAL otherwise,
                             or if L cannot be tiled with it).  The spins do
                             not depend on it. */
} hsg_config;

/* Create a context: validates cfg (copied; the caller's arrays may be freed
 * afterwards), allocates all device buffers on the current CUDA device, sets
 * every coupling to 0 and every spin to (0,0,1), the temperature labels to
 * the identity and all counters and accumulators to 0.  *out receives the
 * handle (NULL on failure). */
hsg_status hsg_lattice_create(const hsg_config *cfg, hsg_t *out);

/* Release every resource of h (NULL is ignored).  Synchronises its stream. */
void hsg_destroy(hsg_t h);

/* Couplings of one sample from host float32 [N][3][6]: entry [i][mu][e] is
 * element e = (xx,yy,zz,xy,xz,yz) of the symmetric matrix on the bond
 * (i, i+e_mu), mu = 0,1,2 = +x,+y,+z.  Rounded once to the storage precision.
 * Invalidates the stored energies. */
hsg_status hsg_set_couplings(hsg_t h, int sample, const float *J6);

/* The stored couplings of one sample as float32 [N][3][6] (exact values;
 * for HSG_BIMODAL the decoded matrices, computed in FP32 as below). */
hsg_status hsg_get_couplings(hsg_t h, int sample, float *J6_out);

/* Bimodal couplings of one sample (Sec. II.A), for contexts created with
 * HSG_BIMODAL: host uint8 [N][3], natural site order, one byte per bond
 * (i, i+e_mu).  Bit 0 is the sign of the isotropic coupling J = +-1, bits 1-6
 * the signs of D^xx, D^yy, D^zz, D^xy, D^xz, D^yz = +-D (a set bit means
 * negative), bit 7 must be 0.  The kernels use the entries
 * (J + D^xx, J + D^yy, J + D^zz, D^xy, D^xz, D^yz), each sum rounded to FP32.
 * HSG_EINVAL if the context is not bimodal or a bit 7 is set (nothing
 * stored).  hsg_set_couplings returns HSG_EINVAL on a bimodal context: the
 * signs cannot be recovered from the matrices when D = 1. */
hsg_status hsg_set_couplings_bimodal(hsg_t h, int sample, const uint8_t *bits);
hsg_status hsg_get_couplings_bimodal(hsg_t h, int sample, uint8_t *bits_out);

/* Spins of one lattice slot from / to host float32 [N][3].  Spins are stored
 * as given (no normalisation). */
hsg_status hsg_set_spins(hsg_t h, int sample, int slot, const float *s);
hsg_status hsg_get_spins(hsg_t h, int sample, int slot, float *s_out);

/* Every lattice slot of one sample at once, host float32 [R][N][3] (slots
 * 0 .. R-1, each [N][3] in natural site order), staged in chunks of at most
 * 256 MiB instead of R calls.  Synchronous like the one-slot calls; the
 * pointer may be pinned or pageable.  HSG_EINVAL on a NULL argument or a bad
 * sample (nothing stored); HSG_ENOMEM if the staging buffer cannot be
 * allocated. */
hsg_status hsg_set_spins_sample(hsg_t h, int sample, const float *s);
hsg_status hsg_get_spins_sample(hsg_t h, int sample, float *s_out);

/* The same with a caller-owned DEVICE buffer float32 [N][3] (natural site
 * order) on the context's device, e.g. a torch CUDA tensor: enqueued on the
 * configured stream without synchronising, so the buffer must stay valid
 * (and, for the getter, unread) until the stream reaches the copy.  No host
 * copy is involved. */
hsg_status hsg_set_spins_device(hsg_t h, int sample, int slot, const float *d_s);
hsg_status hsg_get_spins_device(hsg_t h, int sample, int slot, float *d_out);

/* n checkerboard sweeps of every lattice (App. A.1): heat-bath draws from
 * P(s) ~ exp(beta s.h) at each lattice's current temperature; overrelaxation
 * reflects s about h, s' = 2h(h.s)/h^2 - s (unchanged where h = 0).  Each
 * heat-bath sweep advances the heat-bath counter by one.  The last
 * overrelaxation sweep also leaves the energies current. */
hsg_status hsg_sweep_hb(hsg_t h, int n);
hsg_status hsg_sweep_or(hsg_t h, int n);

/* n sequential overrelaxation sweeps of every lattice (App. A.1): the sites
 * are visited one at a time in the natural order i = x + L (y + L z), each
 * reflected about the field of its neighbours' current values (earlier sites
 * already updated), so the update travels through the lattice as a wave.
 * Executed exactly by hyperplanes x + y + z = tau, one lattice group per CTA
 * held in shared memory: needs 12 V L^3 <= 200 KiB for every L (L <= 20 with
 * two lattices per element, L <= 24 with one), HSG_EINVAL otherwise (nothing
 * done).  The stored energies become stale (recomputed on demand).  Not used
 * by hsg_run_steps, whose sweeps are checkerboard. */
hsg_status hsg_sweep_or_sequential(hsg_t h, int n);

/* Recompute the energy E = -sum_bonds s_x^T J s_y (Eq. (1)) of every lattice
 * (FP32 terms, FP64 sums). */
hsg_status hsg_energy(hsg_t h);

/* Energies of all lattices, double [S][R] by slot (computed first if stale). */
hsg_status hsg_get_energies(hsg_t h, double *E_out);

/* Overwrite the stored energies (double [S][R]); used to drive hsg_pt_swap
 * with chosen values.  They stay current until the next sweep. */
hsg_status hsg_set_energies(hsg_t h, const double *E);

/* One parallel-tempering sweep of every replica set (App. A.1): pairs of
 * neighbouring temperature indices k = 0 .. N_T-2 in order; the exchange of
 * labels k, k+1 is accepted iff D >= 0 or r < exp(D), D = (beta_k -
 * beta_{k+1})(E[perm k] - E[perm k+1]) in FP64.  Advances the PT counter. */
hsg_status hsg_pt_swap(hsg_t h);

/* Temperature labels, int [S][n_replicas][N_T]: the slot at each temperature. */
hsg_status hsg_get_perm(hsg_t h, int *perm_out);
hsg_status hsg_set_perm(hsg_t h, const int *perm);

/* Accepted PT exchanges, long long [S][n_replicas][max(N_T-1,1)]. */
hsg_status hsg_get_pt_accepts(hsg_t h, long long *acc_out);

/* Accumulate one measurement of the observables listed at HSG_NOBS. */
hsg_status hsg_measure(hsg_t h);

/* n_steps Monte Carlo steps (Sec. III): one heat-bath sweep, n_or
 * overrelaxation sweeps, the energies, one PT sweep when N_T > 1, and a
 * measurement after every measure_every-th step (counted over the life of
 * the context).  Streaming contexts replay captured CUDA graphs; persistent
 * ones launch the shared-memory-resident steps (see hsg_config). */
hsg_status hsg_run_steps(hsg_t h, int n_steps);

/* Accumulated observables, double [S][N_T][HSG_NOBS], and the number of
 * measurements, long long [S][N_T] (counts may be NULL). */
hsg_status hsg_read_observables(hsg_t h, double *obs_out, long long *counts_out);
hsg_status hsg_reset_observables(hsg_t h);

/* Counters: out[0] heat-bath sweeps, out[1] PT sweeps, out[2] steps.
 * hsg_set_counters sets all three (for resuming a run elsewhere). */
hsg_status hsg_get_counters(hsg_t h, uint64_t out[3]);
hsg_status hsg_set_counters(hsg_t h, const uint64_t in[3]);

/* How the sweeps of `sample` run: out[0] = 1 for the fused one-pass kernel,
 * 0 for two half-sweep kernels; out[1] = rows per band of the fused kernel
 * (L for whole planes); out[2] = kernel launches per sweep; out[3], out[4] =
 * lattice groups per thread of the fused overrelaxation and heat-bath
 * kernels (0 for the half-sweeps). */
hsg_status hsg_get_sweep_plan(hsg_t h, int sample, int out[5]);

/* Resident steps (persistent contexts) of `sample`'s lattice size: out[0] =
 * bond residency (0 global, 1 shared as stored, 2 shared as FP32), out[1] =
 * lattice groups per work item, out[2] = threads per CTA, out[3] = lattice
 * groups per CTA (N_T / V per whole replica set), out[4] = whole replica sets
 * per CTA, out[5] = 1 when all lattice sizes run in one launch; zeros
 * otherwise. */
hsg_status hsg_get_resident_plan(hsg_t h, int sample, int out[6]);

/* Autotuner (Sec. III's sweeps; the tiling is free, the results do not
 * depend on it).  For each lattice size of the context it times the
 * candidate launch shapes on the context's own couplings and spins and keeps
 * the fastest: the band height and lattice groups per thread of the fused
 * overrelaxation sweep, or the two-pass half-sweeps instead (timed as
 * overrelaxation sweeps whose output is discarded, or that run on a copy of
 * the state), then the groups per thread of the fused heat-bath sweep at
 * that band height, and, for persistent contexts, the groups per work item
 * and threads per CTA of the resident steps (timed on scratch copies of the
 * spins, labels, energies and acceptances).  The state is not changed.  A choice is remembered for the process per (L, lattices per
 * element, precision, lattices of that L, N_T, bond residency), so later
 * contexts of the same
 * shape take it without timing.  Synchronous; a new shape must beat the
 * current one by 2% to replace it.  HSG_EINVAL on NULL, HSG_ENOMEM if the
 * scratch copies cannot be allocated, HSG_ECUDA / HSG_ETIMEOUT from the timed
 * launches. */
hsg_status hsg_autotune(hsg_t h);

/* Number of compute kernels this context has enqueued so far (sweeps,
 * energies, PT, measurement and counter updates, including those replayed
 * from graphs; data-transfer helpers are not counted). */
hsg_status hsg_get_launch_count(hsg_t h, uint64_t *out);

/* Checkpoint: spins, couplings, temperature labels, energies, counters and
 * accumulators to a binary file, and back into a context created with the
 * same configuration.  Philox is counter based, so a resumed run is
 * bit-identical to an uninterrupted one. */
hsg_status hsg_save(hsg_t h, const char *path);
hsg_status hsg_load(hsg_t h, const char *path);

/* Wait for all work enqueued by h.  HSG_ETIMEOUT if a kernel's bounded
 * device-side wait gave up since the last check. */
hsg_status hsg_synchronize(hsg_t h);

/* Exercises the failure path of the bounded device-side waits: launches one
 * fused sweep that first waits, with the given bound, on a barrier nothing
 * completes; the kernel records the expiry, waits for its own copies in
 * flight and returns without writing spins.  Returns HSG_ETIMEOUT when the
 * mechanism works (the context stays usable and unchanged); HSG_ESTATE if no
 * sample uses the fused sweep. */
hsg_status hsg_selftest_wait_timeout(hsg_t h, long long timeout_cycles);

/* Philox4x32-10 evaluated on the device: in = host uint32 [n][6] rows
 * (c0,c1,c2,c3,k0,k1), out = host uint32 [n][4].  For checking the device
 * generator against other implementations. */
hsg_status hsg_philox4x32_10(const uint32_t *in, long n, uint32_t *out);

/* Energies without any allocation by the library.  The paper has no
 * counterpart to this call; it exists for callers that cannot let a library
 * call cudaMalloc or cudaFree -- hosts that give out device memory only from
 * an arena they plan themselves, or latency-critical loops that must never
 * wait in the CUDA driver's allocator.
 *   spins  device float [n_samples*lattices_per_sample][3][N]: component
 *          planes of each lattice, site i = x + L*(y + L*z), lattices of a
 *          sample consecutive;
 *   J6     device float [n_samples][3][N][6]: bond (i, i+e_mu) of each sample
 *          at [mu][i], entries (xx,yy,zz,xy,xz,yz);
 *   E_out  device double [n_samples*lattices_per_sample], receives
 *          E = -sum_bonds s_x^T J s_y (FP32 terms, FP64 sums);
 *   stream cudaStream_t to run on (NULL = legacy default stream).
 * All three buffers belong to the caller.  Before anything is launched each
 * is checked to be device (or managed) memory usable by the current device,
 * inside one allocation large enough for the sizes given, and aligned (spins
 * 4 bytes, J6 and E_out 8 bytes); HSG_EINVAL otherwise.  The work is enqueued
 * asynchronously.  The only working memory is a fixed device array of
 * HSG_NOALLOC_SCRATCH_DOUBLES doubles (2 MiB) inside the library, which every
 * GPU that loads the library holds until the process exits; a request needing
 * more than that (lattices x ceil(L^3/512) partial sums) is rejected with
 * HSG_EINVAL before anything runs.  The first call in each CUDA context (per
 * device, and again after the context is destroyed and re-created) looks up
 * the array's device address with that context current; make that first call
 * before any stream capture (a first call on a capturing stream returns
 * HSG_ESTATE and enqueues nothing).  All calls on a device share the array and
 * it keeps the last call's contents (each call writes every entry it reads,
 * so nothing needs clearing), so calls that overlap on the GPU race and give
 * wrong results: order them on one stream. */
#define HSG_NOALLOC_SCRATCH_DOUBLES 262144
hsg_status hsg_energy_noalloc(const float *spins, const float *J6, int L, int n_samples,
                              int lattices_per_sample, double *E_out, void *stream);

/* Message of the last failure in the calling thread ("" if none). */
const char *hsg_last_error(void);

/* ABI version of this header. */
int hsg_version(void);
#define HSG_VERSION 3  /* bumped with every change of hsg_config or of a signature */

#ifdef __cplusplus
}
#endif
#endif /* HSG_H */
