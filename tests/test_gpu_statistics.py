"""Long-run parity of the CUDA path with the FP64 oracle (statistical), and
parity at the full size of the throughput workload (sampled lattices).

Trajectories under identical random streams separate after a few sweeps
(overrelaxation is chaotic), and at low temperature a single chain's time
average depends on the valley it settles in, so one chain's binning error
does not describe the spread between runs.  The long-run averages are
therefore compared between ensembles of independent chains of the same
Markov chain -- same couplings, independent initial spins and random streams
-- with the pooled-variance two-sample t statistic; under the hypothesis
that GPU and oracle sample the same process it is ~N(0,1) at any time,
equilibrated or not.  Threshold: |t| < 3 per observable (the 3-sigma
agreement the parity target asks of long-run averages), with a 4-sigma bound
where many temperatures are compared at once, plus a bound on the mean of
t^2.
"""
import json
import os

import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import SWEEP_TOL, frame_ambiguous_diff

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _block_means(obs, counts, n_rep):
    n = counts[..., None].astype(float)
    m = np.empty_like(obs)
    m[..., 0:2] = obs[..., 0:2] / (n * n_rep)
    m[..., 2:8] = obs[..., 2:8] / (n * (n_rep // 2))
    m[..., 8] = obs[..., 8] / (n[..., 0] * n_rep)
    return m


def _t_stat(a, b):
    """Pooled two-sample t statistic along axis 0 of chain averages a, b."""
    a, b = np.asarray(a), np.asarray(b)
    na, nb = len(a), len(b)
    va, vb = a.var(0, ddof=1), b.var(0, ddof=1)
    sp2 = ((na - 1) * va + (nb - 1) * vb) / (na + nb - 2)
    return (a.mean(0) - b.mean(0)) / np.sqrt(sp2 * (1.0 / na + 1.0 / nb) + 1e-300)


def _gpu_chains(L, beta, n_rep, n_chains, steps, measure_every, layout, seed=1, precision="f32"):
    """n_chains independent chains on the couplings of generator sample 0
    (stored as FP32, or rounded once to FP16 with precision="f16"): chain c =
    context sample c (its own initial spins and random streams)."""
    prec = hsg.F16 if precision == "f16" else hsg.F32
    lat = hsg.Lattice([L] * n_chains, beta, n_replicas=n_rep, coupling_prec=prec,
                      layout=layout, n_or=8, measure_every=measure_every, seed=seed)
    J6 = gi.couplings(L, seed, 0, precision=precision)
    for c in range(n_chains):
        lat.set_couplings(c, J6)
        for j in range(lat.R):
            lat.set_spins(c, j, gi.random_spins(L, seed, c, j))
    return lat, J6


def test_long_run_L8_single_temperature_matches_oracle():
    """Plain FP32 form, L=8, T=0.5, 2 replicas, 1 HB + 8 OR per step,
    observables every step, 1000 steps: averages over steps 201-1000 of 32
    GPU chains against 8 oracle chains."""
    L, beta, seed, steps, skip = 8, 2.0, 1, 1000, 200
    lat, J6 = _gpu_chains(L, [beta], 2, 32, steps, 1, hsg.PLAIN, seed)
    lat.run_steps(skip)
    lat.reset_observables()
    lat.run_steps(steps - skip)
    o, c = lat.read_observables()
    gpu = _block_means(o[:, 0], c[:, 0], 2)                  # [chain, obs]
    cpu = []
    for ch in range(8):
        smp = oracle.Sample(L, J6, gi.random_spins_batch(L, seed, ch, 2), [beta], 2, seed,
                            sample_index=ch)
        smp.run(skip, 8, 0)
        smp.run(steps - skip, 8, 1)
        cpu.append(_block_means(smp.obs[0], smp.counts[0], 2))
    t = _t_stat(gpu, cpu)
    for j, name in [(0, "e"), (2, "q2"), (5, "c2")]:
        assert abs(t[j]) < 3, (name, np.mean(np.asarray(gpu)[:, j]), np.mean(np.asarray(cpu)[:, j]), t[j])
    # a real comparison: the chains differ and the observable is resolved
    assert np.asarray(gpu)[:, 0].std() > 0


@pytest.mark.parametrize("golden", ["pt_L16_oracle.json", "pt_L16_f16_oracle.json"])
def test_parallel_tempering_L16_matches_stored_oracle(golden):
    """L=16, the couplings of sample 0, 16 temperatures evenly spaced in
    [0.15, 0.75] x 2 replicas, 20000 steps of HB + 8 OR + PT, observables
    every 10 steps.  Averages over the second half of 16 GPU chains against
    the 8 oracle chains stored by tests/golden/make_pt_L16_oracle.py, for
    e, q2, q2(k_min) and q2_CG at every temperature (64 statistics): all
    |t| < 4 and mean t^2 < 2; the energies |t| < 3.  Once with the couplings
    stored as FP32 and once with the same draws rounded to FP16 (the
    precision form: the oracle runs in FP64 on the identical FP16 values)."""
    with open(os.path.join(HERE, "golden", golden)) as f:
        ref = json.load(f)
    L, NT, n_rep, seed = ref["L"], ref["n_temps"], ref["n_replicas"], ref["seed"]
    beta = gi.linear_betas(*ref["T_range"], NT)
    steps, block = ref["steps"], ref["block_steps"]
    lat, _ = _gpu_chains(L, beta, n_rep, 16, steps, ref["measure_every"], hsg.BATCHED, seed,
                         precision=ref.get("couplings", "f32"))
    lat.run_steps(steps // 2)
    lat.reset_observables()
    lat.run_steps(steps // 2)
    o, c = lat.read_observables()
    gpu = _block_means(o, c, n_rep)                           # [chain, T, obs]
    ch = np.asarray(ref["chains"])                            # [chain, block, T, obs]
    cpu = ch[:, ch.shape[1] // 2:].mean(axis=1)               # equal-size blocks
    t = _t_stat(gpu, cpu)                                     # [T, obs]
    # the per-observable agreement, printed for the record (pytest -s)
    # (relative differences of the means at the lowest temperature; a relative
    # difference over all temperatures would be dominated by overlaps whose
    # means are compatible with zero)
    g_mean, c_mean = np.mean(gpu, 0), cpu.mean(0)
    print(f"\n{golden}: max |t| over the temperatures: e {np.abs(t[:, 0]).max():.2f}, "
          f"q2 {np.abs(t[:, 2]).max():.2f}, q2(k_min) {np.abs(t[:, 4]).max():.2f}, q2_CG {np.abs(t[:, 5]).max():.2f}; "
          f"relative difference of the means at T = {ref['T_range'][0]}: "
          + ", ".join(f"{n} {abs(g_mean[-1, j] - c_mean[-1, j]) / abs(c_mean[-1, j]):.2e}"
                      for j, n in [(0, "e"), (2, "q2"), (4, "q2(k_min)"), (5, "q2_CG")]))
    assert np.all(np.abs(t[:, 0]) < 3), t[:, 0]
    tt = t[:, [0, 2, 4, 5]]
    assert np.all(np.abs(tt) < 4), tt
    assert np.mean(tt ** 2) < 2.0, np.mean(tt ** 2)
    # Schwinger-Dyson identity (App. A.4.3) at the high temperatures, where
    # the chains equilibrate: the chain average vanishes within its error
    hot = slice(0, NT // 2)                                   # smallest beta = highest T
    sd = np.asarray(gpu)[:, hot, 8]
    z_sd = sd.mean(0) / (sd.std(0, ddof=1) / np.sqrt(len(sd)))
    assert np.all(np.abs(z_sd) < 4), z_sd


# the two streaming workloads bench.py times: L, samples, temperatures, and
# the (sample, slot) pairs checked against the oracle
FULL_SIZE = {
    "L64_S8_R64": (64, 8, 32, [(0, 0), (0, 1), (0, 63), (3, 20), (7, 62), (7, 63)]),
    "L32_S64_R48": (32, 64, 24, [(0, 0), (0, 1), (0, 47), (31, 20), (63, 46), (63, 47)]),
}


# coupling forms: storage precision, layout
FORMS = {"f16": (hsg.F16, hsg.BATCHED), "f32_plain": (hsg.F32, hsg.PLAIN),
         "bimodal_batched": (hsg.BIMODAL, hsg.BATCHED), "bimodal_plain": (hsg.BIMODAL, hsg.PLAIN)}
BIMODAL_D = 1.0


@pytest.mark.parametrize("name,form", [("L64_S8_R64", "f16"), ("L32_S64_R48", "f16"), ("L64_S8_R64", "f32_plain"),
                                       ("L64_S8_R64", "bimodal_batched"), ("L64_S8_R64", "bimodal_plain")])
def test_full_size_throughput_workload_sampled_parity(name, form):
    """The launch configurations bench.py times (L=64, 8 samples x 64
    lattices, the default, and L=32, 64 samples x 48 lattices; FP16
    couplings with two lattices per element, and at L=64 the same
    FP16-quantised values stored as FP32 with one lattice per element, and
    the one-byte bimodal couplings with D = 1 in both layouts; fused sweep in
    bands of 8 rows):
    one heat-bath and one overrelaxation sweep from the initial state,
    checked per half-sweep on whole sampled lattices, plus the fused energies
    and one PT sweep of every replica set against the oracle."""
    L, S, NT, sampled = FULL_SIZE[name]
    prec, layout = FORMS[form]
    n_rep, seed = 2, 1
    beta = gi.linear_betas(0.15, 0.75, NT)
    lat = hsg.Lattice([L] * S, beta, n_replicas=n_rep, coupling_prec=prec, layout=layout,
                      n_or=8, measure_every=10, seed=seed, bimodal_D=BIMODAL_D)
    plan = lat.get_sweep_plan(0)
    assert plan["fused"] and plan["band_rows"] == 8
    J9s = []
    for s in range(S):
        if prec == hsg.BIMODAL:
            bits = gi.bimodal_bits(L, seed, s)
            lat.set_couplings_bimodal(s, bits)
            J9s.append(oracle.bimodal_j9(bits, BIMODAL_D))
        else:
            J6 = gi.couplings(L, seed, s, precision="f16")
            lat.set_couplings(s, J6)
            J9s.append(oracle.j9_from_j6(J6))
        lat.set_spins_sample(s, np.stack([gi.random_spins(L, seed, s, j) for j in range(lat.R)]))

    n_amb_total = 0
    for kind in (oracle.HB, oracle.OR):
        hb_t = int(lat.get_counters()[0])
        before = {sl: lat.get_spins(*sl).astype(np.float64) for sl in sampled}
        (lat.sweep_hb if kind == oracle.HB else lat.sweep_or)(1)
        for (s, slot) in sampled:
            after = lat.get_spins(s, slot).astype(np.float64)
            col = _colours(L)
            J9 = J9s[s]
            t = _temp_of(lat)[s, slot]
            ref = before[(s, slot)].copy()
            oracle.half_sweep(L, J9, ref, 0, kind, float(beta[t]), seed, s * lat.R + slot, hb_t)
            mixed = np.ascontiguousarray(np.where((col == 0)[:, None], after, before[(s, slot)]))
            oracle.half_sweep(L, J9, mixed, 1, kind, float(beta[t]), seed, s * lat.R + slot, hb_t)
            ref = np.where((col == 0)[:, None], ref, mixed)
            diff = np.abs(after - ref).max(axis=1)
            if kind == oracle.HB:
                # frame-ambiguous sites (field at the equator h_z = 0) excepted
                h = oracle.fields(L, J9, before[(s, slot)], 0) + oracle.fields(L, J9, mixed, 1)
                amb = np.abs(h[:, 2]) < 1e-4 * np.linalg.norm(h, axis=1)
                # isotropic field directions put a fraction 1e-4 there: a
                # Poisson count, bounded 6 sigma (+6) above its mean
                lam = 1e-4 * amb.size
                assert amb.sum() <= lam + 6 * np.sqrt(lam) + 6, amb.sum()
                # there the draw may be made in either frame of the field
                diff[amb] = frame_ambiguous_diff(after[amb], ref[amb], h[amb])
                n_amb_total += int(amb.sum())
            assert diff.max() <= SWEEP_TOL, ((s, slot), kind, diff.max())
    # the sampled lattices hold ~1e-4 of their sites at the equator (over a
    # hundred at L = 64), so the either-frame comparison is exercised
    n_sites = len(sampled) * L ** 3
    if n_sites >= 10 ** 6:
        assert n_amb_total > 0
    # energies fused into that overrelaxation sweep, and one PT sweep
    E = lat.get_energies()
    for (s, slot) in sampled:
        ref = oracle.energy(L, J9s[s], lat.get_spins(s, slot).astype(np.float64))
        assert abs(E[s, slot] - ref) <= 2e-6 * abs(ref)
    perm = lat.get_perm().copy()
    pt_t = int(lat.get_counters()[1])
    lat.pt_swap()
    for s in range(S):
        for r in range(n_rep):
            oracle.pt_sweep(beta, E[s], perm[s, r], seed, s * n_rep + r, pt_t)
    assert np.array_equal(lat.get_perm(), perm)


def _colours(L):
    i = np.arange(L ** 3)
    return (i % L + (i // L) % L + i // (L * L)) % 2


def _temp_of(lat):
    perm = lat.get_perm()
    t = np.empty((lat.S, lat.R), dtype=np.int64)
    for s in range(lat.S):
        for r in range(lat.n_replicas):
            t[s, perm[s, r]] = np.arange(lat.NT)
    return t


@pytest.mark.parametrize("name", sorted(FULL_SIZE))
def test_full_size_measurement_matches_oracle(name):
    """The measurement (Sec. II.B overlaps and chiral overlaps, App. A.4.3
    Schwinger-Dyson residual, energies) at the full size of the streaming
    bench workloads, after one Monte Carlo step: every temperature of the
    first and the last sample against the oracle's measurement of the same
    spins and labels."""
    L, S, NT, _ = FULL_SIZE[name]
    n_rep, seed = 2, 1
    beta = gi.linear_betas(0.15, 0.75, NT)
    lat = hsg.Lattice([L] * S, beta, n_replicas=n_rep, coupling_prec=hsg.F16, layout=hsg.BATCHED,
                      n_or=8, measure_every=0, seed=seed)
    J9 = {}
    for s in range(S):
        J6 = gi.couplings(L, seed, s, precision="f16")
        lat.set_couplings(s, J6)
        if s in (0, S - 1):
            J9[s] = oracle.j9_from_j6(J6)
        lat.set_spins_sample(s, np.stack([gi.random_spins(L, seed, s, j) for j in range(lat.R)]))
    lat.run_steps(1)
    lat.reset_observables()
    lat.measure()
    obs, counts = lat.read_observables()
    assert np.all(counts == 1)
    E, perm, N = lat.get_energies(), lat.get_perm(), L ** 3
    for s in J9:
        st = lat.get_spins_sample(s).astype(np.float64)
        ref = np.zeros((NT, hsg.NOBS))
        for k in range(NT):
            for r in range(n_rep):
                e = E[s, perm[s, r, k]] / N
                ref[k, 0] += e
                ref[k, 1] += e * e
                ref[k, 8] += oracle.sd_residual(L, J9[s], st[perm[s, r, k]], 1 / beta[k])
            ref[k, 2:8] = oracle.measure_pair(L, st[perm[s, 0, k]], st[perm[s, 1, k]])
        assert np.allclose(obs[s, :, :2], ref[:, :2], rtol=1e-12, atol=0)   # from the same E
        scale = np.abs(ref).max(axis=0) + 1e-30
        assert np.all(np.abs(obs[s] - ref) <= 2e-5 * scale + 1e-9), np.abs(obs[s] - ref).max(axis=0)
