"""Long-run parity of the CUDA path with the FP64 oracle (statistical), and
parity at the full size of the throughput workload (sampled lattices).

Trajectories under identical random streams separate after a few sweeps
(overrelaxation is chaotic), so after that the GPU run and the oracle run are
independent realisations of the same Markov chain.  Their long-run averages
must agree within 3 sigma, sigma from the spread of block averages (binning)
of each run.
"""
import json
import os

import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import SWEEP_TOL

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _block_means(obs, counts, n_rep):
    n = counts[..., None].astype(float)
    m = np.empty_like(obs)
    m[..., 0:2] = obs[..., 0:2] / (n * n_rep)
    m[..., 2:8] = obs[..., 2:8] / (n * (n_rep // 2))
    m[..., 8] = obs[..., 8] / (n[..., 0] * n_rep)
    return m


def _mean_err(blocks):
    b = np.asarray(blocks)
    return b.mean(0), b.std(0, ddof=1) / np.sqrt(len(b))


def test_long_run_L8_single_temperature_matches_oracle():
    """Plain FP32 form, L=8, T=0.5, 2 replicas, 1 HB + 8 OR per step,
    observables every step: 1000 steps on both sides, 20 blocks of 50,
    the first 4 blocks discarded."""
    L, beta, seed = 8, 2.0, 1
    J6 = gi.couplings(L, seed, 0)
    spins = gi.random_spins_batch(L, seed, 0, 2)
    lat = hsg.Lattice(L, [beta], n_replicas=2, coupling_prec=hsg.F32, layout=hsg.PLAIN, n_or=8,
                      measure_every=1, seed=seed)
    lat.set_couplings(0, J6)
    for j in range(2):
        lat.set_spins(0, j, spins[j])
    smp = oracle.Sample(L, J6, spins, [beta], 2, seed)
    gpu, cpu = [], []
    for b in range(20):
        lat.reset_observables()
        lat.run_steps(50)
        o, c = lat.read_observables()
        gpu.append(_block_means(o[0, 0], c[0, 0], 2))
        smp.obs[:] = 0
        smp.counts[:] = 0
        smp.run(50, 8, 1)
        cpu.append(_block_means(smp.obs[0], smp.counts[0], 2))
    mg, eg = _mean_err(gpu[4:])
    mc, ec = _mean_err(cpu[4:])
    for j, name in [(0, "e"), (2, "q2"), (5, "c2")]:
        z = (mg[j] - mc[j]) / np.sqrt(eg[j] ** 2 + ec[j] ** 2)
        assert abs(z) < 3, (name, mg[j], mc[j], z)
    # the chains did separate: the comparison is statistical, not trivial
    assert not np.allclose(lat.get_spins(0, 0), smp.spins[0], atol=1e-3)


def test_parallel_tempering_L16_matches_stored_oracle():
    """L=16, one sample, 16 temperatures evenly spaced in [0.15, 0.75] x 2
    replicas, 20000 steps of HB + 8 OR + PT, observables every 10 steps.
    The oracle's block averages were stored by tests/golden/make_pt_L16_oracle.py.
    Means over the last 10 blocks of 1000 steps agree per temperature and
    observable: |z| < 4 everywhere (16 temperatures x 4 observables) and
    mean z^2 below 2.5; energies, which equilibrate fastest, within 3 sigma."""
    with open(os.path.join(HERE, "golden", "pt_L16_oracle.json")) as f:
        ref = json.load(f)
    L, NT, n_rep, seed = ref["L"], ref["n_temps"], ref["n_replicas"], ref["seed"]
    beta = gi.linear_betas(*ref["T_range"], NT)
    lat = hsg.Lattice(L, beta, n_replicas=n_rep, coupling_prec=hsg.F32, layout=hsg.BATCHED,
                      n_or=ref["n_or"], measure_every=ref["measure_every"], seed=seed)
    lat.set_couplings(0, gi.couplings(L, seed, 0))
    for j in range(lat.R):
        lat.set_spins(0, j, gi.random_spins(L, seed, 0, j))
    gpu = []
    for b in range(ref["steps"] // ref["block_steps"]):
        lat.reset_observables()
        lat.run_steps(ref["block_steps"])
        o, c = lat.read_observables()
        gpu.append(_block_means(o[0], c[0], n_rep))
    keep = slice(len(gpu) // 2, None)
    mg, eg = _mean_err(gpu[keep])
    mc, ec = _mean_err(np.asarray(ref["block_means"])[keep])
    zs = []
    for j in (0, 2, 4, 5):                       # e, q2, q2(k_min), q2_CG
        z = (mg[:, j] - mc[:, j]) / np.sqrt(eg[:, j] ** 2 + ec[:, j] ** 2)
        zs.append(z)
        if j == 0:
            assert np.all(np.abs(z) < 3), z
    zs = np.concatenate(zs)
    assert np.all(np.abs(zs) < 4), zs
    assert np.mean(zs ** 2) < 2.5, np.mean(zs ** 2)
    # Schwinger-Dyson identity (App. A.4.3) at the higher temperatures
    hot = slice(0, NT // 2)                      # smallest beta = highest T
    z_sd = mg[hot, 8] / eg[hot, 8]
    assert np.all(np.abs(z_sd) < 4), z_sd


def test_full_size_throughput_workload_sampled_parity():
    """The launch configuration bench.py times (L=64, 8 samples x 64
    lattices, FP16 couplings, two lattices per element, fused sweep in bands
    of 16 rows): one heat-bath and one overrelaxation sweep from the initial
    state, checked per half-sweep on whole sampled lattices, plus the fused
    energies and one PT sweep against the oracle."""
    L, S, NT, n_rep, seed = 64, 8, 32, 2, 1
    beta = gi.linear_betas(0.15, 0.75, NT)
    lat = hsg.Lattice([L] * S, beta, n_replicas=n_rep, coupling_prec=hsg.F16, layout=hsg.BATCHED,
                      n_or=8, measure_every=10, seed=seed)
    plan = lat.get_sweep_plan(0)
    assert plan["fused"] and plan["band_rows"] == 16
    J = [gi.couplings(L, seed, s, precision="f16") for s in range(S)]
    for s in range(S):
        lat.set_couplings(s, J[s])
        for j in range(lat.R):
            lat.set_spins(s, j, gi.random_spins(L, seed, s, j))
    sampled = [(0, 0), (0, 1), (0, 63), (3, 20), (7, 62), (7, 63)]

    for kind in (oracle.HB, oracle.OR):
        hb_t = int(lat.get_counters()[0])
        before = {sl: lat.get_spins(*sl).astype(np.float64) for sl in sampled}
        (lat.sweep_hb if kind == oracle.HB else lat.sweep_or)(1)
        for (s, slot) in sampled:
            after = lat.get_spins(s, slot).astype(np.float64)
            col = _colours(L)
            J9 = oracle.j9_from_j6(J[s])
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
                assert amb.sum() <= 3
                diff = diff[~amb]
            assert diff.max() <= SWEEP_TOL, ((s, slot), kind, diff.max())
    # energies fused into that overrelaxation sweep, and one PT sweep
    E = lat.get_energies()
    for (s, slot) in sampled:
        ref = oracle.energy(L, oracle.j9_from_j6(J[s]), lat.get_spins(s, slot).astype(np.float64))
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
