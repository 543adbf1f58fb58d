"""Pins of the oracle's Monte Carlo step (Sec. III, App. A.1): the step driver is
exactly the documented composition of sweeps, energies, parallel tempering and
measurements, and the equilibrium Schwinger-Dyson identity (App. A.4.3) holds
within errors."""
import numpy as np

import hsg_inputs as gi
import oracle


def _explicit_steps(L, J6, spins, beta, n_rep, seed, sample, n_steps, n_or, m_every):
    """The step written out call by call with the documented counters."""
    N = L ** 3
    nT = len(beta)
    R = n_rep * nT
    J9 = oracle.j9_from_j6(J6)
    s = [spins[j].astype(np.float64).copy() for j in range(R)]
    perm = [np.arange(nT, dtype=np.int32) + r * nT for r in range(n_rep)]
    obs = np.zeros((nT, oracle.N_OBS))
    hb_t = pt_t = 0
    for step in range(1, n_steps + 1):
        temp_of = np.empty(R, dtype=int)
        for r in range(n_rep):
            temp_of[perm[r]] = np.arange(nT)
        E = np.zeros(R)
        for slot in range(R):
            b = beta[temp_of[slot]]
            oracle.sweep(L, J9, s[slot], oracle.HB, b, seed, sample * R + slot, hb_t)
            for _ in range(n_or):
                oracle.sweep(L, J9, s[slot], oracle.OR)
            E[slot] = oracle.energy(L, J9, s[slot])
        hb_t += 1
        if nT > 1:
            for r in range(n_rep):
                oracle.pt_sweep(beta, E, perm[r], seed, sample * n_rep + r, pt_t)
        pt_t += 1
        if step % m_every == 0:
            for k in range(nT):
                for r in range(n_rep):
                    e = E[perm[r][k]] / N
                    obs[k, 0] += e
                    obs[k, 1] += e * e
                    obs[k, 8] += oracle.sd_residual(L, J9, s[perm[r][k]], 1 / beta[k])
                for p in range(0, n_rep - 1, 2):
                    obs[k, 2:8] += oracle.measure_pair(L, s[perm[p][k]], s[perm[p + 1][k]])
    return np.stack(s), np.concatenate(perm), obs, E


def test_run_is_the_documented_composition():
    L, n_rep, seed, sample = 4, 2, 77, 3
    beta = gi.linear_betas(0.3, 1.2, 3)
    J6 = gi.couplings(L, seed=seed, sample=sample)
    R = n_rep * len(beta)
    spins = gi.random_spins_batch(L, seed, sample, R)
    ref_s, ref_perm, ref_obs, ref_E = _explicit_steps(L, J6, spins, beta, n_rep, seed,
                                                      sample, 6, 3, 2)
    smp = oracle.Sample(L, J6, spins, beta, n_rep, seed, sample_index=sample)
    smp.run(6, 3, 2, n_threads=2)
    assert np.array_equal(smp.spins, ref_s)
    assert np.array_equal(smp.perm, ref_perm)
    assert np.array_equal(smp.energies, ref_E)
    assert np.allclose(smp.obs, ref_obs, rtol=0, atol=1e-15)
    assert smp.counts.tolist() == [3, 3, 3]
    assert smp.hb_t[0] == 6 and smp.pt_t[0] == 6


def test_schwinger_dyson_identity_in_equilibrium():
    L = 4
    beta = np.array([0.5, 1.0])
    J6 = gi.couplings(L, seed=31)
    spins = gi.random_spins_batch(L, 31, 0, 4)
    smp = oracle.Sample(L, J6, spins, beta, 2, seed=31)
    smp.run(200, 2, 0)
    blocks = []
    for _ in range(20):
        smp.obs[:] = 0
        smp.counts[:] = 0
        smp.run(100, 2, 1)
        blocks.append(smp.obs[:, 8] / (smp.counts * 2))
    blocks = np.array(blocks)
    mean = blocks.mean(0)
    err = blocks.std(0, ddof=1) / np.sqrt(len(blocks))
    assert np.all(np.abs(mean) < 5 * err), (mean, err)
    # the identity is not trivially zero: its two terms are large
    assert np.all(err < 0.2)
