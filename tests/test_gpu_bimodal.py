"""Bimodal couplings stored in one byte per bond (Sec. II.A: J = +-1,
D^ab = +-D): decoding, sweeps, energies, resident steps and measurement
against the oracle, which decodes the same bytes itself."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import SWEEP_TOL, compare_sweep, state

pytestmark = pytest.mark.gpu
SEED = 3


def make_bimodal(Ls, betas, D, n_rep=2, layout=hsg.PLAIN, n_or=8, measure_every=0, **kw):
    lat = hsg.Lattice(list(Ls), betas, n_replicas=n_rep, coupling_prec=hsg.BIMODAL, layout=layout,
                      n_or=n_or, measure_every=measure_every, seed=SEED, bimodal_D=D, **kw)
    bits, J9s = [], []
    for s, L in enumerate(Ls):
        b = gi.bimodal_bits(L, SEED, s)
        lat.set_couplings_bimodal(s, b)
        bits.append(b)
        J9s.append(oracle.bimodal_j9(b, D))
        for slot in range(lat.R):
            lat.set_spins(s, slot, gi.random_spins(L, SEED, s, slot))
    return lat, bits, J9s


@pytest.mark.parametrize("D", [0.5, 1.0])
def test_bytes_roundtrip_and_decoded_matrices(D):
    lat, bits, J9s = make_bimodal([8, 6], [1.0], D)
    for s in range(2):
        assert np.array_equal(lat.get_couplings_bimodal(s), bits[s])
        J6 = lat.get_couplings(s).astype(np.float64)
        J9 = J9s[s]
        want = np.stack([J9[..., 0], J9[..., 4], J9[..., 8], J9[..., 1], J9[..., 2], J9[..., 5]], -1)
        assert np.array_equal(J6, want)


def test_float_setter_and_bad_bytes_rejected():
    lat, bits, _ = make_bimodal([6], [1.0], 0.5)
    with pytest.raises(hsg.HsgError):
        lat.set_couplings(0, np.zeros((6 ** 3, 3, 6), np.float32))
    bad = bits[0].copy()
    bad[5, 1] |= 0x80
    with pytest.raises(hsg.HsgError):
        lat.set_couplings_bimodal(0, bad)
    assert np.array_equal(lat.get_couplings_bimodal(0), bits[0])      # unchanged


CASES = [
    # Ls, betas, n_rep, layout, D, sweep kernel
    ([8], [2.0], 2, hsg.PLAIN, 0.5, hsg.SWEEP_AUTO),
    ([12, 8], [0.7, 1.9, 4.0], 2, hsg.BATCHED, 1.0, hsg.SWEEP_AUTO),
    ([16], [1.0, 3.0], 2, hsg.BATCHED, 0.5, hsg.SWEEP_TWO_PASS),
    ([40], [1.2, 3.0], 1, hsg.PLAIN, 1.0, hsg.SWEEP_AUTO),      # banded fused sweep
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_per_sweep_parity_ten_sweeps(case):
    Ls, betas, n_rep, layout, D, kernel = CASES[case]
    lat, _, J9s = make_bimodal(Ls, betas, D, n_rep=n_rep, layout=layout, sweep_kernel=kernel)
    for kind in [oracle.HB] + [oracle.OR] * 8 + [oracle.HB]:
        hb_t = int(lat.get_counters()[0])
        before = state(lat)
        (lat.sweep_hb if kind == oracle.HB else lat.sweep_or)(1)
        d, _, du = compare_sweep(lat, None, before, state(lat), kind, hb_t, J9s=J9s)
        assert d <= SWEEP_TOL and du <= SWEEP_TOL, (kind, d, du)


def test_energies_match_oracle():
    lat, _, J9s = make_bimodal([12, 8], [0.5, 2.0], 1.0, layout=hsg.BATCHED)
    lat.sweep_hb(2)
    lat.sweep_or(3)
    E = lat.get_energies()
    st = state(lat)
    for s, L in enumerate([12, 8]):
        for slot in range(lat.R):
            ref = oracle.energy(L, J9s[s], st[s][slot])
            assert abs(E[s, slot] - ref) <= 2e-6 * abs(ref)


@pytest.mark.parametrize("Ls", [[8, 12], [16]], ids=["whole_sets", "split_sets"])
def test_resident_steps_equal_streaming_steps(Ls):
    """Whole replica sets per CTA (L = 8, 12) and parts of sets with PT
    between launches (L = 16, one-byte bonds resident beside one group)."""
    betas = gi.linear_betas(0.2, 0.8, 8)
    a, _, _ = make_bimodal(Ls, betas, 0.5, n_rep=2, layout=hsg.BATCHED, n_or=3, measure_every=2)
    b, _, _ = make_bimodal(Ls, betas, 0.5, n_rep=2, layout=hsg.BATCHED, n_or=3, measure_every=2,
                           persistent=True)
    a.run_steps(6)
    b.run_steps(6)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    Ea, Eb = a.get_energies(), b.get_energies()
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-9 * np.abs(Ea).max())


def test_measurement_schwinger_dyson_terms_use_the_bimodal_field():
    """The measured Schwinger-Dyson residual needs the local field, so it
    checks the decoding inside the measurement kernel against the oracle."""
    betas = [0.8, 3.0]
    lat, _, J9s = make_bimodal([8, 16], betas, 1.0, n_rep=2, layout=hsg.BATCHED)
    lat.run_steps(3)
    lat.reset_observables()
    lat.measure()
    obs, counts = lat.read_observables()
    st = state(lat)
    perm = lat.get_perm()
    for s, L in enumerate([8, 16]):
        for k, beta in enumerate(betas):
            # accumulated per temperature as the sum over the replicas
            sd = sum(oracle.sd_residual(L, J9s[s], st[s][perm[s, r, k]], 1.0 / beta) for r in range(2))
            assert abs(obs[s, k, 8] - sd) <= 2e-5 * max(1.0, abs(sd)), (s, k, obs[s, k, 8], sd)


def test_checkpoint_resume_is_bit_identical_and_checks_D(tmp_path):
    betas = gi.linear_betas(0.3, 1.0, 2)
    a, _, _ = make_bimodal([8], betas, 0.5, layout=hsg.BATCHED, measure_every=1)
    a.run_steps(3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.run_steps(3)
    b = hsg.Lattice([8], betas, n_replicas=2, coupling_prec=hsg.BIMODAL, layout=hsg.BATCHED,
                    measure_every=1, seed=SEED, bimodal_D=0.5)
    b.load(path)
    b.run_steps(3)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_couplings_bimodal(0), b.get_couplings_bimodal(0))
    c = hsg.Lattice([8], betas, n_replicas=2, coupling_prec=hsg.BIMODAL, layout=hsg.BATCHED,
                    measure_every=1, seed=SEED, bimodal_D=1.0)
    with pytest.raises(hsg.HsgError):
        c.load(path)                                   # another D: refused
