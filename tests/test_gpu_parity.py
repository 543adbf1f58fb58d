"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Per-sweep parity: from identical input states and identical Philox streams,
one GPU sweep and one oracle sweep agree per site within 2e-5 (max |ds|),
checked over 10 consecutive sweeps (the oracle restarted from the GPU's state
before each sweep).  Heat-bath sweeps are also compared free-running.
Integer work (Philox words, PT labels and acceptance counts) is bit-exact.
Sizes span several thread blocks with a ragged tail, mixed L, both layouts
and both coupling precisions.
"""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import SWEEP_TOL, compare_sweep, make, max_diff, state, temp_of

pytestmark = pytest.mark.gpu


def test_device_philox_matches_oracle_bitwise():
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 2**32, size=(20000, 6), dtype=np.uint64).astype(np.uint32)
    rows[:100, :4] = 0                       # zero counters
    rows[100:200, 4:] = 0xFFFFFFFF           # all-ones keys
    dev = hsg.philox4x32_10(rows)
    ref = np.stack([oracle.philox4x32(r[:4], r[4:])[0] for r in rows])
    assert np.array_equal(dev, ref)


@pytest.mark.parametrize("prec", [hsg.F32, hsg.F16])
@pytest.mark.parametrize("layout", [hsg.PLAIN, hsg.BATCHED])
def test_couplings_and_spins_roundtrip(prec, layout):
    lat, J = make([6, 8], [0.5, 1.0], n_rep=2, prec=prec, layout=layout)
    for s, L in enumerate([6, 8]):
        assert np.array_equal(lat.get_couplings(s), J[s])
        for slot in range(lat.R):
            assert np.array_equal(lat.get_spins(s, slot), gi.random_spins(L, 1, s, slot))


CASES = [
    # (Ls, betas, n_rep, prec, layout)
    ([8], [2.0], 2, hsg.F32, hsg.PLAIN),                 # the L=8, T=0.5 plain workload
    ([8], [2.0], 2, hsg.F32, hsg.BATCHED),
    ([12, 8], [0.7, 1.9, 4.0], 2, hsg.F16, hsg.BATCHED),  # mixed L, ragged blocks
    ([6], [0.0, 1.0, 5.0], 3, hsg.F16, hsg.PLAIN),         # beta = 0, odd replicas
    ([4], [1.3], 1, hsg.F32, hsg.PLAIN),                   # smallest lattice
    ([16], [1.0, 6.0], 2, hsg.F16, hsg.PLAIN),
    ([40], [1.2, 3.0], 2, hsg.F16, hsg.BATCHED),          # fused sweep in bands of rows
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_per_sweep_parity_ten_sweeps(case):
    Ls, betas, n_rep, prec, layout = CASES[case]
    lat, J = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout)
    kinds = [oracle.HB] + [oracle.OR] * 8 + [oracle.HB]
    worst, n_amb, n_sites = 0.0, 0, 0
    for kind in kinds:
        hb_t = int(lat.get_counters()[0])
        before = state(lat)
        if kind == oracle.HB:
            lat.sweep_hb(1)
        else:
            lat.sweep_or(1)
        after = state(lat)
        d, amb, du = compare_sweep(lat, J, before, after, kind, hb_t)
        worst = max(worst, d)
        n_amb += amb
        n_sites += lat.R * sum(L ** 3 for L in Ls)
        assert d <= SWEEP_TOL, (kind, d)
        assert du <= SWEEP_TOL, (kind, du)
    assert worst > 0.0          # the two sides really are different programs
    assert n_amb <= max(3, 1e-3 * n_sites)


def test_heat_bath_free_running_ten_sweeps():
    lat, J = make([8], [2.0], n_rep=2)
    ref = state(lat)
    for t in range(10):
        lat.sweep_hb(1)
        for slot in range(lat.R):
            oracle.sweep(8, oracle.j9_from_j6(J[0]), ref[0][slot], oracle.HB, 2.0, lat.seed, slot, t)
    assert max_diff(state(lat), ref) <= SWEEP_TOL


def test_energies_match_oracle_on_the_same_state():
    lat, J = make([12, 8], [0.5, 2.0], n_rep=2, prec=hsg.F16, layout=hsg.BATCHED)
    lat.sweep_hb(2)
    lat.sweep_or(3)         # energies fused into the last white half-sweep
    E_fused = lat.get_energies()
    lat.energy()            # standalone evaluation
    E_direct = lat.get_energies()
    st = state(lat)
    for s, L in enumerate([12, 8]):
        J9 = oracle.j9_from_j6(J[s])
        for slot in range(lat.R):
            ref = oracle.energy(L, J9, st[s][slot])
            assert abs(E_fused[s, slot] - ref) <= 2e-6 * abs(ref)
            assert abs(E_direct[s, slot] - ref) <= 2e-6 * abs(ref)


def test_ferromagnet_energies_seven_digits():
    """App. A.4.3: with ferromagnetic couplings the GPU energies equal an
    independent CPU program's to the 7th significant digit."""
    L = 8
    lat, J = make([L], [2.0], n_rep=2, law="ferro")
    up = np.zeros((L ** 3, 3), dtype=np.float32)
    up[:, 2] = 1.0
    for slot in range(lat.R):
        lat.set_spins(0, slot, up)
    lat.run_steps(3)
    E = lat.get_energies()
    st = state(lat)
    J9 = oracle.j9_from_j6(J[0])
    for slot in range(lat.R):
        ref = oracle.energy(L, J9, st[0][slot])
        assert abs(E[0, slot] - ref) <= 5e-8 * abs(ref), (E[0, slot], ref)
        assert -3 * L ** 3 < ref < -2.0 * L ** 3     # ordered at T = 0.5


# 7 temperatures; 33 (a warp's lanes take two pairs each); 300 (more than the
# warp-per-set kernel stages: the thread-per-set kernel)
@pytest.mark.parametrize("NT,L", [(7, 6), (33, 4), (300, 4)])
def test_pt_labels_bit_exact(NT, L):
    betas = gi.linear_betas(0.2, 1.5, NT)
    lat, J = make([L, L, L], betas, n_rep=3)
    rng = np.random.default_rng(4)
    N = L ** 3
    perm = lat.get_perm().copy()
    acc = np.zeros((3, 3, NT - 1), dtype=np.int64)
    for t in range(40):
        E = rng.normal(-1.5 * N, 0.05 * N, size=(3, lat.R))
        lat.set_energies(E)
        lat.pt_swap()
        for s in range(3):
            for r in range(3):
                oracle.pt_sweep(betas, E[s], perm[s, r], lat.seed, s * 3 + r, t, acc[s, r])
        assert np.array_equal(lat.get_perm(), perm)
    assert np.array_equal(lat.get_pt_accepts(), acc)
    assert 0 < acc.sum() < 40 * acc.size


def _oracle_measure(lat, J, st, E):
    obs = np.zeros((lat.S, lat.NT, hsg.NOBS))
    perm = lat.get_perm()
    for s, L in enumerate(lat.Ls):
        N = L ** 3
        J9 = oracle.j9_from_j6(J[s])
        for k in range(lat.NT):
            for r in range(lat.n_replicas):
                slot = perm[s, r, k]
                e = E[s, slot] / N
                obs[s, k, 0] += e
                obs[s, k, 1] += e * e
                if lat.beta[k] > 0:
                    obs[s, k, 8] += oracle.sd_residual(L, J9, st[s][slot], 1 / lat.beta[k])
            for p in range(0, lat.n_replicas - 1, 2):
                obs[s, k, 2:8] += oracle.measure_pair(L, st[s][perm[s, p, k]], st[s][perm[s, p + 1, k]])
    return obs


@pytest.mark.parametrize("layout,Ls", [(hsg.PLAIN, [12, 8]), (hsg.BATCHED, [12, 8]),
                                       (hsg.BATCHED, [16, 8])])
def test_measurement_matches_oracle(layout, Ls):
    """Small lattices (N < 4096) are measured one warp per replica pair, L=16
    by blocks over chunks of sites."""
    betas = [0.0, 0.8, 3.0]
    lat, J = make(Ls, betas, n_rep=4, prec=hsg.F16, layout=layout)
    lat.run_steps(4)
    lat.reset_observables()
    lat.measure()
    obs, counts = lat.read_observables()
    ref = _oracle_measure(lat, J, state(lat), lat.get_energies())
    assert np.all(counts == 1)
    assert np.allclose(obs[..., :2], ref[..., :2], rtol=1e-12, atol=0)   # from the same E
    scale = np.abs(ref).max(axis=(0, 1)) + 1e-30
    assert np.all(np.abs(obs - ref) <= 2e-5 * scale + 1e-9), np.abs(obs - ref).max(axis=(0, 1))


def test_run_steps_is_the_step_composition():
    """The graph-replayed step equals the explicit call sequence bit for bit."""
    betas = gi.linear_betas(0.3, 1.0, 4)
    a, _ = make([8, 12], betas, n_rep=2, prec=hsg.F16, layout=hsg.BATCHED, n_or=3, measure_every=2)
    b, _ = make([8, 12], betas, n_rep=2, prec=hsg.F16, layout=hsg.BATCHED, n_or=3, measure_every=2)
    a.run_steps(6)
    for step in range(1, 7):
        b.sweep_hb(1)
        b.sweep_or(3)
        b.pt_swap()
        if step % 2 == 0:
            b.measure()
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    oa, ca = a.read_observables()
    ob, cb = b.read_observables()
    assert np.array_equal(oa, ob) and np.array_equal(ca, cb)
    assert ca.min() == 3
    assert list(a.get_counters()) == [6, 6, 6]


def test_run_step_matches_oracle_step_from_equilibrium():
    """One whole Monte Carlo step (HB + 8 OR + energies + PT) from an
    equilibrated state: spins within the per-sweep tolerance accumulated
    over the step's 9 sweeps, labels identical."""
    betas = gi.linear_betas(0.5, 1.0, 3)
    lat, J = make([8], betas, n_rep=2)
    lat.run_steps(200)
    st = state(lat)
    perm0 = lat.get_perm()
    hb_t, pt_t, steps = (int(x) for x in lat.get_counters())
    smp = oracle.Sample(8, J[0], np.stack(st[0]), betas, 2, lat.seed)
    smp.perm[:] = perm0.reshape(-1)
    smp.hb_t[0], smp.pt_t[0], smp.steps[0] = hb_t, pt_t, steps
    lat.run_steps(1)
    smp.run(1, 8, 0)
    assert np.array_equal(lat.get_perm().reshape(-1), smp.perm)
    d = max(np.abs(lat.get_spins(0, j) - smp.spins[j]).max() for j in range(lat.R))
    assert d < 1e-3, d


def test_checkpoint_resume_is_bit_identical(tmp_path):
    betas = gi.linear_betas(0.3, 1.0, 4)
    a, _ = make([8], betas, n_rep=2, layout=hsg.BATCHED, measure_every=1)
    a.run_steps(3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.run_steps(3)
    b = hsg.Lattice([8], betas, n_replicas=2, layout=hsg.BATCHED, measure_every=1, seed=a.seed)
    b.load(path)
    b.run_steps(3)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.read_observables()[0], b.read_observables()[0])
    assert np.array_equal(a.get_counters(), b.get_counters())


@pytest.mark.parametrize("persistent", [1, 2])
def test_checkpoint_resume_bit_identical_with_resident_steps(tmp_path, persistent):
    """Save a mixed-size context running resident steps (one launch per size,
    or both sizes in one launch) and resume it in a fresh context of the same
    shape, which may even use the other resident mode: the continued run
    equals the uninterrupted one bit for bit (spins, labels, acceptances,
    observables, counters)."""
    betas = gi.linear_betas(0.3, 1.2, 8)
    a, _ = make([12, 8], betas, n_rep=2, prec=hsg.F16, layout=hsg.BATCHED, n_or=2, measure_every=2,
                persistent=persistent)
    a.run_steps(4)
    path = str(tmp_path / "ck_res.bin")
    a.save(path)
    a.run_steps(4)
    other = 3 - persistent
    b = hsg.Lattice([12, 8], betas, n_replicas=2, coupling_prec=hsg.F16, layout=hsg.BATCHED, n_or=2,
                    measure_every=2, seed=a.seed, persistent=other)
    b.load(path)
    b.run_steps(4)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    assert np.array_equal(a.get_pt_accepts(), b.get_pt_accepts())
    assert np.array_equal(a.get_counters(), b.get_counters())
    oa, ca = a.read_observables()
    ob, cb = b.read_observables()
    assert np.array_equal(ca, cb) and np.allclose(oa, ob, rtol=1e-9, atol=1e-12)


def test_mismatched_checkpoint_rejected(tmp_path):
    a, _ = make([8], [1.0], n_rep=2)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    b = hsg.Lattice([6], [1.0], n_replicas=2)
    with pytest.raises(hsg.HsgError, match="EINVAL"):
        b.load(path)


def test_or_conserves_energy_and_norm_on_gpu():
    lat, _ = make([16], [1.0], n_rep=2, prec=hsg.F16, layout=hsg.BATCHED)
    lat.energy()
    E0 = lat.get_energies()
    lat.sweep_or(50)
    E1 = lat.get_energies()
    assert np.all(np.abs(E1 - E0) <= 1e-4 * np.abs(E0))
    for slot in range(lat.R):
        n = np.linalg.norm(lat.get_spins(0, slot), axis=1)
        assert np.abs(n - 1).max() < 1e-4


FUSED_CASES = [
    # (Ls, n_rep, prec, layout, band_rows): whole-plane and banded tilings of
    # the fused sweep (band_rows 0: the library's choice)
    ([8, 12], 2, hsg.F32, hsg.PLAIN, 0),
    ([16], 2, hsg.F16, hsg.BATCHED, 0),
    ([24], 1, hsg.F16, hsg.BATCHED, 0),                # whole planes
    ([24], 1, hsg.F16, hsg.BATCHED, 8),
    ([32], 1, hsg.F16, hsg.BATCHED, 0),
    ([32], 1, hsg.F16, hsg.BATCHED, 16),
    ([40], 1, hsg.F16, hsg.BATCHED, 0),
    ([48], 1, hsg.F32, hsg.PLAIN, 0),
    ([64], 1, hsg.F16, hsg.BATCHED, 16),
    ([64], 1, hsg.F16, hsg.BATCHED, 8),                # compile-time L = 64, 8-row tiling
    ([64], 1, hsg.F32, hsg.PLAIN, 8),
]


@pytest.mark.parametrize("case", range(len(FUSED_CASES)))
def test_fused_sweep_equals_two_pass_bitwise(case):
    """The fused one-pass sweep and the two-pass half-sweeps sum each field in
    the same order, so they must give identical spins, energies and labels."""
    Ls, n_rep, prec, layout, band = FUSED_CASES[case]
    betas = gi.linear_betas(0.4, 1.2, 2)
    runs = []
    for kernel in (hsg.SWEEP_AUTO, hsg.SWEEP_TWO_PASS):
        lat = hsg.Lattice(Ls, betas, n_replicas=n_rep, coupling_prec=prec, layout=layout, n_or=3,
                          measure_every=2, seed=5, sweep_kernel=kernel,
                          band_rows=band if kernel == hsg.SWEEP_AUTO else 0)
        if kernel == hsg.SWEEP_AUTO and band:
            assert lat.get_sweep_plan(0)["band_rows"] == band
        pstr = "f16" if prec == hsg.F16 else "f32"
        for s, L in enumerate(Ls):
            lat.set_couplings(s, gi.couplings(L, 5, s, precision=pstr))
            for j in range(lat.R):
                lat.set_spins(s, j, gi.random_spins(L, 5, s, j))
        lat.sweep_hb(1)
        lat.sweep_or(2)
        E1 = lat.get_energies()
        lat.run_steps(3)
        runs.append((state(lat), E1, lat.get_energies(), lat.get_perm(), lat.read_observables()[0]))
        lat.destroy()
    (sa, e1a, e2a, pa, oa), (sb, e1b, e2b, pb, ob) = runs
    assert all(np.array_equal(x, y) for rx, ry in zip(sa, sb) for x, y in zip(rx, ry))
    assert np.allclose(e1a, e1b, rtol=1e-12) and np.allclose(e2a, e2b, rtol=1e-12)
    assert np.array_equal(pa, pb)
    assert np.allclose(oa, ob, rtol=1e-9, atol=1e-12)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A device-side wait that runs out is reported as HSG_ETIMEOUT on the
    host; nothing hangs and the context keeps working."""
    lat, J = make([8], [2.0], n_rep=2, layout=hsg.BATCHED)
    before = state(lat)
    assert lat.selftest_wait_timeout(100000) == 4          # HSG_ETIMEOUT
    assert all(np.array_equal(x, y) for rx, ry in zip(before, state(lat)) for x, y in zip(rx, ry))
    hb_t = int(lat.get_counters()[0])
    lat.sweep_hb(1)
    lat.synchronize()
    d, _, _ = compare_sweep(lat, J, before, state(lat), oracle.HB, hb_t)
    assert d <= SWEEP_TOL


def test_device_pointer_spins_roundtrip():
    """Spins set from and read into torch CUDA tensors (no host copy) equal
    the host-buffer path, for both layouts and a slot of each parity."""
    import torch
    for layout in (hsg.PLAIN, hsg.BATCHED):
        lat, _ = make([8, 12], [1.0, 2.0], n_rep=2, prec=hsg.F16, layout=layout)
        for s, L in enumerate([8, 12]):
            for slot in (1, 2):
                host = gi.random_spins(L, 9, s, slot)
                dev = torch.from_numpy(host).cuda()
                lat.set_spins_device(s, slot, dev)
                assert np.array_equal(lat.get_spins(s, slot), host)
                out = torch.empty_like(dev)
                lat.get_spins_device(s, slot, out)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), host)


SIZES = [(L, prec, layout) for L in (4, 6, 10, 14, 18, 20) for prec in (hsg.F32, hsg.F16)
         for layout in (hsg.PLAIN, hsg.BATCHED)]


@pytest.mark.parametrize("L,prec,layout", SIZES,
                         ids=[f"L{L}_{'f16' if p else 'f32'}_{'B' if lay else 'P'}" for L, p, lay in SIZES])
def test_per_half_sweep_parity_across_sizes(L, prec, layout):
    """One heat-bath and two overrelaxation sweeps per half-sweep against the
    oracle at lattice sizes the other cases do not use (whole-plane and
    banded fused tilings), both coupling precisions and both layouts."""
    lat, J = make([L], [0.6, 2.2], n_rep=2, prec=prec, layout=layout)
    for kind in (oracle.HB, oracle.OR, oracle.OR):
        hb_t = int(lat.get_counters()[0])
        before = state(lat)
        (lat.sweep_hb if kind == oracle.HB else lat.sweep_or)(1)
        d, amb, du = compare_sweep(lat, J, before, state(lat), kind, hb_t)
        assert d <= SWEEP_TOL and du <= SWEEP_TOL, (kind, d, du)
        assert amb <= max(3, 1e-3 * lat.R * L ** 3)
    lat.destroy()


def test_a_smaller_context_does_not_shrink_another_contexts_limits():
    """Kernel shared-memory limits belong to the kernels, which every context
    shares: creating a context that needs less (smaller rings, smaller
    measurement tables) after one that needs more must leave the first
    runnable.  Both then run whole measured steps and match one context
    alone bit for bit."""
    big = dict(Ls=[32], betas=[0.6, 1.3], n_rep=2)
    small = dict(Ls=[8], betas=[0.6, 1.3], n_rep=2)

    def make_ctx(c, **kw):
        lat = hsg.Lattice(c["Ls"], c["betas"], n_replicas=c["n_rep"], coupling_prec=hsg.F16,
                          layout=hsg.BATCHED, n_or=2, measure_every=1, seed=3, **kw)
        for s, L in enumerate(c["Ls"]):
            lat.set_couplings(s, gi.couplings(L, 3, s, precision="f16"))
            lat.set_spins_sample(s, gi.random_spins_batch(L, 3, s, lat.R))
        return lat

    alone = make_ctx(big, band_rows=8, fused_groups=2)
    alone.run_steps(2)
    ref = state(alone), alone.read_observables()[0].copy()
    alone.destroy()
    a = make_ctx(big, band_rows=8, fused_groups=2)     # the larger fused ring and measurement table
    b = make_ctx(small, band_rows=8, fused_groups=1)   # created after, needing less of both
    b.run_steps(2)
    a.run_steps(2)
    got = state(a), a.read_observables()[0].copy()
    assert all(np.array_equal(x, y) for rx, ry in zip(ref[0], got[0]) for x, y in zip(rx, ry))
    assert np.array_equal(ref[1], got[1])
    a.destroy()
    b.destroy()
