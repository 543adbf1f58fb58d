"""Sequential overrelaxation sweeps (App. A.1) on the GPU -- executed by
hyperplanes x+y+z = tau -- against the oracle's site-by-site sweep."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import make, state

pytestmark = pytest.mark.gpu

CASES = [
    # Ls, n_rep, prec, layout, equilibrate first
    ([8], 2, hsg.F32, hsg.PLAIN, False),
    ([8], 2, hsg.F32, hsg.PLAIN, True),
    ([12, 8], 2, hsg.F16, hsg.BATCHED, True),
    ([16], 1, hsg.F16, hsg.BATCHED, True),
    ([6, 10], 3, hsg.F32, hsg.PLAIN, False),
]


def _per_site_parity(L, J9, before, after):
    """Largest |ds| between the GPU's update of each site and the oracle's
    update of that site from the same inputs: the neighbours visited earlier
    in the natural order (index < i) at their new GPU values, the later ones
    at their old values, and the site's own old value.  (A whole sweep is a
    chain of 3L-2 dependent hyperplanes, along which overrelaxation amplifies
    the binary32 rounding, as it does from sweep to sweep.)"""
    worst = 0.0
    mixed = before.copy()
    for i in range(L ** 3):
        h = oracle.local_field(L, J9, mixed, i)
        ref = oracle.or_update(h, before[i])
        worst = max(worst, float(np.abs(after[i] - ref).max()))
        mixed[i] = after[i]
    return worst


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sequential_sweep_matches_oracle_site_by_site(case):
    Ls, n_rep, prec, layout, equil = CASES[case]
    betas = gi.linear_betas(0.5, 1.5, 2)
    lat, J = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout)
    if equil:
        lat.run_steps(50)
    before = state(lat)
    lat.sweep_or_sequential(1)
    after = state(lat)
    worst_site, worst_sweep = 0.0, 0.0
    for s, L in enumerate(Ls):
        J9 = oracle.j9_from_j6(J[s])
        for slot in range(lat.R):
            worst_site = max(worst_site, _per_site_parity(L, J9, before[s][slot], after[s][slot]))
            ref = before[s][slot].copy()
            oracle.sweep_sequential(L, J9, ref)
            worst_sweep = max(worst_sweep, float(np.abs(after[s][slot] - ref).max()))
    assert 0 < worst_site <= 2e-5, worst_site
    assert worst_sweep <= 2e-3, worst_sweep        # the whole wave, rounding amplified


def test_bimodal_sequential_sweeps_conserve_energy():
    L, D = 8, 0.5
    lat = hsg.Lattice([L, L], [1.0, 2.0], n_replicas=2, coupling_prec=hsg.BIMODAL, layout=hsg.BATCHED,
                      bimodal_D=D, seed=4)
    J9 = []
    for s in range(2):
        bits = gi.bimodal_bits(L, 4, s)
        lat.set_couplings_bimodal(s, bits)
        J9.append(oracle.bimodal_j9(bits, D))
        for j in range(lat.R):
            lat.set_spins(s, j, gi.random_spins(L, 4, s, j))
    E0 = lat.get_energies()
    before = state(lat)
    lat.sweep_or_sequential(1)
    after = state(lat)
    assert _per_site_parity(L, J9[1], before[1][3], after[1][3]) <= 2e-5
    lat.sweep_or_sequential(9)
    E1 = lat.get_energies()                    # recomputed: the sweeps made them stale
    assert np.allclose(E1, E0, rtol=1e-4, atol=1e-3)
    assert np.abs(np.linalg.norm(state(lat)[0][0], axis=1) - 1).max() < 1e-5


def test_lattices_too_large_for_shared_memory_are_refused():
    lat, _ = make([32], [1.0], n_rep=2, prec=hsg.F16, layout=hsg.BATCHED)
    before = state(lat)
    with pytest.raises(hsg.HsgError):
        lat.sweep_or_sequential(1)
    assert all(np.array_equal(x, y) for rx, ry in zip(before, state(lat)) for x, y in zip(rx, ry))


def test_bench_small_lattice_workload_sampled_site_parity():
    """The sequential sweep at the size and configuration bench.py times it
    (the mixed small-lattice workload: 256 samples of L=8 and 256 of L=12, 32
    lattices each, FP16 couplings, two lattices per element): per-site parity
    with the oracle on sampled lattices of both sizes, and the whole-sweep
    drift bound."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w = bench.WORKLOADS["L8x256_L12x256_R32_f16"]
    samples, J, spins, beta = bench.make_inputs(w, 0)
    lat = bench.build_lattice(hsg, w, samples, J, spins, beta, hsg.F16, hsg.BATCHED)
    del spins
    sampled = [(0, 0), (0, 1), (255, 31), (256, 0), (300, 17), (511, 31)]
    before = {sl: lat.get_spins(*sl).astype(np.float64) for sl in sampled}
    lat.sweep_or_sequential(1)
    for (s, slot) in sampled:
        L = lat.Ls[s]
        J9 = oracle.j9_from_j6(J[s])
        after = lat.get_spins(s, slot).astype(np.float64)
        worst = _per_site_parity(L, J9, before[(s, slot)], after)
        assert 0 < worst <= 2e-5, ((s, slot), worst)
        ref = before[(s, slot)].copy()
        oracle.sweep_sequential(L, J9, ref)
        assert np.abs(after - ref).max() <= 2e-3
    lat.destroy()
