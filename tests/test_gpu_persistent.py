"""Shared-memory-resident steps (the whole Monte Carlo step of Sec. III in one
launch per stretch of steps) against the streaming path and the oracle."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import SWEEP_TOL, compare_sweep, make, state, temp_of

pytestmark = pytest.mark.gpu

CASES = [
    # Ls, n_temps, n_rep, prec, layout, n_or, measure_every, steps
    ([8, 12], 8, 2, hsg.F16, hsg.BATCHED, 3, 2, 6),
    ([12, 8, 8], 4, 3, hsg.F32, hsg.PLAIN, 8, 3, 7),
    ([10], 6, 2, hsg.F32, hsg.BATCHED, 2, 0, 5),
    ([8], 1, 2, hsg.F16, hsg.PLAIN, 1, 1, 3),
    # L=12 with FP32 bonds: the bonds stay in global memory (spins 166 KB)
    ([12, 8], 8, 2, hsg.F32, hsg.BATCHED, 2, 2, 4),
    # heat-bath only: the energies come from the white heat-bath half-sweep
    ([8, 12], 4, 2, hsg.F16, hsg.BATCHED, 0, 2, 4),
    # three lattice groups per replica set: one group per work item
    ([8, 12], 6, 2, hsg.F16, hsg.BATCHED, 2, 2, 4),
    # replica sets larger than shared memory: parts of a set per CTA, one
    # step per launch, PT as its own kernel
    ([16], 8, 2, hsg.F16, hsg.BATCHED, 3, 2, 5),
    ([20], 4, 2, hsg.F32, hsg.PLAIN, 2, 2, 4),
    # mixed: L = 8 sets would fit whole, but L = 16 makes every step split
    ([16, 8], 4, 2, hsg.F16, hsg.BATCHED, 2, 2, 4),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{'-'.join(map(str, c[0]))}_T{c[1]}")
def test_persistent_steps_equal_streaming_steps(case):
    """Same spins bit for bit, same labels and acceptances, energies and
    observables equal up to the summation order of the energies."""
    Ls, NT, n_rep, prec, layout, n_or, me, steps = case
    betas = gi.linear_betas(0.2, 1.2, NT)
    a, _ = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout, n_or=n_or, measure_every=me)
    b, _ = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout, n_or=n_or, measure_every=me,
                persistent=True)
    a.run_steps(steps - 2)
    a.run_steps(2)
    b.run_steps(steps - 2)
    b.run_steps(2)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    assert np.array_equal(a.get_pt_accepts(), b.get_pt_accepts())
    assert np.array_equal(a.get_counters(), b.get_counters())
    Ea, Eb = a.get_energies(), b.get_energies()
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-9 * np.abs(Ea).max()), np.abs(Ea - Eb).max()
    oa, ca = a.read_observables()
    ob, cb = b.read_observables()
    assert np.array_equal(ca, cb)
    if me:
        assert ca.min() == steps // me
    assert np.allclose(oa, ob, rtol=1e-9, atol=1e-12)
    # one launch per stretch of steps between measurements (+ counter bump)
    assert b.get_launch_count() < a.get_launch_count()


JOINT = [
    # Ls, n_temps, n_rep, prec, layout, steps: the L = 12 with L = 8
    # specialisation (L = 8 CTAs holding 4, 2 sets; FP16 and FP32 bonds) and
    # the generic joint kernel (other sizes, bonds from global memory)
    ([12, 8, 8, 12], 8, 4, hsg.F16, hsg.BATCHED, 5),
    ([8, 12], 8, 2, hsg.F16, hsg.BATCHED, 4),
    ([8, 12], 4, 2, hsg.F32, hsg.BATCHED, 4),
    ([6, 10, 6], 4, 2, hsg.F16, hsg.PLAIN, 4),
    ([10, 4], 6, 3, hsg.F32, hsg.BATCHED, 4),
    # L = 12 with FP32 bonds and 8 temperatures: too large for the
    # specialisation's resident bonds, so the generic joint kernel takes it
    ([12, 8], 8, 2, hsg.F32, hsg.BATCHED, 4),
]


@pytest.mark.parametrize("case", JOINT, ids=lambda c: f"L{'-'.join(map(str, c[0]))}_T{c[1]}_R{c[2]}")
def test_joint_launch_of_two_lattice_sizes_equals_streaming(case):
    """persistent = 2: the resident steps of both lattice sizes in one launch
    per stretch of steps (CTAs of the smaller size holding several whole
    replica sets of one sample) give the streaming path's spins bit for bit,
    the same labels, acceptances and counters, and energies and observables
    equal up to the summation order of the energies; one resident launch per
    stretch instead of one per lattice size."""
    Ls, NT, n_rep, prec, layout, steps = case
    betas = gi.linear_betas(0.2, 1.2, NT)
    a, _ = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout, n_or=2, measure_every=2)
    b, _ = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout, n_or=2, measure_every=2, persistent=2)
    c, _ = make(Ls, betas, n_rep=n_rep, prec=prec, layout=layout, n_or=2, measure_every=2, persistent=1)
    small = Ls.index(min(Ls))
    plan = b.get_resident_plan(small)
    assert plan["one_launch"] and plan["sets_per_cta"] >= 1
    assert not c.get_resident_plan(small)["one_launch"]
    n = []
    for lat in (a, b, c):
        l0 = lat.get_launch_count()
        lat.run_steps(steps)
        n.append(lat.get_launch_count() - l0)
    stretches = (steps + 1) // 2
    assert n[1] == n[2] - stretches, n           # one resident launch instead of two per stretch
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    assert np.array_equal(a.get_pt_accepts(), b.get_pt_accepts())
    assert np.array_equal(a.get_counters(), b.get_counters())
    Ea, Eb = a.get_energies(), b.get_energies()
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-9 * np.abs(Ea).max()), np.abs(Ea - Eb).max()
    oa, ca = a.read_observables()
    ob, cb = b.read_observables()
    assert np.array_equal(ca, cb)
    assert np.allclose(oa, ob, rtol=1e-9, atol=1e-12)
    for lat in (a, b, c):
        lat.destroy()


def test_joint_launch_refused_when_sets_cannot_be_held_whole():
    """persistent = 2 needs every replica set held whole by one CTA: L = 16
    with 8 temperatures splits its sets (393 KB), so the context is refused;
    so is a context with three lattice sizes."""
    with pytest.raises(hsg.HsgError, match="whole"):
        hsg.Lattice([16, 8], gi.linear_betas(0.2, 1.2, 8), n_replicas=2, coupling_prec=hsg.F16,
                    layout=hsg.BATCHED, persistent=2)
    with pytest.raises(hsg.HsgError, match="two lattice sizes"):
        hsg.Lattice([4, 6, 8], gi.linear_betas(0.2, 1.2, 2), n_replicas=2, coupling_prec=hsg.F16,
                    layout=hsg.BATCHED, persistent=2)


@pytest.mark.parametrize("Ls,prec,layout,persistent", [([8, 12], hsg.F16, hsg.BATCHED, 1),
                                                      ([12, 8], hsg.F32, hsg.BATCHED, 2),
                                                      ([8], hsg.F32, hsg.PLAIN, 1)])
def test_resident_step_matches_oracle_per_half_sweep(Ls, prec, layout, persistent):
    """The resident kernel checked against the oracle directly, not through
    the streaming path: one resident step of heat-bath sweeps only
    (n_or = 0), per half-sweep from the GPU's state before the step (every
    site within 2e-5; frame-ambiguous sites on u and the norm), then the
    labels the kernel's in-kernel PT sweep left against the oracle's PT
    sweep on the kernel's energies, and those energies against the oracle's
    energy of the new spins."""
    betas = gi.linear_betas(0.4, 1.5, 4)
    lat, J = make(Ls, betas, n_rep=2, prec=prec, layout=layout, n_or=0, measure_every=0, persistent=persistent)
    lat.run_steps(20)                            # away from the initial state
    before, tmp, perm0 = state(lat), temp_of(lat), lat.get_perm().copy()
    hb_t, pt_t, _ = (int(x) for x in lat.get_counters())
    lat.run_steps(1)
    after = state(lat)
    worst, n_amb, worst_u = compare_sweep(lat, J, before, after, oracle.HB, hb_t, tmp=tmp)
    assert worst <= SWEEP_TOL and worst_u <= SWEEP_TOL, (worst, worst_u)
    assert n_amb <= 1e-3 * sum(L ** 3 for L in Ls) * lat.R + 6
    E = lat.get_energies()
    for s, L in enumerate(Ls):
        J9 = oracle.j9_from_j6(J[s])
        for slot in range(lat.R):
            ref = oracle.energy(L, J9, after[s][slot])
            assert abs(E[s, slot] - ref) <= 2e-6 * abs(ref), (s, slot, E[s, slot], ref)
        for r in range(lat.n_replicas):
            p = perm0[s, r].copy()
            oracle.pt_sweep(betas, E[s], p, lat.seed, s * lat.n_replicas + r, pt_t)
            assert np.array_equal(lat.get_perm()[s, r], p), (s, r)


def test_persistent_step_matches_oracle_step_from_equilibrium():
    """One whole step (HB + 8 OR + energies + PT) of the resident kernel from
    an equilibrated state (overrelaxation amplifies rounding differences less
    there): labels identical to the oracle's, spins within the per-sweep
    tolerance accumulated over the step's 9 sweeps, energies of the final
    state to FP32 summation accuracy."""
    betas = gi.linear_betas(0.5, 1.0, 4)
    lat, J = make([8], betas, n_rep=2, prec=hsg.F32, layout=hsg.BATCHED, persistent=True)
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
    E = lat.get_energies()[0]
    for j in range(lat.R):
        ref = oracle.energy(8, oracle.j9_from_j6(J[0]), lat.get_spins(0, j).astype(np.float64))
        assert abs(E[j] - ref) <= 2e-6 * abs(ref)


@pytest.mark.parametrize("name,mode", [("L8x256_L12x256_R32_f16", 1), ("L8x256_L12x256_R32_f16", 2),
                                       ("L16_S512_R32_f16", 1)])
def test_bench_resident_workloads_equal_streaming(name, mode):
    """The resident workloads at the size and launch configuration bench.py
    times, with shapes chosen by the autotuner: the mixed small lattices (256
    samples of L=8 and 256 of L=12, 4 replicas x 8 temperatures; whole
    replica sets per CTA, PT in the kernel) and the mid-size lattices (512
    samples of L=16, 2 replicas x 16 temperatures; parts of replica sets per
    CTA, PT as its own kernel), FP16 couplings, two lattices per element.
    One bench step of 10 MCS with resident launches equals the streaming
    kernels on every lattice bit for bit, with the same labels, acceptances
    and counters, and energies and observables equal up to their summation
    order.  Mode 2 runs both lattice sizes of the mixed workload in one
    resident launch per step (one launch fewer than mode 1)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w = bench.WORKLOADS[name]
    samples, J, spins, beta = bench.make_inputs(w, 0)
    modes = (False, mode, 1) if mode == 2 else (False, mode)
    lats = [bench.build_lattice(hsg, w, samples, J, spins, beta, hsg.F16, hsg.BATCHED, persistent=p)
            for p in modes]
    del spins
    launches = []
    for lat in lats:
        l0 = lat.get_launch_count()
        lat.run_steps(bench.MCS_PER_STEP)
        launches.append(lat.get_launch_count() - l0)
    a, b = lats[0], lats[1]
    assert launches[1] < launches[0], launches
    if mode == 2:
        assert launches[1] == launches[2] - 1, launches
        assert b.get_resident_plan(0)["one_launch"]
    for s in range(a.S):
        assert np.array_equal(a.get_spins_sample(s), b.get_spins_sample(s)), s
    assert np.array_equal(a.get_perm(), b.get_perm())
    assert np.array_equal(a.get_pt_accepts(), b.get_pt_accepts())
    assert np.array_equal(a.get_counters(), b.get_counters())
    Ea, Eb = a.get_energies(), b.get_energies()
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-9 * np.abs(Ea).max())
    oa, ca = a.read_observables()
    ob, cb = b.read_observables()
    assert np.array_equal(ca, cb) and ca.min() == 1
    assert np.allclose(oa, ob, rtol=1e-9, atol=1e-12)
    for lat in lats:
        lat.destroy()
