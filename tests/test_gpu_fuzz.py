"""Seeded random configurations: the ways of running a Monte Carlo step
(fused one-pass sweeps, two-pass half-sweeps, shared-memory-resident steps,
and whatever shapes the autotuner picks)
must give the same spins bit for bit, the same temperature labels and
acceptances, and energies equal up to their summation order.  The draws
cover mixed L, odd replica counts, one temperature, beta = 0, both layouts
and all three coupling formats."""
import numpy as np
import pytest

import hsg_inputs as gi
import paper_1309_1599_b300 as hsg
from _gpu_helpers import state

pytestmark = pytest.mark.gpu


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    layout = hsg.BATCHED if rng.random() < 0.6 else hsg.PLAIN
    V = 2 if layout == hsg.BATCHED else 1
    n_L = int(rng.integers(1, 3))
    Ls = sorted({int(x) for x in rng.choice([4, 6, 8, 10, 12, 16], size=n_L)}, reverse=bool(rng.random() < 0.5))
    NT = int(rng.choice([1, 2, 3, 4, 6, 8]))
    if V == 2 and NT % 2:
        NT += 1
    n_rep = int(rng.integers(1, 4))
    if V == 2 and (NT * n_rep) % 2:
        n_rep += 1
    betas = np.sort(rng.uniform(0.0, 3.0, NT))
    if rng.random() < 0.3:
        betas[0] = 0.0
    betas = np.unique(betas)
    NT = len(betas)
    if V == 2 and NT % 2:
        betas = np.append(betas, betas[-1] + 0.5)
    prec = [hsg.F32, hsg.F16, hsg.BIMODAL][int(rng.integers(0, 3))]
    n_or = int(rng.integers(0, 4))
    me = int(rng.integers(0, 3))
    return dict(Ls=Ls, betas=list(betas), n_rep=n_rep, layout=layout, prec=prec, n_or=n_or, me=me)


def _make(c, **kw):
    lat = hsg.Lattice(c["Ls"], c["betas"], n_replicas=c["n_rep"], coupling_prec=c["prec"], layout=c["layout"],
                      n_or=c["n_or"], measure_every=c["me"], seed=7, bimodal_D=0.6, **kw)
    for s, L in enumerate(c["Ls"]):
        if c["prec"] == hsg.BIMODAL:
            lat.set_couplings_bimodal(s, gi.bimodal_bits(L, 7, s))
        else:
            lat.set_couplings(s, gi.couplings(L, 7, s, precision="f16" if c["prec"] == hsg.F16 else "f32"))
        lat.set_spins_sample(s, gi.random_spins_batch(L, 7, s, lat.R))
    return lat


def _result(lat, steps):
    lat.run_steps(steps)
    return state(lat), lat.get_perm().copy(), lat.get_pt_accepts().copy(), lat.get_energies().copy()


@pytest.mark.parametrize("seed", range(20))
def test_random_configurations_agree_across_step_kernels(seed):
    c = _config(seed)
    steps = 4
    tuned = _make(c)
    tuned.autotune()                        # may change band heights or leave the fused sweep
    runs = {"fused": _result(_make(c), steps),
            "two_pass": _result(_make(c, sweep_kernel=hsg.SWEEP_TWO_PASS), steps),
            "autotuned": _result(tuned, steps)}
    try:
        res = _make(c, persistent=True)
    except hsg.HsgError:
        res = None                          # a lattice group too large for shared memory
    if res is not None:
        runs["resident"] = _result(res, steps)
    if len(c["Ls"]) == 2:
        try:
            joint = _make(c, persistent=2)
        except hsg.HsgError:
            joint = None                    # replica sets that cannot be held whole
        if joint is not None:
            assert joint.get_resident_plan(0)["one_launch"]
            runs["joint"] = _result(joint, steps)
    ref = runs["fused"]
    for name, r in runs.items():
        assert all(np.array_equal(x, y) for rx, ry in zip(ref[0], r[0]) for x, y in zip(rx, ry)), (name, c)
        assert np.array_equal(ref[1], r[1]), (name, c)
        assert np.array_equal(ref[2], r[2]), (name, c)
        assert np.allclose(ref[3], r[3], rtol=1e-9, atol=1e-9 * max(1.0, np.abs(ref[3]).max())), (name, c)


def _bands(L):
    """Band heights the fused sweep accepts at L (divisors >= 8, and whole
    planes when L*L/2 threads fit in a block)."""
    out = [B for B in range(8, L) if L % B == 0 and (B + 2) * (L // 2) <= 576]
    if L * (L // 2) <= 576:
        out.append(L)
    return out


TILINGS = [(L, B) for L in (16, 20, 24, 28, 32, 40, 48, 56, 64) for B in _bands(L)]


@pytest.mark.parametrize("L,band", TILINGS, ids=[f"L{L}_b{B}" for L, B in TILINGS])
def test_every_fused_tiling_equals_the_two_pass_sweep(L, band):
    """Each band height the fused sweep accepts, including the compile-time
    specialisations (L = 32 and 64 in 8-row bands), gives the two-pass
    kernel's spins bit for bit over heat-bath and overrelaxation sweeps."""
    c = dict(Ls=[L], betas=[0.7, 1.9], n_rep=1, layout=hsg.BATCHED, prec=hsg.F16, n_or=2, me=0)
    a = _make(c, band_rows=band)
    plan = a.get_sweep_plan(0)
    assert plan["fused"] and plan["band_rows"] == band
    b = _make(c, sweep_kernel=hsg.SWEEP_TWO_PASS)
    ra, rb = _result(a, 2), _result(b, 2)
    assert all(np.array_equal(x, y) for rx, ry in zip(ra[0], rb[0]) for x, y in zip(rx, ry))
    assert np.array_equal(ra[1], rb[1])
    a.destroy()
    b.destroy()


def _ring_bytes(L, band, gp):
    """Shared memory of the fused sweep's ring with gp lattice groups of two
    lattices per element."""
    rows = L if band == L else band + 4
    return 4 * 3 * gp * rows * L * 2 * 4


TILINGS_GP2 = [(L, B) for L, B in TILINGS if _ring_bytes(L, B, 2) <= 200 * 1024
               and (L if B == L else B + 2) * (L // 2) <= 384]


GP2_CASES = [(L, B, hsg.F16) for L, B in TILINGS_GP2] + [(16, 16, hsg.F32), (64, 8, hsg.F32), (20, 20, hsg.BIMODAL),
                                                      (32, 8, hsg.BIMODAL)]


@pytest.mark.parametrize("L,band,prec", GP2_CASES,
                         ids=[f"L{L}_b{B}_p{p}" for L, B, p in GP2_CASES])
def test_two_groups_per_thread_equal_the_two_pass_sweep(L, band, prec):
    """Two lattice groups per thread (each coupling loaded and converted once
    for four lattices), at each band height whose ring fits: the two-pass
    kernel's spins bit for bit over heat-bath and overrelaxation sweeps, the
    same labels and acceptances, and the energies of one group per thread in
    the same bands exactly (the same partial sums in the same order)."""
    c = dict(Ls=[L, L], betas=[0.7, 1.9], n_rep=2, layout=hsg.BATCHED, prec=prec, n_or=2, me=0)
    a = _make(c, band_rows=band, fused_groups=2)
    plan = a.get_sweep_plan(0)
    assert plan["fused"] and plan["band_rows"] == band
    assert plan["groups_per_thread_or"] == 2 and plan["groups_per_thread_hb"] == 2
    b = _make(c, sweep_kernel=hsg.SWEEP_TWO_PASS)
    one = _make(c, band_rows=band, fused_groups=1)
    ra, rb, r1 = _result(a, 2), _result(b, 2), _result(one, 2)
    assert all(np.array_equal(x, y) for rx, ry in zip(ra[0], rb[0]) for x, y in zip(rx, ry))
    assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[2], rb[2])
    assert np.array_equal(ra[3], r1[3])
    for lat in (a, b, one):
        lat.destroy()


def test_two_groups_per_thread_needs_whole_group_pairs():
    """fused_groups = 2 with 2 lattices per sample, or the plain layout, is
    refused before anything is allocated."""
    with pytest.raises(hsg.HsgError, match="fused_groups"):
        hsg.Lattice(16, [0.5, 1.0], n_replicas=1, coupling_prec=hsg.F16, layout=hsg.BATCHED, fused_groups=2)
    with pytest.raises(hsg.HsgError, match="fused_groups"):
        hsg.Lattice(16, [0.5, 1.0], n_replicas=2, coupling_prec=hsg.F16, layout=hsg.PLAIN, fused_groups=2)


RESIDENT = [(L, layout, NT) for L in (4, 6, 8, 10, 12, 14, 16, 18, 20)
            for layout in (hsg.PLAIN, hsg.BATCHED) for NT in (2, 16)]


@pytest.mark.parametrize("L,layout,NT", RESIDENT,
                         ids=[f"L{L}_{'B' if lay else 'P'}_T{NT}" for L, lay, NT in RESIDENT])
def test_resident_steps_equal_streaming_steps_at_every_size(L, layout, NT):
    """Resident steps at every even L up to 20, one and two lattices per
    element, with replica sets that fit one CTA (N_T = 2) and, from L = 8
    or 10 on, sets split over several CTAs (N_T = 16), against the streaming
    path: same spins, labels and acceptances."""
    c = dict(Ls=[L], betas=list(gi.linear_betas(0.3, 1.5, NT)), n_rep=2, layout=layout, prec=hsg.F16,
             n_or=2, me=0)
    a = _make(c)
    b = _make(c, persistent=True)
    ra, rb = _result(a, 3), _result(b, 3)
    assert all(np.array_equal(x, y) for rx, ry in zip(ra[0], rb[0]) for x, y in zip(rx, ry))
    assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[2], rb[2])
    assert np.allclose(ra[3], rb[3], rtol=1e-9, atol=1e-9 * max(1.0, np.abs(ra[3]).max()))
    a.destroy()
    b.destroy()
