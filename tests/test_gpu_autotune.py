"""The autotuner times candidate launch shapes on a context's own data: it
must leave the state untouched, keep a valid plan, and (since the tiling
does not change the arithmetic) give the same trajectories as an untuned
context."""
import numpy as np
import pytest

import hsg_inputs as gi
import paper_1309_1599_b300 as hsg
from _gpu_helpers import make, state

pytestmark = pytest.mark.gpu


def _snapshot(lat):
    return state(lat), lat.get_perm().copy(), lat.get_counters().copy(), lat.get_launch_count()


@pytest.mark.parametrize("Ls,NT,persistent", [
    ([32, 40], 8, False),
    ([8, 12], 8, True),
    # one small lattice: a handful of CTAs, where the two-pass sweep can win
    ([16], 4, False),
    # mixed: the small bucket may switch to two-pass while L = 64 stays fused
    ([16, 64], 4, False),
    # resident steps on parts of replica sets (L = 16), PT between launches
    ([16], 8, True),
])
def test_autotune_keeps_state_and_trajectories(Ls, NT, persistent):
    betas = gi.linear_betas(0.3, 1.1, NT)
    kw = dict(n_rep=2, prec=hsg.F16, layout=hsg.BATCHED, n_or=3, measure_every=2, persistent=persistent)
    a, _ = make(Ls, betas, **kw)
    b, _ = make(Ls, betas, **kw)
    a.run_steps(2)
    b.run_steps(2)
    before = _snapshot(a)
    a.autotune()
    after = _snapshot(a)
    assert all(np.array_equal(x, y) for rx, ry in zip(before[0], after[0]) for x, y in zip(rx, ry))
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[2], after[2])
    assert before[3] == after[3]                       # tuning launches are not counted
    for s, L in enumerate(Ls):
        plan = a.get_sweep_plan(s)
        if plan["fused"]:
            assert L % plan["band_rows"] == 0
        if persistent:
            rp = a.get_resident_plan(s)
            assert rp["groups_per_item"] in (1, 2) and rp["threads"] % 32 == 0 and rp["threads"] >= 512
    a.run_steps(4)
    b.run_steps(4)
    assert all(np.array_equal(x, y) for rx, ry in zip(state(a), state(b)) for x, y in zip(rx, ry))
    assert np.array_equal(a.get_perm(), b.get_perm())
    assert np.array_equal(a.get_pt_accepts(), b.get_pt_accepts())
    Ea, Eb = a.get_energies(), b.get_energies()
    assert np.allclose(Ea, Eb, rtol=1e-9, atol=1e-9 * np.abs(Ea).max())
    oa, ob = a.read_observables()[0], b.read_observables()[0]
    assert np.allclose(oa, ob, rtol=1e-9, atol=1e-12)
    # a second context of the same shapes takes the remembered choices
    c, _ = make(Ls, betas, **kw)
    c.autotune()
    for s in range(len(Ls)):
        assert c.get_sweep_plan(s) == a.get_sweep_plan(s)
        assert c.get_resident_plan(s) == a.get_resident_plan(s)
    for lat in (a, b, c):
        lat.destroy()
