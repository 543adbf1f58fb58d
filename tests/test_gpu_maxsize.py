"""The largest lattice the library accepts, L = 512 (134 M sites): one
heat-bath and one overrelaxation sweep (the two-pass half-sweep kernel, which
serves every L the fused sweep's tiles do not fit) checked against the oracle
per half-sweep on sampled sites.  Bimodal one-byte couplings keep the host
copies small (402 MB of bonds, 1.6 GB per spin array)."""
import numpy as np
import pytest

import oracle
import paper_1309_1599_b300 as hsg
from _gpu_helpers import frame_ambiguous_diff

pytestmark = pytest.mark.gpu

L = 512
D = 0.7
SEED = 11
TOL = 2e-5          # per half-sweep, as in the other parity tests
N_SAMPLED = 3000


def _site_update(i, bits, nb_state, own_state, kind, beta, lattice, t):
    """The oracle's update of site i from the neighbour spins in nb_state."""
    ups = [oracle.neighbour(L, i, mu, +1) for mu in range(3)]
    dns = [oracle.neighbour(L, i, mu, -1) for mu in range(3)]
    Jup = oracle.bimodal_j9(bits[i], D).reshape(3, 9)
    Jdn = np.stack([oracle.bimodal_j9(bits[dns[mu], mu:mu + 1], D)[0] for mu in range(3)])
    s_up = nb_state[ups].astype(np.float64)
    s_dn = nb_state[dns].astype(np.float64)
    h = oracle.site_field(Jup, Jdn, s_up, s_dn)
    if kind == oracle.OR:
        return oracle.or_update(h, own_state[i].astype(np.float64)), h
    w0, w1 = oracle.hb_words(SEED, i, lattice, t)
    return oracle.hb_draw(h, beta, w0, w1), h


@pytest.mark.parametrize("kind", [oracle.OR, oracle.HB])
def test_largest_lattice_sampled_half_sweep_parity(kind):
    N = L ** 3
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 128, size=(N, 3), dtype=np.uint8)
    s0 = rng.standard_normal((N, 3)).astype(np.float32)
    s0 /= np.linalg.norm(s0, axis=1, keepdims=True)
    beta = 1.7
    lat = hsg.Lattice([L], [beta], n_replicas=1, coupling_prec=hsg.BIMODAL, layout=hsg.PLAIN,
                      n_or=1, measure_every=0, seed=SEED, bimodal_D=D)
    assert not lat.get_sweep_plan(0)["fused"]
    lat.set_couplings_bimodal(0, bits)
    lat.set_spins(0, 0, s0)
    t = int(lat.get_counters()[0])
    (lat.sweep_hb if kind == oracle.HB else lat.sweep_or)(1)
    s1 = lat.get_spins(0, 0)
    lat.destroy()

    # sampled sites of both colours, including the lattice's corners
    sites = np.concatenate([[0, L - 1, N - 1, N - L, L * L - 1], rng.integers(0, N, N_SAMPLED)])
    colour = (sites % L + (sites // L) % L + sites // (L * L)) % 2
    worst, n_amb = 0.0, 0
    for i, c in zip(sites, colour):
        # black sites see the old white spins; white sites the new black ones
        nb_state = s0 if c == 0 else s1
        ref, h = _site_update(int(i), bits, nb_state, s0, kind, beta, 0, t)
        if kind == oracle.HB and abs(h[2]) < 1e-4 * np.linalg.norm(h):
            n_amb += 1               # frame-ambiguous (field at the equator): either frame
            d = frame_ambiguous_diff(s1[i][None].astype(np.float64), ref[None], h[None])[0]
            worst = max(worst, float(d))
            continue
        worst = max(worst, float(np.abs(s1[i] - ref).max()))
    assert n_amb <= 3
    assert worst <= TOL, worst
