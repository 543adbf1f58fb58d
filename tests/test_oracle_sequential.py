"""Pins of the oracle's sequential overrelaxation sweep (App. A.1): sites
visited one at a time in the natural order i = x + L (y + L z), each
reflected about the field of its neighbours' current values."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle


def _general_j9(L, seed):
    """Non-symmetric 3x3 bond matrices, so that J versus J^T matters."""
    return np.random.default_rng(seed).normal(size=(L ** 3, 3, 9))


def test_equals_the_site_by_site_composition_in_natural_order():
    L = 4
    J9 = _general_j9(L, 1)
    s0 = gi.random_spins(L, 1, 0).astype(np.float64)
    ref = s0.copy()
    for i in range(L ** 3):
        ref[i] = oracle.or_update(oracle.local_field(L, J9, ref, i), ref[i])
    got = s0.copy()
    oracle.sweep_sequential(L, J9, got)
    assert np.array_equal(got, ref)


def test_equals_the_hyperplane_wavefront_order():
    """Every neighbour visited before a site in natural order has a smaller
    x+y+z (periodic wraps included) and every later one a larger x+y+z, so
    updating the hyperplanes x+y+z = tau in increasing tau, sites of one
    hyperplane from the same state, is the same sweep."""
    L = 6
    J9 = _general_j9(L, 2)
    s0 = gi.random_spins(L, 2, 0).astype(np.float64)
    ref = s0.copy()
    idx = np.arange(L ** 3)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    for tau in range(3 * L - 2):
        plane = idx[x + y + z == tau]
        new = {i: oracle.or_update(oracle.local_field(L, J9, ref, i), ref[i]) for i in plane}
        for i, v in new.items():
            ref[i] = v
    got = s0.copy()
    oracle.sweep_sequential(L, J9, got)
    assert np.allclose(got, ref, rtol=0, atol=1e-13)


def test_conserves_energy_and_norms_and_differs_from_checkerboard():
    L = 8
    J9 = oracle.j9_from_j6(gi.couplings(L, 3, 0))
    s0 = gi.random_spins(L, 3, 0).astype(np.float64)
    s = s0.copy()
    for _ in range(5):
        oracle.sweep_sequential(L, J9, s)
    assert oracle.energy(L, J9, s) == pytest.approx(oracle.energy(L, J9, s0), abs=1e-9)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-12)
    cb = s0.copy()
    oracle.sweep(L, J9, cb, oracle.OR)
    one = s0.copy()
    oracle.sweep_sequential(L, J9, one)
    assert np.abs(one - cb).max() > 1e-3


def _reflect(L, s, J9):
    """Point reflection x -> L-1-x (all axes): site i -> N-1-i; the bond
    (i, i+mu) becomes the bond stored at the image of i+mu, transposed."""
    N = L ** 3
    idx = np.arange(N)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    img = (L - 1 - x) + L * ((L - 1 - y) + L * (L - 1 - z))
    s_r = np.empty_like(s)
    s_r[img] = s
    J_r = np.empty_like(J9)
    for mu, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        up = ((x + dx) % L) + L * (((y + dy) % L) + L * ((z + dz) % L))
        J_r[img[up], mu] = J9[idx, mu].reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9)
    return s_r, J_r, img


def test_sweep_on_the_reflected_lattice_undoes_the_sweep():
    """The reflection reverses the natural order, and a sequential
    overrelaxation sweep in reverse order is the inverse of the forward one
    (each reflection is an involution about a field that does not depend on
    the site itself)."""
    L = 6
    J9 = _general_j9(L, 4)
    s0 = gi.random_spins(L, 4, 0).astype(np.float64)
    s = s0.copy()
    oracle.sweep_sequential(L, J9, s)
    s_r, J_r, img = _reflect(L, s, J9)
    oracle.sweep_sequential(L, J_r, s_r)
    back = s_r[img]
    assert np.allclose(back, s0, atol=1e-10)
    assert np.abs(s - s0).max() > 1e-2           # the sweep did change the state
