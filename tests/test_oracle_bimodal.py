"""Pins of the oracle's bimodal couplings (Sec. II.A): J = +-1 and the six
independent entries D^ab (a >= b) of a symmetric anisotropy = +-D, one sign
bit each in a byte (bit 0: J; bits 1..6: D^xx, D^yy, D^zz, D^xy, D^xz, D^yz;
set = negative)."""
import itertools

import numpy as np
import pytest

import hsg_inputs as gi
import oracle

# matrix position of each anisotropy bit (symmetric: both triangles)
ENTRY = {1: [(0, 0)], 2: [(1, 1)], 3: [(2, 2)], 4: [(0, 1), (1, 0)], 5: [(0, 2), (2, 0)],
         6: [(1, 2), (2, 1)]}


@pytest.mark.parametrize("D", [0.5, 1.0])
def test_each_sign_bit_flips_its_entries(D):
    base = oracle.bimodal_j9(np.zeros((1, 1), np.uint8), D).reshape(3, 3)
    assert np.array_equal(base, np.full((3, 3), D) + np.eye(3))          # J = +1, all D = +D
    iso = oracle.bimodal_j9(np.array([[1]], np.uint8), D).reshape(3, 3)
    assert np.array_equal(iso, np.full((3, 3), D) - np.eye(3))           # J = -1
    for bit, cells in ENTRY.items():
        M = oracle.bimodal_j9(np.array([[1 << bit]], np.uint8), D).reshape(3, 3)
        want = base.copy()
        for (a, b) in cells:
            want[a, b] = (1.0 if a == b else 0.0) - D
        assert np.array_equal(M, want), bit


@pytest.mark.parametrize("D", [0.5, 1.0, 0.3])
def test_moments_of_the_law_over_all_bytes(D):
    """Uniform bytes realise the paper's moments: zero means, unit variance of
    the isotropic coupling, D^2 for every anisotropy entry, the isotropic
    part shared by the three diagonal entries, the entries otherwise
    independent."""
    M = oracle.bimodal_j9(np.arange(128, dtype=np.uint8).reshape(-1, 1), D).reshape(128, 3, 3)
    assert np.allclose(M, np.transpose(M, (0, 2, 1)))
    assert np.allclose(M.mean(0), 0.0, atol=1e-15)
    m2 = (M ** 2).mean(0)
    assert np.allclose(np.diag(m2), 1.0 + D * D)
    assert np.allclose(m2[np.triu_indices(3, 1)], D * D)
    assert np.isclose((M[:, 0, 0] * M[:, 1, 1]).mean(), 1.0)           # shared J
    assert np.isclose((M[:, 0, 1] * M[:, 0, 2]).mean(), 0.0)           # independent D
    iso = np.trace(M, axis1=1, axis2=2) / 3                            # J + sum D_aa / 3
    assert np.isclose((iso ** 2).mean(), 1.0 + D * D / 3)


def test_time_reversal_of_all_signs_negates_the_matrix():
    b = np.arange(128, dtype=np.uint8).reshape(-1, 1)
    assert np.array_equal(oracle.bimodal_j9(b ^ 0x7F, 0.5), -oracle.bimodal_j9(b, 0.5))


def test_isotropic_limit_energy_of_aligned_spins():
    """D = 0: J I on every bond, so aligned spins have E = -sum of the signs."""
    L = 4
    bits = gi.bimodal_bits(L, 3, 0)
    J9 = oracle.bimodal_j9(bits, 0.0)
    s = np.tile([0.0, 0.0, 1.0], (L ** 3, 1))
    signs = np.where(bits & 1, -1.0, 1.0)
    assert oracle.energy(L, J9, s) == pytest.approx(-signs.sum(), abs=1e-12)


def test_generator_bits_are_fair_and_bit7_clear():
    bits = gi.bimodal_bits(16, 1, 0)
    assert bits.dtype == np.uint8 and bits.shape == (16 ** 3, 3)
    assert not np.any(bits & 0x80)
    freq = [(bits >> k & 1).mean() for k in range(7)]
    assert np.allclose(freq, 0.5, atol=4 * 0.5 / np.sqrt(bits.size))
    assert not np.array_equal(gi.bimodal_bits(16, 1, 0), gi.bimodal_bits(16, 1, 1))
