"""Pins of the oracle's counter-based generator and uniform mappings.

The paper's own generator (App. A.4.1) is replaced by Philox (Salmon et al.,
SC'11).  The oracle implements Philox4x32-10 and, with the same round
structure, Philox4x64-10.  The 64-bit member is checked bit for bit against
numpy's independent Philox4x64-10; the 32-bit member, which the Monte Carlo
uses, is checked with the tests App. A.4.3 names for generators: uniformity,
and a "horizontal" test across parallel streams.
"""
import numpy as np
import pytest
from scipy import stats

import oracle


def test_philox4x64_matches_numpy():
    rng = np.random.default_rng(7)
    for _ in range(64):
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        ctr = rng.integers(1, 2**64, size=4, dtype=np.uint64)
        ours = oracle.philox4x64(ctr, key)[0]
        # numpy's Philox increments its 256-bit counter before each block.
        prev = ctr.copy()
        prev[0] = prev[0] - np.uint64(1)
        ref = np.random.Philox(key=key, counter=prev).random_raw(4).astype(np.uint64)
        assert np.array_equal(ours, ref)


def _block(n, lattice=0, t=0, tag=1, seed=1):
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1] = lattice
    ctr[:, 2] = t
    ctr[:, 3] = tag
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    return oracle.philox4x32(ctr, key)


def test_philox4x32_uniform_bytes():
    out = _block(1 << 14)
    for w in range(4):
        counts = np.bincount((out[:, w] >> 24).astype(np.int64), minlength=256)
        p = stats.chisquare(counts).pvalue
        assert 1e-5 < p < 1 - 1e-5, (w, p)


def test_philox4x32_horizontal_streams():
    # First word of each of many streams (one per lattice id), as in the
    # "horizontal" test of App. A.4.3: uniform, and no correlation between
    # neighbouring streams.
    n = 4096
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(n)
    ctr[:, 3] = 1
    out = oracle.philox4x32(ctr, np.array([1, 0], dtype=np.uint32))
    u = (out[:, 0] >> 9).astype(np.float64) / 2**23
    assert stats.kstest(u, "uniform").pvalue > 1e-5
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(n)


def test_philox4x32_avalanche():
    rng = np.random.default_rng(3)
    flips = []
    key = np.array([0x1234, 0x5678], dtype=np.uint32)
    for _ in range(200):
        c = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        bit = rng.integers(0, 128)
        c2 = c.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        a = oracle.philox4x32(c, key)[0]
        b = oracle.philox4x32(c2, key)[0]
        flips.append(sum(bin(int(x ^ y)).count("1") for x, y in zip(a, b)))
    flips = np.array(flips)
    assert abs(flips.mean() - 64) < 5 * 4 / np.sqrt(len(flips)) + 0.5


def test_uniform23_exact_and_open():
    assert oracle.uniform23(0) == 2.0**-24
    assert oracle.uniform23(0xFFFFFFFF) == 1.0 - 2.0**-24
    for w in (0, 1 << 9, 0x80000000, 0xFFFFFFFF, 0x12345678):
        r = oracle.uniform23(w)
        assert np.float64(np.float32(r)) == r          # exact in binary32
        assert np.float64(np.float32(1.0 - r)) == 1.0 - r
        assert 0.0 < r < 1.0


def test_uniform52_exact_and_open():
    assert oracle.uniform52(0, 0) == 2.0**-53
    r = oracle.uniform52(0xFFFFFFFF, 0xFFFFFFFF)
    assert r == 1.0 - 2.0**-53 and r < 1.0


def test_hb_words_pairing():
    # Lattices 2m and 2m+1 share one Philox block: words (0,1) and (2,3).
    out = _block(1, lattice=3, t=5, seed=99)[0]
    assert oracle.hb_words(99, 0, 6, 5) == (int(out[0]), int(out[1]))
    assert oracle.hb_words(99, 0, 7, 5) == (int(out[2]), int(out[3]))
