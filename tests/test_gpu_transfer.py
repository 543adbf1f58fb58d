"""Host <-> device transfers of the C ABI: the device-side packing of
couplings (storage order, FP16 rounding) and the whole-sample spin calls,
including transfers larger than one staging chunk (256 MiB)."""
import numpy as np
import pytest

import hsg_inputs as gi
import paper_1309_1599_b300 as hsg

pytestmark = pytest.mark.gpu


def _edge_values(n, rng):
    """FP32 values that exercise FP16 rounding: ties to even, the largest
    finite value, overflow to infinity, subnormals, signed zeros."""
    v = rng.standard_normal(n).astype(np.float32) * 4
    special = np.array([0.0, -0.0, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, -(1.0 + 2.0 ** -11),
                        65504.0, 65519.0, 65520.0, -1e6, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                        6.1e-5, 1e-8], dtype=np.float32)
    v[: special.size] = special
    return v


@pytest.mark.parametrize("L", [8, 160])
def test_f16_couplings_round_like_numpy(L):
    """set_couplings rounds FP32 to FP16 on the device, to nearest even, as
    numpy does; L = 160 spans two staging chunks."""
    rng = np.random.default_rng(L)
    N = L ** 3
    J6 = _edge_values(N * 18, rng).reshape(N, 3, 6)
    lat = hsg.Lattice([L], [1.0], n_replicas=1, coupling_prec=hsg.F16, layout=hsg.PLAIN)
    lat.set_couplings(0, J6)
    got = lat.get_couplings(0)
    with np.errstate(over="ignore"):               # 65520 and -1e6 round to +-inf
        want = J6.astype(np.float16).astype(np.float32)
    assert np.array_equal(got, want, equal_nan=True)
    assert np.array_equal(np.signbit(got), np.signbit(want))
    lat.destroy()


def test_f32_couplings_stored_exactly():
    rng = np.random.default_rng(3)
    L = 10
    J6 = rng.standard_normal((L ** 3, 3, 6)).astype(np.float32)
    lat = hsg.Lattice([L, 8], [1.0, 2.0], n_replicas=2, coupling_prec=hsg.F32, layout=hsg.BATCHED)
    lat.set_couplings(0, J6)
    assert np.array_equal(lat.get_couplings(0), J6)
    lat.destroy()


@pytest.mark.parametrize("layout", [hsg.PLAIN, hsg.BATCHED])
def test_sample_spin_calls_match_per_slot_calls(layout):
    Ls = [6, 8]
    lat = hsg.Lattice(Ls, [0.5, 1.0, 2.0, 3.0], n_replicas=2, coupling_prec=hsg.F16, layout=layout)
    for s, L in enumerate(Ls):
        lat.set_couplings(s, gi.couplings(L, 1, s, precision="f16"))
        block = np.stack([gi.random_spins(L, 1, s, j) for j in range(lat.R)])
        lat.set_spins_sample(s, block)
        for j in range(lat.R):
            assert np.array_equal(lat.get_spins(s, j), block[j])
        lat.set_spins(s, 3, gi.random_spins(L, 9, s, 3))
        block[3] = gi.random_spins(L, 9, s, 3)
        assert np.array_equal(lat.get_spins_sample(s), block)
    lat.destroy()


def test_sample_spin_calls_span_staging_chunks():
    """L = 64 with R = 96 lattices: 302 MB of spins, two staging chunks."""
    L, NT = 64, 48
    lat = hsg.Lattice([L], gi.linear_betas(0.2, 1.0, NT), n_replicas=2, coupling_prec=hsg.F16,
                      layout=hsg.BATCHED)
    rng = np.random.default_rng(5)
    block = rng.standard_normal((lat.R, L ** 3, 3)).astype(np.float32)
    lat.set_spins_sample(0, block)
    for j in (0, 47, 48, lat.R - 1):
        assert np.array_equal(lat.get_spins(0, j), block[j])
    out = lat.get_spins_sample(0)
    assert np.array_equal(out, block)
    lat.destroy()


def test_sample_spin_calls_reject_bad_arguments():
    lat = hsg.Lattice([8], [1.0], n_replicas=2)
    buf = np.zeros((2, 512, 3), np.float32)
    assert lat._lib.hsg_set_spins_sample(lat._h, 0, None) == 1          # HSG_EINVAL
    assert lat._lib.hsg_set_spins_sample(lat._h, 5, hsg._ptr(buf)) == 1
    assert lat._lib.hsg_get_spins_sample(lat._h, 0, None) == 1
    assert lat._lib.hsg_get_spins_sample(lat._h, -1, hsg._ptr(buf)) == 1
    lat.destroy()
