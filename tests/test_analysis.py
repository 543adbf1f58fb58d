"""The host analysis tail (Secs. II.B, III, V): pinned to closed forms and
compared with the oracle's loop-by-loop restatement."""
import math

import numpy as np
import pytest

import oracle.analysis as oa
from paper_1309_1599_b300 import analysis as an


# ---------------------------------------------------------------- pins
@pytest.mark.parametrize("L,m", [(8, 0.5), (16, 0.2), (64, 0.05)])
def test_xi_of_an_ornstein_zernike_propagator_is_its_inverse_mass(L, m):
    """chi(k) = 1 / (khat^2 + m^2) with khat = 2 sin(k/2): Eq. (4) gives
    xi = 1/m exactly on any L."""
    khat2 = (2 * math.sin(math.pi / L)) ** 2
    chi0, chik = 1 / m ** 2, 1 / (khat2 + m ** 2)
    assert an.xi_second_moment(chi0, chik, L) == pytest.approx(1 / m, rel=1e-12)
    assert math.isnan(an.xi_second_moment(1.0, 2.0, L))


def test_xi_of_a_lattice_field_from_its_fourier_sums():
    """A field q_x = sum over modes with an OZ spectrum: the Fourier sums of
    the field give back xi = 1/m within the spectrum's statistical error."""
    L, m = 16, 0.4
    rng = np.random.default_rng(5)
    k = 2 * np.pi * np.fft.fftfreq(L)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    khat2 = 4 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2 + np.sin(kz / 2) ** 2)
    chi0 = chik = 0.0
    for _ in range(3000):
        noise = rng.standard_normal((L, L, L)) + 1j * rng.standard_normal((L, L, L))
        q = np.fft.ifftn(noise / np.sqrt(khat2 + m * m)).real
        Q = np.fft.fftn(q) / L ** 3
        chi0 += L ** 3 * abs(Q[0, 0, 0]) ** 2
        chik += L ** 3 * (abs(Q[1, 0, 0]) ** 2 + abs(Q[0, 1, 0]) ** 2 + abs(Q[0, 0, 1]) ** 2) / 3
    assert an.xi_second_moment(chi0, chik, L) == pytest.approx(1 / m, rel=0.1)


def test_jackknife_of_the_mean_is_the_standard_error():
    x = np.random.default_rng(1).normal(size=(37, 3))
    est, err = an.jackknife(x)
    assert np.allclose(est, x.mean(0))
    assert np.allclose(err, x.std(0, ddof=1) / np.sqrt(len(x)))
    # a linear function scales the error
    est2, err2 = an.jackknife(x, lambda m: 3 * m[0] - m[1])
    assert err2 == pytest.approx(np.std(3 * x[:, 0] - x[:, 1], ddof=1) / np.sqrt(len(x)))


def test_log_bins_double_and_end_with_the_last_half():
    for n in (2, 16, 1024, 1000):
        bins = an.log_bins(n)
        assert bins[-1] == (n - n // 2, n)
        assert all(b[1] == c[0] for b, c in zip(bins, bins[1:]))          # contiguous
        if n & (n - 1) == 0:
            assert [b - a for a, b in bins] == [2 ** i for i in range(len(bins))]
            assert bins[0] == (1, 2)
    ramp = np.arange(16.0)
    assert np.allclose(an.bin_means(ramp), [1.0, 2.5, 5.5, 11.5])


def test_thermalization_test_on_a_relaxing_series():
    """O_n(t) = exp(-t/tau) + noise: the differences to the last bin decay to
    zero within their jackknife errors for late bins, not for early ones."""
    rng = np.random.default_rng(2)
    t = np.arange(4096)
    series = np.exp(-t / 40.0)[None, :] + 0.05 * rng.standard_normal((30, t.size))
    bins = np.stack([an.bin_means(s) for s in series])
    delta, err = an.thermalization_test(bins)
    assert delta[-1] == 0 and err[-1] == 0
    assert delta[0] > 10 * err[0]                 # first bins far from equilibrium
    assert np.all(np.abs(delta[-4:-1]) < 4 * err[-4:-1] + 1e-3)


def test_crossing_of_two_lines_is_exact():
    T = np.linspace(0.1, 0.9, 9)
    y1, y2 = 1.0 + 2.0 * (T - 0.43), 1.0 + 5.0 * (T - 0.43)
    tc, y, d1, d2 = an.crossing(T, y1, y2)
    assert tc == pytest.approx(0.43) and y == pytest.approx(1.0)
    assert d1 == pytest.approx(2.0) and d2 == pytest.approx(5.0)
    assert an.crossing(T, y1, y1 + 1) is None


@pytest.mark.parametrize("nu,eta,Tc", [(1.5, -0.2, 0.28), (2.4, 0.3, 0.17)])
def test_quotients_recover_exponents_of_exact_scaling(nu, eta, Tc):
    """Data with exact finite-size scaling and linear scaling functions,
    xi_L = L (a + b L^(1/nu) (T - Tc)), chi_L = L^(2-eta) (c + d L^(1/nu) (T - Tc)):
    the quotients give nu, eta and Tc exactly (Sec. V)."""
    T = np.linspace(Tc - 0.1, Tc + 0.1, 11)
    L = 8
    xi = {s: s * (0.6 - 0.9 * s ** (1 / nu) * (T - Tc)) for s in (L, 2 * L)}
    chi = {s: s ** (2 - eta) * (1.3 - 0.4 * s ** (1 / nu) * (T - Tc)) for s in (L, 2 * L)}
    r = an.quotients(T, xi[L], xi[2 * L], chi[L], chi[2 * L], L)
    assert r["T"] == pytest.approx(Tc, abs=1e-12)
    assert r["xi_over_L"] == pytest.approx(0.6)
    assert r["nu"] == pytest.approx(nu, rel=1e-9)
    assert r["eta"] == pytest.approx(eta, abs=1e-9)


def test_jackknife_quotients_on_noisy_scaling_samples():
    """Per-sample thermal means built from exact scaling plus sample noise:
    the jackknife estimates cover the true values."""
    nu, eta, Tc, L = 1.5, -0.2, 0.28, 8
    T = np.linspace(0.18, 0.38, 11)
    rng = np.random.default_rng(7)

    def means(s, n):
        xi = s * (0.6 - 0.9 * s ** (1 / nu) * (T - Tc))
        chi0 = s ** (2 - eta) * (1.3 - 0.4 * s ** (1 / nu) * (T - Tc))
        chik = chi0 / (1 + (2 * np.sin(np.pi / s) * xi) ** 2)     # Eq. (4) inverted
        N = s ** 3
        out = np.zeros((n, T.size, 9))
        out[..., an.Q2] = chi0 / N * (1 + 0.01 * rng.standard_normal((n, T.size)))
        out[..., an.Q2K] = chik / N * (1 + 0.01 * rng.standard_normal((n, T.size)))
        return out

    r = an.jackknife_quotients(T, means(L, 40), means(2 * L, 40), L)
    for key, true in (("T", Tc), ("nu", nu), ("eta", eta)):
        val, err = r[key]
        assert err > 0 and abs(val - true) < 4 * err + 1e-3, (key, val, err, true)


def test_observable_means_normalisation():
    obs = np.zeros((1, 2, 9))
    counts = np.array([[10, 5]])
    obs[0, 0, an.E] = 10 * 4 * -1.5          # 4 replicas: every lattice
    obs[0, 0, an.Q2] = 10 * 2 * 0.25         # 2 pairs
    obs[0, 1, an.SD] = 5 * 4 * 0.1
    m = an.observable_means(obs, counts, 4)
    assert m[0, 0, an.E] == pytest.approx(-1.5) and m[0, 0, an.Q2] == pytest.approx(0.25)
    assert m[0, 1, an.SD] == pytest.approx(0.1)


# ---------------------------------------------------------------- oracle parity
def test_package_matches_oracle_on_random_inputs():
    rng = np.random.default_rng(11)
    for L in (8, 12, 24):
        chi0, chik = rng.uniform(2, 5), rng.uniform(0.5, 2)
        assert an.xi_second_moment(chi0, chik, L) == pytest.approx(oa.xi(chi0, chik, L), rel=1e-13)
    x = rng.normal(size=(17, 4))
    f = lambda m: m[0] * m[1] - m[2] / (1 + m[3] ** 2)
    e1, s1 = an.jackknife(x, f)
    e2, s2 = oa.jackknife(x.tolist(), f)
    assert e1 == pytest.approx(e2, rel=1e-12) and s1 == pytest.approx(s2, rel=1e-10)
    for n in range(2, 300):
        assert an.log_bins(n) == oa.log_bins(n)
    for _ in range(20):
        T = np.sort(rng.uniform(0.1, 1.0, 12))
        tc = rng.uniform(0.3, 0.8)
        y1 = 1 + rng.uniform(1, 3) * (T - tc) + 0.01 * rng.standard_normal(12)
        y2 = 1 + rng.uniform(4, 6) * (T - tc) + 0.01 * rng.standard_normal(12)
        a, b = an.crossing(T, y1, y2), oa.linear_crossing(T, y1, y2)
        assert (a is None) == (b is None)
        if a is not None:
            assert np.allclose(a, b, rtol=1e-9, atol=1e-12)
    assert math.isclose(oa.quotient_nu(1.0, 2 ** (1 + 1 / 1.7)), 1.7)
    assert math.isclose(oa.quotient_eta(1.0, 2 ** (2 - 0.1)), 0.1)
