"""Pins of the oracle's single-spin updates, local field and energy against
closed forms, invariants and numerical quadrature (App. A.1, Eq. (1))."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle


def langevin(k):
    return 1.0 / np.tanh(k) - 1.0 / k


def _moments_u(k):
    """<u>, <u^2> for density ~ exp(k u) on [-1,1]."""
    Lk = langevin(k) if k > 1e-4 else k / 3.0
    u2 = 1.0 - 2.0 * Lk / k if k > 1e-4 else 1.0 / 3.0 + 2 * k * k / 45
    return Lk, u2


@pytest.mark.parametrize("kappa", [1e-6, 0.1, 1.0, 10.0, 100.0])
def test_hb_langevin_moments(kappa):
    rng = np.random.default_rng(int(kappa * 1000) + 1)
    h = rng.standard_normal(3)
    h *= 3.7 / np.linalg.norm(h)
    beta = kappa / 3.7
    n = 200_000
    s = oracle.hb_draw_batch(h, beta, seed=11, lattice=4, t=int(kappa * 10), n=n)
    hhat = h / np.linalg.norm(h)
    u = s @ hhat
    mu, u2 = _moments_u(kappa)
    var = u2 - mu * mu
    assert abs(u.mean() - mu) < 5 * np.sqrt(var / n)
    # second moment: variance of u^2 bounded by <u^4> <= <u^2>
    assert abs((u * u).mean() - u2) < 5 * np.sqrt(max(u2 - u2 * u2, 1e-12) / n) + 1e-12
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    # azimuth: isotropic around h, checked in a frame unrelated to the
    # construction used by the draw
    e = np.cross(hhat, rng.standard_normal(3))
    e /= np.linalg.norm(e)
    f = np.cross(hhat, e)
    a, b = s @ e, s @ f
    perp = (1.0 - u2) / 2.0
    assert abs(a.mean()) < 5 * np.sqrt(perp / n)
    assert abs(b.mean()) < 5 * np.sqrt(perp / n)
    assert abs((a * a).mean() - perp) < 5 * np.sqrt(2 * perp * perp / n) + 1e-9
    assert abs((a * b).mean()) < 5 * np.sqrt(perp * perp / n) + 1e-9
    # single-site Schwinger-Dyson identity (App. A.4.3): 2T<s.h> = h^2 - <(s.h)^2>
    sh = s @ h
    T = 1.0 / beta
    resid = 2 * T * sh - (h @ h - sh * sh)
    assert abs(resid.mean()) < 5 * resid.std() / np.sqrt(n)


def test_hb_zero_field_is_uniform():
    n = 100_000
    s = oracle.hb_draw_batch(np.zeros(3), 2.0, seed=5, lattice=0, t=0, n=n)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    assert np.all(np.abs(s.mean(axis=0)) < 5 * np.sqrt(1 / 3 / n))
    assert np.all(np.abs((s * s).mean(axis=0) - 1 / 3) < 5 * np.sqrt(4 / 45 / n))


def test_hb_small_kappa_branch_is_continuous():
    h = np.array([0.3, -0.2, 0.9])
    for w0, w1 in [(0x12345678, 0x9ABCDEF0), (0xFFFFFFFF, 1), (0, 0x80000000)]:
        a = oracle.hb_draw(h, 1e-31 / np.linalg.norm(h) * 0.5, w0, w1)   # kappa < 1e-30
        b = oracle.hb_draw(h, 1e-29 / np.linalg.norm(h), w0, w1)        # kappa > 1e-30
        assert np.allclose(a, b, atol=1e-12)


def _sphere_quadrature(n_theta=96, n_phi=192):
    x, w = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    pts = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    wts = (np.repeat(w, n_phi) * (2 * np.pi / n_phi))
    return pts, wts


@pytest.mark.parametrize("symmetric,beta", [(True, 0.7), (False, 0.7), (False, 2.5)])
def test_two_site_detailed_balance(symmetric, beta):
    """<s1^T J s2> of the heat-bath chain on two coupled spins equals
    d ln Z / d beta with Z = int ds2 4 pi sinh(beta |J s2|) / (beta |J s2|)
    (the s1 integral done exactly), integrated numerically over s2."""
    rng = np.random.default_rng(17 + int(beta * 10) + int(symmetric))
    J = rng.standard_normal((3, 3))
    if symmetric:
        J = (J + J.T) / 2
    pts, wts = _sphere_quadrature()
    a = np.linalg.norm(pts @ J.T, axis=1)      # |J s2|
    ba = beta * a
    z = np.sinh(ba) / ba
    dz = (np.cosh(ba) - np.sinh(ba) / ba) / beta
    exact = (wts @ dz) / (wts @ z)
    n = 400_000
    nb = 40
    means = []
    for b in range(nb):
        m, _ = oracle.two_site_chain(J, beta, seed=3, lattice=100 + b, n_skip=200,
                                     n_iter=n // nb)
        means.append(m)
    means = np.array(means)
    err = means.std(ddof=1) / np.sqrt(nb)
    assert abs(means.mean() - exact) < 5 * err, (means.mean(), exact, err)


def test_or_single_site_invariants():
    rng = np.random.default_rng(2)
    for _ in range(100):
        h = rng.standard_normal(3) * 4
        s = rng.standard_normal(3)
        s /= np.linalg.norm(s)
        s1 = oracle.or_update(h, s)
        assert abs(np.linalg.norm(s1) - 1) < 1e-14
        assert abs(s1 @ h - s @ h) < 1e-13
        assert np.allclose(oracle.or_update(h, s1), s, atol=1e-14)
    s = np.array([0.0, 0.6, 0.8])
    assert np.array_equal(oracle.or_update(np.zeros(3), s), s)


def _general_couplings(L, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((L ** 3, 3, 9))


def test_local_field_is_minus_energy_gradient():
    L = 4
    J9 = _general_couplings(L, 1)
    s = gi.random_spins(L, 3).astype(np.float64)
    d = 1e-6
    for i in [0, 5, 17, 63]:
        h = oracle.local_field(L, J9, s, i)
        g = np.zeros(3)
        for a in range(3):
            sp, sm = s.copy(), s.copy()
            sp[i, a] += d
            sm[i, a] -= d
            g[a] = -(oracle.energy(L, J9, sp) - oracle.energy(L, J9, sm)) / (2 * d)
        assert np.allclose(h, g, rtol=1e-7, atol=1e-7)


def test_or_sweeps_conserve_energy():
    L = 6
    J9 = oracle.j9_from_j6(gi.couplings(L, seed=1))
    s = gi.random_spins(L, 1).astype(np.float64)
    E0 = oracle.energy(L, J9, s)
    for _ in range(100):
        oracle.sweep(L, J9, s, oracle.OR)
    assert abs(oracle.energy(L, J9, s) - E0) < 1e-12 * abs(E0) * 100 ** 0.5
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-6)


def test_or_sweep_is_black_then_white():
    """Each overrelaxation half-sweep is an involution (fields of the other
    colour are fixed), so a full sweep -- black half, then white half -- is
    undone exactly by the white half followed by the black half."""
    L = 6
    J9 = oracle.j9_from_j6(gi.couplings(L, seed=5))
    s0 = gi.random_spins(L, 5).astype(np.float64)
    s = s0.copy()
    oracle.sweep(L, J9, s, oracle.OR)
    assert np.abs(s - s0).min() > 0 or np.abs(s - s0).max() > 1e-3
    colour = (np.arange(L ** 3) % L + (np.arange(L ** 3) // L) % L + np.arange(L ** 3) // L ** 2) % 2
    moved = np.linalg.norm(s - s0, axis=1) > 1e-9
    assert moved[colour == 0].mean() > 0.99 and moved[colour == 1].mean() > 0.99
    oracle.half_sweep(L, J9, s, 1, oracle.OR)
    oracle.half_sweep(L, J9, s, 0, oracle.OR)
    assert np.allclose(s, s0, atol=1e-12)


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_or_global_rotation_equivariance():
    L = 4
    rng = np.random.default_rng(9)
    J9 = oracle.j9_from_j6(gi.couplings(L, seed=2)).reshape(-1, 3, 3, 3)
    s = gi.random_spins(L, 2).astype(np.float64)
    R = _random_rotation(rng)
    Jr = np.einsum("ab,imbc,dc->imad", R, J9, R)
    sr = s @ R.T
    for _ in range(5):
        oracle.sweep(L, J9.reshape(-1, 3, 9), s, oracle.OR)
        oracle.sweep(L, Jr.reshape(-1, 3, 9), sr, oracle.OR)
    assert np.allclose(sr, s @ R.T, atol=1e-11)


def test_or_local_gauge_equivariance():
    """s_x -> R_x s_x, J_{x,mu} -> R_x J R_{x+mu}^T leaves Eq. (1) invariant;
    overrelaxation must map trajectories exactly.  The gauged couplings are
    not symmetric, so this pins which of J, J^T acts on each neighbour."""
    L = 4
    N = L ** 3
    rng = np.random.default_rng(10)
    J9 = oracle.j9_from_j6(gi.couplings(L, seed=3)).reshape(N, 3, 3, 3)
    s = gi.random_spins(L, 3).astype(np.float64)
    Rs = np.stack([_random_rotation(rng) for _ in range(N)])
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    idx = lambda x, y, z: (x % L) + L * ((y % L) + L * (z % L))
    Jg = np.empty_like(J9)
    for i in range(N):
        xi, yi, zi = i % L, (i // L) % L, i // (L * L)
        for mu, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
            j = idx(xi + dx, yi + dy, zi + dz)
            Jg[i, mu] = Rs[i] @ J9[i, mu] @ Rs[j].T
    sg = np.einsum("iab,ib->ia", Rs, s)
    E0 = oracle.energy(L, J9.reshape(N, 3, 9), s)
    assert abs(oracle.energy(L, Jg.reshape(N, 3, 9), sg) - E0) < 1e-11
    for _ in range(5):
        oracle.sweep(L, J9.reshape(N, 3, 9), s, oracle.OR)
        oracle.sweep(L, Jg.reshape(N, 3, 9), sg, oracle.OR)
    assert np.allclose(sg, np.einsum("iab,ib->ia", Rs, s), atol=1e-10)


def test_z2_time_reversal():
    """Sec. II.A: s -> -s is a symmetry; energies equal and overrelaxation
    commutes with the flip."""
    L = 4
    J9 = oracle.j9_from_j6(gi.couplings(L, seed=4))
    s = gi.random_spins(L, 4).astype(np.float64)
    m = -s
    assert abs(oracle.energy(L, J9, s) - oracle.energy(L, J9, m)) < 1e-12
    for _ in range(3):
        oracle.sweep(L, J9, s, oracle.OR)
        oracle.sweep(L, J9, m, oracle.OR)
    assert np.allclose(m, -s, atol=1e-12)


def test_ferromagnet_ground_state_and_low_T():
    L = 6
    N = L ** 3
    J9 = oracle.j9_from_j6(gi.ferromagnet(L))
    s = np.zeros((N, 3))
    s[:, 2] = 1.0
    assert oracle.energy(L, J9, s) == -3.0 * N
    # spin-wave equipartition at low T: <E>/N = -3 + T + O(T^2)
    T = 0.05
    es = []
    for t in range(600):
        oracle.sweep(L, J9, s, oracle.HB, 1 / T, seed=1, lattice=0, t=t)
        oracle.sweep(L, J9, s, oracle.OR)
        if t >= 100:
            es.append(oracle.energy(L, J9, s) / N)
    assert abs(np.mean(es) + 3 - T) < 0.1 * T


def test_neighbour_is_periodic_and_inverse():
    """The gather's index arithmetic: forward and backward steps undo each
    other, wrap at the faces, and move along x, y, z by 1, L, L^2."""
    L = 6
    rng = np.random.default_rng(4)
    for i in rng.integers(0, L ** 3, 200):
        for mu in range(3):
            up = oracle.neighbour(L, i, mu, +1)
            assert oracle.neighbour(L, up, mu, -1) == i
            c = [i % L, (i // L) % L, i // (L * L)]
            c[mu] = (c[mu] + 1) % L
            assert up == c[0] + L * (c[1] + L * c[2])
    assert oracle.neighbour(L, L - 1, 0, +1) == 0
    assert oracle.neighbour(L, 0, 2, -1) == (L - 1) * L * L


def test_site_field_from_gathered_data_is_minus_energy_gradient():
    """site_field on a site's own bonds and neighbours is -dE/ds_x (the
    energy is linear in one spin, so a unit step gives the derivative)."""
    L = 4
    rng = np.random.default_rng(8)
    J9 = rng.standard_normal((L ** 3, 3, 9))
    s = rng.standard_normal((L ** 3, 3))
    for i in (0, 5, 21, 63):
        Jup = np.stack([J9[i, mu] for mu in range(3)])
        Jdn = np.stack([J9[oracle.neighbour(L, i, mu, -1), mu] for mu in range(3)])
        s_up = np.stack([s[oracle.neighbour(L, i, mu, +1)] for mu in range(3)])
        s_dn = np.stack([s[oracle.neighbour(L, i, mu, -1)] for mu in range(3)])
        h = oracle.site_field(Jup, Jdn, s_up, s_dn)
        E0 = oracle.energy(L, J9, s)
        for a in range(3):
            t = s.copy()
            t[i, a] += 1.0
            assert abs(-(oracle.energy(L, J9, t) - E0) - h[a]) < 1e-9
