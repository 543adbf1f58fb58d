"""Pins of the oracle's parallel tempering (App. A.1) and observables
(Sec. II.B): exact acceptance rule, acceptance frequency, closed forms of the
overlap and chirality Fourier sums on constructed states, and a library FFT."""
import numpy as np
import pytest

import hsg_inputs as gi
import oracle


def test_pt_deterministic_cases():
    beta = np.array([0.5, 1.0, 2.0])
    # lattice 0 at beta 0.5 with lower energy than lattice 1 at beta 1.0:
    # delta = (0.5 - 1.0) * (-10 - 0) = +5 >= 0 -> always accepted.
    E = np.array([-10.0, 0.0, 1000.0])
    perm = np.array([0, 1, 2], dtype=np.int32)
    acc = np.zeros(2, dtype=np.int64)
    oracle.pt_sweep(beta, E, perm, seed=1, replica_set=0, t_pt=0, accepted=acc)
    # pair 0 swaps -> perm = [1, 0, 2]; pair 1 compares lattice 0 (now at
    # beta 1.0, E=-10) with lattice 2 (beta 2.0, E=1000):
    # delta = (1 - 2) * (-10 - 1000) = +1010 -> accepted -> [1, 2, 0].
    assert perm.tolist() == [1, 2, 0]
    assert acc.tolist() == [1, 1]
    # the reverse ordering has delta = -5 and -1010: exp(-1010) = 0 rejects
    perm = np.array([0, 1, 2], dtype=np.int32)
    E = np.array([0.0, -10.0, -2000.0])
    acc[:] = 0
    rejected = 0
    for t in range(200):
        p = perm.copy()
        oracle.pt_sweep(beta, E, p, seed=1, replica_set=0, t_pt=t, accepted=acc)
        if p[0] == 0:
            rejected += 1
    # exp(-5) = 0.0067: of 200 proposals, about 1.3 accepted
    assert rejected >= 190


def test_pt_acceptance_frequency():
    beta = np.array([1.0, 1.3])
    E = np.array([0.0, 2.0])        # delta = (1 - 1.3)(0 - 2) = 0.6 -> always
    E2 = np.array([2.0, 0.0])       # delta = -0.6 -> exp(-0.6) = 0.5488
    n = 20000
    acc = np.zeros(1, dtype=np.int64)
    for t in range(n):
        p = np.array([0, 1], dtype=np.int32)
        oracle.pt_sweep(beta, E2, p, seed=7, replica_set=3, t_pt=t, accepted=acc)
    pacc = np.exp(-0.6)
    assert abs(acc[0] / n - pacc) < 5 * np.sqrt(pacc * (1 - pacc) / n)
    acc[:] = 0
    for t in range(100):
        p = np.array([0, 1], dtype=np.int32)
        oracle.pt_sweep(beta, E, p, seed=7, replica_set=3, t_pt=t, accepted=acc)
    assert acc[0] == 100


def _coords(L):
    i = np.arange(L ** 3)
    return i % L, (i // L) % L, i // (L * L)


def test_overlap_uniform_state():
    L = 6
    s = np.tile(np.array([0.6, 0.0, 0.8]), (L ** 3, 1))
    Q0, Qk, C0, Ck = oracle.overlap_fourier(L, s, s)
    assert abs(Q0 - 1) < 1e-14
    assert np.abs(Qk).max() < 1e-14
    assert np.abs(C0).max() < 1e-14 and np.abs(Ck).max() < 1e-14
    m = oracle.measure_pair(L, s, s)
    assert np.allclose(m, [1, 1, 0, 0, 0, 0], atol=1e-14)


@pytest.mark.parametrize("nu", [0, 1, 2])
def test_overlap_cosine_modulation(nu):
    L = 8
    xc = _coords(L)[nu]
    th = 2 * np.pi * xc / L
    sa = np.tile([0.0, 0.0, 1.0], (L ** 3, 1))
    sb = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], axis=1)
    Q0, Qk, _, _ = oracle.overlap_fourier(L, sa, sb)
    # q_x = cos(2 pi x_nu / L): q(0) = 0, q(k_nu) = 1/2, other k vanish
    expect = np.zeros((3, 2))
    expect[nu, 0] = 0.5
    assert abs(Q0) < 1e-14
    assert np.allclose(Qk, expect, atol=1e-14)
    m = oracle.measure_pair(L, sa, sb)
    assert abs(m[2] - 0.25 / 3) < 1e-14


@pytest.mark.parametrize("axis,m,theta", [(0, 1, 0.7), (1, 2, 1.1), (2, 3, 2.0)])
def test_chirality_conical_spiral(axis, m, theta):
    """s_x = (sin t cos(k x_a), sin t sin(k x_a), cos t), k = 2 pi m / L:
    zeta_{x,a} = sin^2 t cos t (sin 2k - 2 sin k) on every site, and the
    chirality along the two other axes vanishes (repeated spins)."""
    L = 8
    k = 2 * np.pi * m / L
    xa = _coords(L)[axis]
    s = np.stack([np.sin(theta) * np.cos(k * xa), np.sin(theta) * np.sin(k * xa),
                  np.full(L ** 3, np.cos(theta))], axis=1)
    zeta = np.sin(theta) ** 2 * np.cos(theta) * (np.sin(2 * k) - 2 * np.sin(k))
    Q0, Qk, C0, Ck = oracle.overlap_fourier(L, s, s)
    expect = np.zeros(3)
    expect[axis] = zeta ** 2
    assert np.allclose(C0, expect, atol=1e-13)
    assert np.abs(Ck).max() < 1e-13
    assert abs(Q0 - 1) < 1e-13


def test_measure_pair_matches_library_fft():
    """The direct Fourier sums agree with numpy's FFT of the same fields:
    q(k) = sum_x q_x exp(+i k.x)/N is ifftn(q) at the lattice momentum."""
    L = 6
    sa = gi.random_spins(L, 5, 0, 0).astype(np.float64)
    sb = gi.random_spins(L, 5, 0, 1).astype(np.float64)
    Q0, Qk, C0, Ck = oracle.overlap_fourier(L, sa, sb)

    def grid(v):      # [N,3] -> [z,y,x,3]
        return v.reshape(L, L, L, 3)

    ga, gb = grid(sa), grid(sb)
    q = (ga * gb).sum(-1)
    Fq = np.fft.ifftn(q)
    ax = {0: 2, 1: 1, 2: 0}      # lattice direction -> array axis
    assert abs(Fq[0, 0, 0].real - Q0) < 1e-13
    for nu in range(3):
        idx = [0, 0, 0]
        idx[ax[nu]] = 1
        assert abs(Fq[tuple(idx)] - (Qk[nu, 0] + 1j * Qk[nu, 1])) < 1e-13
    for mu in range(3):
        def zeta(g):
            up = np.roll(g, -1, axis=ax[mu])
            dn = np.roll(g, +1, axis=ax[mu])
            return (up * np.cross(g, dn)).sum(-1)
        kap = zeta(ga) * zeta(gb)
        Fk = np.fft.ifftn(kap)
        assert abs(Fk[0, 0, 0].real - C0[mu]) < 1e-13
        for nu in range(3):
            idx = [0, 0, 0]
            idx[ax[nu]] = 1
            assert abs(Fk[tuple(idx)] - (Ck[mu, nu, 0] + 1j * Ck[mu, nu, 1])) < 1e-13


def _series_energy(L, J6, beta):
    """High-temperature expansion of <E> to O(beta^3) for couplings on the
    periodic cubic lattice (L >= 6), from the cumulant expansion of
    ln <exp(-beta H)> over independent uniform spins with
    <s_i s_j> = d_ij/3 and <s_i s_j s_k s_l> = (d d + d d + d d)/15."""
    N = L ** 3
    J = oracle.j9_from_j6(J6).reshape(N, 3, 3, 3)
    M = np.einsum("imab,imcb->imac", J, J)            # J J^T (= J^2, symmetric J)
    trM = np.trace(M, axis1=2, axis2=3)
    trM2 = np.einsum("imab,imba->im", M, M)
    m2 = trM / 9
    m4 = (trM ** 2 + 2 * trM2) / 75
    single = (beta * m2 + beta ** 3 * (m4 - 3 * m2 ** 2) / 6).sum()
    x, y, z = (np.arange(N) % L, (np.arange(N) // L) % L, np.arange(N) // (L * L))

    def nb(i, mu, sgn):
        c = [x[i], y[i], z[i]]
        c[mu] = (c[mu] + sgn) % L
        return c[0] + L * (c[1] + L * c[2])

    pair = 0.0
    plaq = 0.0
    for i in range(N):
        Ms = [M[i, mu] for mu in range(3)] + [M[nb(i, mu, -1), mu] for mu in range(3)]
        for a in range(6):
            for b in range(a + 1, 6):
                pair += 6 * np.trace(Ms[a] @ Ms[b]) - 2 * np.trace(Ms[a]) * np.trace(Ms[b])
        for mu in range(3):
            for nu in range(mu + 1, 3):
                J1 = J[i, mu]
                J2 = J[nb(i, mu, +1), nu]
                J3 = J[nb(i, nu, +1), mu]
                J4 = J[i, nu]
                plaq += np.trace(J1 @ J2 @ J3.T @ J4.T)
    return -single - beta ** 3 * pair / 405 - 4 * beta ** 3 * plaq / 81


@pytest.mark.parametrize("beta", [0.0, 0.25])
def test_energy_high_temperature_series(beta):
    L = 6
    N = L ** 3
    J6 = gi.couplings(L, seed=21)
    J9 = oracle.j9_from_j6(J6)
    s = gi.random_spins(L, 21).astype(np.float64)
    n_blocks, per_block = 40, 500
    means, var_sum = [], 0.0
    t = 0
    for b in range(n_blocks):
        es = []
        for _ in range(per_block):
            oracle.sweep(L, J9, s, oracle.HB, beta, seed=2, lattice=0, t=t)
            oracle.sweep(L, J9, s, oracle.OR)
            t += 1
            es.append(oracle.energy(L, J9, s))
        means.append(np.mean(es))
        var_sum += np.var(es)
    means = np.array(means)
    err = means.std(ddof=1) / np.sqrt(n_blocks)
    expect = _series_energy(L, J6, beta)
    assert abs(means.mean() - expect) < 5 * err, (means.mean(), expect, err)
    if beta == 0.0:
        # variance at beta = 0: sum over bonds of ||J_b||_F^2 / 9
        J = oracle.j9_from_j6(J6)
        assert abs(var_sum / n_blocks / ((J ** 2).sum() / 9) - 1) < 0.05
