"""Analysis of the accumulated observables on the host (Secs. II.B, III, V).

The Monte Carlo itself runs in libhsg; what it returns per (sample,
temperature) are sums of observables over measurements.  This module turns
them into the paper's quantities:

  * thermal means of the observables (``observable_means``);
  * susceptibilities chi_SG(k), chi_CG(k) (Sec. II.B) and the second-moment
    correlation length xi of Eq. (4) (``susceptibilities``,
    ``xi_second_moment``);
  * disorder averages with jackknife errors over samples (``jackknife``);
  * logarithmic data binning and the thermalization test of Sec. III
    (``log_bins``, ``run_log_binned``, ``thermalization_test``);
  * the crossing temperature of xi_L/L and xi_2L/2L from low-order fits over
    the four nearest temperatures, and the quotients method for nu and eta
    (Sec. V, Eqs. for nu and eta) (``crossing``, ``quotients``), with
    jackknife errors over samples (``jackknife_quotients``).

Observable order (as libhsg accumulates them): 0 e, 1 e^2, 2 q^2, 3 q^4,
4 |q(k_min)|^2, 5 q_CG^2, 6 q_CG^4, 7 |q_CG(k_min)|^2, 8 Schwinger-Dyson.
"""
from __future__ import annotations

import math
from typing import Callable, Sequence

import numpy as np

E, E2, Q2, Q4, Q2K, C2, C4, C2K, SD = range(9)


# ---------------------------------------------------------------------------
# Thermal means, susceptibilities, correlation length
# ---------------------------------------------------------------------------
def observable_means(obs: np.ndarray, counts: np.ndarray, n_replicas: int) -> np.ndarray:
    """Thermal means <O> from libhsg's accumulated sums.

    obs [..., 9] and counts [...] as read by ``Lattice.read_observables``.
    e, e^2 and the Schwinger-Dyson residual are summed over every lattice at
    the temperature (n_replicas per measurement); the overlaps over the
    replica pairs (n_replicas // 2 per measurement)."""
    obs = np.asarray(obs, dtype=np.float64)
    n = np.asarray(counts, dtype=np.float64)[..., None]
    if n_replicas < 2:
        raise ValueError("overlaps need at least two replicas")
    m = np.empty_like(obs)
    m[..., [E, E2, SD]] = obs[..., [E, E2, SD]] / (n * n_replicas)
    m[..., Q2:SD] = obs[..., Q2:SD] / (n * (n_replicas // 2))
    return m


def susceptibilities(means: np.ndarray, N: int) -> dict:
    """chi = N <|q(k)|^2> at k = 0 and k = k_min for the spin-glass and the
    chiral-glass overlaps (Sec. II.B); |q(k_min)|^2 is averaged over the
    three directions of k_min, the chiral one also over mu."""
    means = np.asarray(means, dtype=np.float64)
    return {"sg0": N * means[..., Q2], "sgk": N * means[..., Q2K],
            "cg0": N * means[..., C2], "cgk": N * means[..., C2K]}


def xi_second_moment(chi0, chik, L: int):
    """Second-moment correlation length, Eq. (4):
    xi = sqrt(chi(0)/chi(k_min) - 1) / (2 sin(k_min/2)), k_min = 2 pi / L.
    NaN where chi(0) <= chi(k_min)."""
    chi0 = np.asarray(chi0, dtype=np.float64)
    chik = np.asarray(chik, dtype=np.float64)
    ratio = np.divide(chi0, chik, out=np.full(np.broadcast(chi0, chik).shape, np.nan), where=chik > 0)
    arg = ratio - 1.0
    out = np.full(arg.shape, np.nan)
    ok = arg >= 0
    out[ok] = np.sqrt(arg[ok]) / (2.0 * math.sin(math.pi / L))
    return out if out.ndim else float(out)


# ---------------------------------------------------------------------------
# Jackknife over samples
# ---------------------------------------------------------------------------
def jackknife(per_sample, fn: Callable[[np.ndarray], np.ndarray] | None = None):
    """Estimate and jackknife error of fn(mean over samples).

    per_sample: array [n_samples, ...] (e.g. thermal means per sample); fn
    maps a disorder average [...] to the quantity of interest (identity if
    None).  Returns (fn(full mean), sqrt((n-1)/n sum_i (fn_i - mean_i fn_i)^2))
    with fn_i evaluated on the mean without sample i."""
    x = np.asarray(per_sample, dtype=np.float64)
    n = x.shape[0]
    if n < 2:
        raise ValueError("the jackknife needs at least two samples")
    f = (lambda a: a) if fn is None else fn
    total = x.sum(axis=0)
    full = np.asarray(f(total / n), dtype=np.float64)
    loo = np.stack([np.asarray(f((total - x[i]) / (n - 1)), dtype=np.float64) for i in range(n)])
    err = np.sqrt((n - 1) / n * ((loo - loo.mean(axis=0)) ** 2).sum(axis=0))
    return full, err


# ---------------------------------------------------------------------------
# Logarithmic binning and the thermalization test (Sec. III)
# ---------------------------------------------------------------------------
def log_bins(n_measurements: int) -> list[tuple[int, int]]:
    """Index ranges [a, b) of the logarithmic bins of a time series of
    n_measurements, in time order: the last bin is the last half, the one
    before it the second quarter, then the second eighth, ...; each bin is
    twice as long as the previous.  The leftover head of the series (its
    first measurement for n = 2^K) belongs to no bin."""
    if n_measurements < 2:
        return []
    bins = []
    b = n_measurements
    while b >= 2:
        a = b - b // 2
        bins.append((a, b))
        b = a
    return bins[::-1]


def bin_means(series) -> np.ndarray:
    """Means of a time series [n_measurements, ...] over its logarithmic bins,
    [n_bins, ...] in time order."""
    x = np.asarray(series, dtype=np.float64)
    return np.stack([x[a:b].mean(axis=0) for a, b in log_bins(x.shape[0])])


def run_log_binned(lat, n_bins: int, base_steps: int) -> np.ndarray:
    """Runs a libhsg Lattice through n_bins logarithmic bins and returns the
    thermal means of each bin, [n_bins, S, N_T, 9].  Bin 0 is base_steps
    Monte Carlo steps long and bin i >= 1 base_steps * 2^(i-1), so the last
    bin is the last half of the run.  The measurement period of the lattice
    must divide base_steps."""
    out = []
    for i in range(n_bins):
        lat.reset_observables()
        lat.run_steps(base_steps * (1 if i == 0 else 2 ** (i - 1)))
        obs, counts = lat.read_observables()
        if np.any(counts == 0):
            raise ValueError("a bin holds no measurement: measure_every must divide base_steps")
        out.append(observable_means(obs, counts, lat.n_replicas))
    return np.stack(out)


def thermalization_test(bins_per_sample):
    """The thermalization test of Sec. III: the disorder average of
    <O_n(i)> - <O_n(i_f)> for every bin i, with its jackknife error over
    samples.  bins_per_sample: [n_samples, n_bins, ...] bin means.  A set of
    samples is thermalized when these differences converge to zero."""
    x = np.asarray(bins_per_sample, dtype=np.float64)
    diff = x - x[:, -1:]
    return jackknife(diff)


# ---------------------------------------------------------------------------
# Crossings and the quotients method (Sec. V)
# ---------------------------------------------------------------------------
def _fit(T, y, n_points: int, order: int, t0: float):
    idx = np.argsort(np.abs(T - t0), kind="stable")[:n_points]
    return np.polynomial.polynomial.polyfit(T[idx], y[idx], order)


def _crossing_of(T, y1, y2, n_points: int, order: int):
    d = y1 - y2
    sign = np.nonzero(np.diff(np.sign(d)) != 0)[0]
    if len(sign) == 0:
        return None
    j = sign[0]
    t0 = T[j] - d[j] * (T[j + 1] - T[j]) / (d[j + 1] - d[j])   # first guess
    c1, c2 = _fit(T, y1, n_points, order, t0), _fit(T, y2, n_points, order, t0)
    roots = np.polynomial.polynomial.polyroots(c1 - c2) if order > 0 else np.array([])
    roots = roots[np.isreal(roots)].real
    if len(roots) == 0:
        return None
    tc = roots[np.argmin(np.abs(roots - t0))]
    return tc, c1, c2


def crossing(T: Sequence[float], y_L, y_2L, n_points: int = 4, order: int = 1):
    """Temperature where y_L(T) and y_2L(T) cross (Sec. V): each curve is
    fitted by a polynomial of the given order over the n_points temperatures
    nearest to the crossing, and the fits are intersected.  Returns
    (T_cross, y_L(T_cross), dy_L/dT, dy_2L/dT) from the fits, or None if the
    curves do not cross in the range."""
    T = np.asarray(T, dtype=np.float64)
    order_T = np.argsort(T)
    T, y1, y2 = T[order_T], np.asarray(y_L, float)[order_T], np.asarray(y_2L, float)[order_T]
    r = _crossing_of(T, y1, y2, n_points, order)
    if r is None:
        return None
    tc, c1, c2 = r
    P = np.polynomial.polynomial
    return tc, P.polyval(tc, c1), P.polyval(tc, P.polyder(c1)), P.polyval(tc, P.polyder(c2))


def quotients(T, xi_L, xi_2L, chi_L, chi_2L, L: int, n_points: int = 4, order: int = 1):
    """Quotients method (Sec. V) for sizes L and 2L at the crossing T* of
    xi_L/L and xi_2L/(2L): returns dict(T=T*, xi_over_L=xi_L(T*)/L, nu, eta)
    with 2^(1+1/nu) = (dxi_2L/dT)/(dxi_L/dT) and 2^(2-eta) =
    chi_2L(T*)/chi_L(T*), derivatives and values from the same fits."""
    T = np.asarray(T, dtype=np.float64)
    c = crossing(T, np.asarray(xi_L) / L, np.asarray(xi_2L) / (2 * L), n_points, order)
    if c is None:
        return None
    tc, y, d1, d2 = c
    # d xi / dT = size * d(xi/size)/dT
    ratio_xi = (2 * L * d2) / (L * d1)
    P = np.polynomial.polynomial
    idx = np.argsort(T)
    Ts = T[idx]
    chi1 = P.polyval(tc, _fit(Ts, np.asarray(chi_L, float)[idx], n_points, order, tc))
    chi2 = P.polyval(tc, _fit(Ts, np.asarray(chi_2L, float)[idx], n_points, order, tc))
    nu = 1.0 / (math.log2(ratio_xi) - 1.0) if ratio_xi > 2.0 else float("nan")
    eta = 2.0 - math.log2(chi2 / chi1) if chi2 > 0 and chi1 > 0 else float("nan")
    return {"T": tc, "xi_over_L": y, "nu": nu, "eta": eta}


def jackknife_quotients(T, means_L, means_2L, L: int, sector: str = "sg", n_points: int = 4,
                        order: int = 1):
    """The quotients of ``quotients`` with jackknife errors over samples
    (Sec. V: each jackknife block is fitted separately).

    means_L [n_L, N_T, 9], means_2L [n_2L, N_T, 9]: per-sample thermal means
    at sizes L and 2L on the same temperatures; sector "sg" or "cg".  The
    two sizes have independent samples; block i leaves out sample i of each
    (the smaller set sets the number of blocks).  Returns {key: (value,
    error)} for T, xi_over_L, nu, eta."""
    a, b = np.asarray(means_L, float), np.asarray(means_2L, float)
    n = min(len(a), len(b))
    if n < 2:
        raise ValueError("the jackknife needs at least two samples per size")
    k0, kk = (Q2, Q2K) if sector == "sg" else (C2, C2K)

    def est(ma, mb):
        xa = xi_second_moment(L ** 3 * ma[:, k0], L ** 3 * ma[:, kk], L)
        xb = xi_second_moment((2 * L) ** 3 * mb[:, k0], (2 * L) ** 3 * mb[:, kk], 2 * L)
        r = quotients(T, xa, xb, L ** 3 * ma[:, k0], (2 * L) ** 3 * mb[:, k0], L, n_points, order)
        return None if r is None else np.array([r["T"], r["xi_over_L"], r["nu"], r["eta"]])

    full = est(a.mean(0), b.mean(0))
    if full is None:
        return None
    sa, sb = a.sum(0), b.sum(0)
    blocks = []
    for i in range(n):
        r = est((sa - a[i]) / (len(a) - 1), (sb - b[i]) / (len(b) - 1))
        if r is None:
            return None
        blocks.append(r)
    blocks = np.stack(blocks)
    err = np.sqrt((n - 1) / n * ((blocks - blocks.mean(0)) ** 2).sum(0))
    return {k: (full[j], err[j]) for j, k in enumerate(("T", "xi_over_L", "nu", "eta"))}
