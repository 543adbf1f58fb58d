"""TEST INFRASTRUCTURE ONLY -- the oracle of the host analysis tail.

Plain, loop-by-loop restatements of the paper's analysis (Secs. II.B, III,
V), written independently of paper_1309_1599_b300.analysis so the tests can
compare the two; only tests/ may import this module.

  xi(chi0, chik, L)      Eq. (4), the second-moment correlation length
  jackknife(x, f)        leave-one-out blocks over samples
  log_bins(n)            Sec. III: bins of doubling length ending with the
                         last half of the series
  linear_crossing(...)   Sec. V: least-squares lines over the four
                         temperatures nearest the crossing, intersected
  quotient_nu / quotient_eta   Sec. V, the quotients method
"""
import math


def xi(chi0, chik, L):
    """Eq. (4) with k_min = 2 pi / L."""
    r = chi0 / chik - 1.0
    if r < 0:
        return float("nan")
    return math.sqrt(r) / (2.0 * math.sin(math.pi / L))


def jackknife(samples, f):
    """samples: list of per-sample vectors (lists of floats); f maps a mean
    vector to a float.  Returns (f(mean), jackknife error)."""
    n = len(samples)
    dim = len(samples[0])
    mean = [sum(s[k] for s in samples) / n for k in range(dim)]
    blocks = []
    for i in range(n):
        m = [sum(samples[j][k] for j in range(n) if j != i) / (n - 1) for k in range(dim)]
        blocks.append(f(m))
    bbar = sum(blocks) / n
    var = sum((b - bbar) ** 2 for b in blocks) * (n - 1) / n
    return f(mean), math.sqrt(var)


def log_bins(n):
    """[(first, last+1)] of each bin, earliest first: the last bin is the
    last half of the n measurements, each earlier bin half as long."""
    out = []
    hi = n
    while hi >= 2:
        length = hi // 2
        out.insert(0, (hi - length, hi))
        hi -= length
    return out


def _line(ts, ys):
    """Least-squares line y = a + b t through the points (normal equations)."""
    m = len(ts)
    st, sy = sum(ts), sum(ys)
    stt = sum(t * t for t in ts)
    sty = sum(t * y for t, y in zip(ts, ys))
    b = (m * sty - st * sy) / (m * stt - st * st)
    a = (sy - b * st) / m
    return a, b


def linear_crossing(T, y1, y2, n_points=4):
    """Crossing of two curves sampled at T: find where y1 - y2 changes sign,
    take the n_points temperatures nearest to the linear-interpolation guess,
    fit a line to each curve, intersect.  Returns (T*, y1(T*), slope1,
    slope2) or None."""
    pts = sorted(zip(T, y1, y2))
    guess = None
    for (ta, a1, a2), (tb, b1, b2) in zip(pts, pts[1:]):
        da, db = a1 - a2, b1 - b2
        if (da > 0) != (db > 0) or da == 0:
            guess = ta - da * (tb - ta) / (db - da)
            break
    if guess is None:
        return None
    near = sorted(pts, key=lambda p: abs(p[0] - guess))[:n_points]
    a1, b1 = _line([p[0] for p in near], [p[1] for p in near])
    a2, b2 = _line([p[0] for p in near], [p[2] for p in near])
    if b1 == b2:
        return None
    tc = (a2 - a1) / (b1 - b2)
    return tc, a1 + b1 * tc, b1, b2


def quotient_nu(dxi_L, dxi_2L):
    """(d xi_2L/dT)/(d xi_L/dT) = 2^(1 + 1/nu)."""
    return 1.0 / (math.log(dxi_2L / dxi_L, 2) - 1.0)


def quotient_eta(chi_L, chi_2L):
    """chi_2L/chi_L = 2^(2 - eta)."""
    return 2.0 - math.log(chi_2L / chi_L, 2)
