"""Shared set-up for the GPU parity tests: build a context from seeded
synthetic inputs and compare its state with the oracle."""
import numpy as np

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg

SEED = 1
# parity tolerance: max |ds| per site after one sweep from identical input
SWEEP_TOL = 2e-5
# Heat-bath sites whose field direction lies within this distance of the
# equator h_z = 0, where the azimuthal frame of the draw (Duff et al.) changes
# sign, may legitimately be drawn in either frame (binary32 and binary64 can
# disagree on the sign of h_z there): such a site must equal the oracle's draw
# in the frame the oracle picked or the same polar part and azimuth in the
# other frame.
FRAME_EPS = 1e-4


def _duff_frame(n, sgn):
    """The orthonormal frame (e1, e2) around unit vectors n [k, 3] of
    T. Duff et al., JCGT 6(1) 2017, for the branch sign sgn [k]."""
    p = -1.0 / (sgn + n[:, 2])
    q = n[:, 0] * n[:, 1] * p
    e1 = np.stack([1.0 + sgn * n[:, 0] ** 2 * p, sgn * q, -sgn * n[:, 0]], axis=1)
    e2 = np.stack([q, sgn + n[:, 1] ** 2 * p, -n[:, 1]], axis=1)
    return e1, e2


def other_frame_draw(h, s_ref):
    """Heat-bath draws s_ref [k, 3] made around fields h [k, 3] in the frame of
    the sign of h_z, re-expressed with the same polar part and azimuth in the
    frame of the opposite sign."""
    n = h / np.linalg.norm(h, axis=1, keepdims=True)
    sgn = np.copysign(1.0, n[:, 2])
    e1, e2 = _duff_frame(n, sgn)
    f1, f2 = _duff_frame(n, -sgn)
    u = (s_ref * n).sum(1)
    a = (s_ref * e1).sum(1)
    b = (s_ref * e2).sum(1)
    return u[:, None] * n + a[:, None] * f1 + b[:, None] * f2


def frame_ambiguous_diff(got, ref, h):
    """Per-site largest component difference of GPU draws `got` from the
    oracle's draws `ref` at frame-ambiguous sites: the smaller of the
    differences from the draw in either frame."""
    d_ref = np.abs(got - ref).max(axis=1)
    d_alt = np.abs(got - other_frame_draw(h, ref)).max(axis=1)
    return np.minimum(d_ref, d_alt)


def make(Ls, beta, n_rep=2, prec=hsg.F32, layout=hsg.PLAIN, n_or=8, measure_every=0,
         seed=SEED, law="gaussian", persistent=False):
    """Context with couplings and random spins from hsg_inputs; returns
    (lattice, couplings per sample as stored, float32 [N,3,6])."""
    Ls = [Ls] if np.isscalar(Ls) else list(Ls)
    lat = hsg.Lattice(Ls, beta, n_replicas=n_rep, coupling_prec=prec, layout=layout,
                      n_or=n_or, measure_every=measure_every, seed=seed, persistent=persistent)
    pstr = "f16" if prec == hsg.F16 else "f32"
    J = []
    for s, L in enumerate(Ls):
        J6 = (gi.couplings(L, seed, s, law=law, precision=pstr) if law != "ferro"
              else gi.ferromagnet(L))
        lat.set_couplings(s, J6)
        J.append(J6)
        for slot in range(lat.R):
            lat.set_spins(s, slot, gi.random_spins(L, seed, s, slot))
    return lat, J


def state(lat):
    """All spins as float64 arrays [sample][slot] of shape [N,3]."""
    return [[lat.get_spins(s, j).astype(np.float64) for j in range(lat.R)]
            for s in range(lat.S)]


def temp_of(lat):
    perm = lat.get_perm()
    t = np.empty((lat.S, lat.R), dtype=np.int64)
    for s in range(lat.S):
        for r in range(lat.n_replicas):
            t[s, perm[s, r]] = np.arange(lat.NT)
    return t


def colours(L):
    i = np.arange(L ** 3)
    return (i % L + (i // L) % L + i // (L * L)) % 2


def compare_sweep(lat, J, before, after, kind, hb_t, J9s=None, tmp=None):
    """Per-half-sweep parity of one GPU sweep: the black half against the
    oracle's black half from `before`; the white half against the oracle's
    white half applied to the GPU's new black spins.  J: couplings per sample
    as given to the library, or J9s: the oracle's own bond matrices per
    sample (bimodal couplings).  tmp: the temperature index of each slot
    during the sweep (default: the context's current labels).  Returns (max
    |ds| over all compared components -- at frame-ambiguous sites the
    smaller of the differences from the oracle's draw in either frame --,
    number of frame-ambiguous sites, max |du| over those sites)."""
    tmp = temp_of(lat) if tmp is None else tmp
    worst, n_amb, worst_u = 0.0, 0, 0.0
    for s, L in enumerate(lat.Ls):
        J9 = J9s[s] if J9s is not None else oracle.j9_from_j6(J[s])
        col = colours(L)
        for slot in range(lat.R):
            beta = float(lat.beta[tmp[s, slot]])
            lid = s * lat.R + slot
            ref = before[s][slot].copy()
            h = oracle.fields(L, J9, ref, 0)
            oracle.half_sweep(L, J9, ref, 0, kind, beta, lat.seed, lid, hb_t)
            mixed = np.where((col == 0)[:, None], after[s][slot], before[s][slot])
            mixed = np.ascontiguousarray(mixed)
            h += oracle.fields(L, J9, mixed, 1)
            oracle.half_sweep(L, J9, mixed, 1, kind, beta, lat.seed, lid, hb_t)
            ref = np.where((col == 0)[:, None], ref, mixed)
            got = after[s][slot]
            amb = np.zeros(L ** 3, dtype=bool)
            if kind == oracle.HB:
                hn = np.linalg.norm(h, axis=1)
                amb = np.abs(h[:, 2]) < FRAME_EPS * hn
                if amb.any():
                    hh = h[amb] / hn[amb, None]
                    du = np.abs(((got[amb] - ref[amb]) * hh).sum(1)).max()
                    worst_u = max(worst_u, float(du))
                    assert np.abs(np.linalg.norm(got[amb], axis=1) - 1).max() < 1e-5
                    n_amb += int(amb.sum())
                    worst = max(worst, float(frame_ambiguous_diff(got[amb], ref[amb], h[amb]).max()))
            if (~amb).any():
                worst = max(worst, float(np.abs(got[~amb] - ref[~amb]).max()))
    return worst, n_amb, worst_u


def max_diff(a, b):
    return max(float(np.abs(x - y).max()) for ra, rb in zip(a, b) for x, y in zip(ra, rb))
