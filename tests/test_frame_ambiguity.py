"""The heat-bath comparison at frame-ambiguous sites (field direction at the
equator h_z = 0, where the Duff et al. frame of the azimuth changes branch):
re-expressing an oracle draw in the other branch's frame must give what the
oracle itself draws when the field's h_z has the other sign."""
import numpy as np

import oracle
from _gpu_helpers import frame_ambiguous_diff, other_frame_draw


def _fields(rng, k, hz):
    h = rng.standard_normal((k, 3)) * 2.0
    h[:, 2] = hz * np.linalg.norm(h[:, :2], axis=1)
    return h


def test_other_frame_is_the_oracle_draw_across_the_equator():
    rng = np.random.default_rng(5)
    for beta in (0.3, 1.0, 4.0):
        h_up = _fields(rng, 64, 1e-12)
        h_dn = h_up.copy()
        h_dn[:, 2] = -h_dn[:, 2]
        words = rng.integers(0, 2 ** 32, size=(64, 2), dtype=np.uint64)
        for i in range(64):
            w0, w1 = int(words[i, 0]), int(words[i, 1])
            s_up = oracle.hb_draw(h_up[i], beta, w0, w1)
            s_dn = oracle.hb_draw(h_dn[i], beta, w0, w1)
            alt = other_frame_draw(h_up[i][None], s_up[None])[0]
            assert np.abs(alt - s_dn).max() < 1e-9
            # the two branches really differ here, so the check has teeth
            assert np.abs(s_up - s_dn).max() > 1e-3 or np.abs(np.dot(s_up, h_up[i])) > 0.999 * np.linalg.norm(h_up[i])


def test_other_frame_keeps_the_polar_part_and_the_norm_and_is_an_involution():
    rng = np.random.default_rng(6)
    h = _fields(rng, 200, 3e-5)
    s = np.stack([oracle.hb_draw(h[i], 1.5, int(a), int(b))
                  for i, (a, b) in enumerate(rng.integers(0, 2 ** 32, size=(200, 2), dtype=np.uint64))])
    alt = other_frame_draw(h, s)
    n = h / np.linalg.norm(h, axis=1, keepdims=True)
    assert np.abs((alt * n).sum(1) - (s * n).sum(1)).max() < 1e-12
    assert np.abs(np.linalg.norm(alt, axis=1) - 1.0).max() < 1e-12
    # re-expressing in the branch of the opposite sign twice: back to s
    h_flip = h.copy()
    h_flip[:, 2] = -h_flip[:, 2]
    back = other_frame_draw(h_flip, alt)
    assert np.abs(back - s).max() < 2e-4  # h and h_flip differ by 2 |n_z| <= 6e-5


def test_frame_ambiguous_diff_accepts_either_frame_and_nothing_else():
    rng = np.random.default_rng(7)
    h = _fields(rng, 50, 1e-6)
    s = np.stack([oracle.hb_draw(h[i], 2.0, int(a), int(b))
                  for i, (a, b) in enumerate(rng.integers(0, 2 ** 32, size=(50, 2), dtype=np.uint64))])
    alt = other_frame_draw(h, s)
    assert frame_ambiguous_diff(s, s, h).max() == 0.0
    assert frame_ambiguous_diff(alt, s, h).max() < 1e-12
    # a draw rotated about the field by a tenth of a radian matches neither
    n = h / np.linalg.norm(h, axis=1, keepdims=True)
    u = (s * n).sum(1, keepdims=True)
    perp = s - u * n
    c, si = np.cos(0.1), np.sin(0.1)
    rot = u * n + c * perp + si * np.cross(n, perp)
    moved = np.linalg.norm(perp, axis=1) > 0.1
    assert (frame_ambiguous_diff(rot, s, h)[moved] > 1e-3).all()
