"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the
oracle: disorder samples (couplings), initial spins and temperature ladders.

This module holds none of the Monte Carlo arithmetic.  It only draws the
quenched disorder and starting configurations that both sides consume as
data.  Random numbers come from numpy's Philox bit generator, keyed by
(seed, stream id), so every array is reproducible from its arguments alone.

Coupling law (Sec. II.A, Eq. (1)): for every bond (x, x+e_mu) the matrix
J = eps*I + D with D symmetric; eps and the six entries D^{ab}, a >= b, are
independent with mean 0, var(eps) = 1 and var(D^{ab}) = D^2.  Two laws:
  * "gaussian": eps ~ N(0,1), D^{ab} ~ N(0, D^2)  (the workloads used here);
  * "bimodal":  eps = +-1, D^{ab} = +-D           (the paper's production law).
The symmetric matrix is returned as its six entries (xx, yy, zz, xy, xz, yz),
computed in float64 and rounded once to the storage precision: "f32" (float32)
or "f16" (IEEE half, round-to-nearest-even), returned as float32 arrays whose
values are exactly representable in the storage precision.

Array layouts (site i = x + L*(y + L*z)):
  couplings  float32 [N, 3, 6]   bond (i, i+e_mu) at [i, mu, :]
  spins      float32 [N, 3]
"""
from __future__ import annotations

import numpy as np

__all__ = ["couplings", "ferromagnet", "random_spins", "random_spins_batch",
           "linear_betas", "geometric_betas", "STREAM_COUPLINGS", "STREAM_SPINS", "bimodal_bits",
           "STREAM_BIMODAL"]

STREAM_COUPLINGS = 0x4A000000
STREAM_SPINS = 0x53000000
STREAM_BIMODAL = 0x42000000


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1),
                                                     int(stream) & (2**64 - 1)]))


def _round(J6: np.ndarray, precision: str) -> np.ndarray:
    if precision == "f32":
        return J6.astype(np.float32)
    if precision == "f16":
        return J6.astype(np.float16).astype(np.float32)
    raise ValueError(f"unknown precision {precision!r}")


def couplings(L: int, seed: int = 1, sample: int = 0, law: str = "gaussian",
              D: float = 1.0, precision: str = "f32") -> np.ndarray:
    """Couplings of disorder sample `sample`, float32 [L^3, 3, 6]."""
    if L < 2:
        raise ValueError("L must be >= 2")
    N = L ** 3
    g = _rng(seed, STREAM_COUPLINGS + sample)
    if law == "gaussian":
        eps = g.standard_normal((N, 3))
        d = g.standard_normal((N, 3, 6)) * D
    elif law == "bimodal":
        eps = np.where(g.integers(0, 2, (N, 3)) == 1, 1.0, -1.0)
        d = np.where(g.integers(0, 2, (N, 3, 6)) == 1, D, -D).astype(np.float64)
    else:
        raise ValueError(f"unknown law {law!r}")
    J6 = d.copy()
    J6[..., 0:3] += eps[..., None]
    return _round(J6, precision)


def bimodal_bits(L: int, seed: int = 1, sample: int = 0) -> np.ndarray:
    """Bimodal couplings of disorder sample `sample` as their sign bytes,
    uint8 [L^3, 3]: seven independent fair bits per bond (bit 0 for the
    isotropic coupling, bits 1..6 for the six anisotropy entries), bit 7
    clear."""
    N = L ** 3
    g = _rng(seed, STREAM_BIMODAL + sample)
    return g.integers(0, 128, (N, 3), dtype=np.uint8)


def ferromagnet(L: int) -> np.ndarray:
    """J = identity on every bond (the ferromagnetic check of App. A.4.3)."""
    J6 = np.zeros((L ** 3, 3, 6), dtype=np.float32)
    J6[..., 0:3] = 1.0
    return J6


def random_spins(L: int, seed: int = 1, sample: int = 0, slot: int = 0) -> np.ndarray:
    """Spins uniform on the unit sphere, float32 [L^3, 3]: z = 2 r1 - 1,
    phi = 2 pi r2, computed in float64 and rounded once."""
    N = L ** 3
    g = _rng(seed, STREAM_SPINS + (sample << 16) + slot)
    r = g.random((N, 2))
    z = 2.0 * r[:, 0] - 1.0
    phi = 2.0 * np.pi * r[:, 1]
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    s = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    return s.astype(np.float32)


def random_spins_batch(L: int, seed: int, sample: int, n_lattices: int) -> np.ndarray:
    """random_spins for slots 0..n_lattices-1 of one sample, [R, L^3, 3]."""
    return np.stack([random_spins(L, seed, sample, j) for j in range(n_lattices)])


def linear_betas(T_min: float, T_max: float, n: int) -> np.ndarray:
    """Temperatures evenly spaced in [T_min, T_max]; returns beta = 1/T in
    increasing order (float64)."""
    if n == 1:
        return np.array([1.0 / T_min])
    T = T_min + np.arange(n) * (T_max - T_min) / (n - 1)
    return np.sort(1.0 / T)


def geometric_betas(T_min: float, T_max: float, n: int) -> np.ndarray:
    """Temperatures in a geometric sequence (the ladder of Table I)."""
    if n == 1:
        return np.array([1.0 / T_min])
    T = T_min * (T_max / T_min) ** (np.arange(n) / (n - 1))
    return np.sort(1.0 / T)
