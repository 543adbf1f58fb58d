"""FP64 CPU oracle for the anisotropic Heisenberg spin-glass Monte Carlo.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference (``hsg_oracle.c``, plain C in IEEE double, plus this ctypes wrapper)
that the CUDA path is checked against.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA library and never imports it.

Every function follows the paper (Baity-Jesi et al., arXiv:1309.1599):
  * Hamiltonian, Eq. (1), Sec. II.A           -> energy, local_field
  * heat-bath and overrelaxation, App. A.1    -> hb_draw, or_update, sweep
  * parallel tempering, App. A.1              -> pt_sweep
  * overlaps and chiralities, Sec. II.B       -> overlap_fourier, measure_pair
  * Schwinger-Dyson identity, App. A.4.3      -> sd_residual
  * one Monte Carlo step, Sec. III / App. A.1 -> Sample.run
  * bimodal couplings, Sec. II.A              -> bimodal_j9
  * sequential overrelaxation, App. A.1       -> sweep_sequential
  * host analysis (xi, jackknife, log bins, crossings), Secs. II.B, III, V
                                              -> oracle.analysis (pure Python)

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``):
  philox4x32   Philox round structure pinned bit for bit through the
               64-bit member against numpy's independent Philox4x64-10;
               the 32-bit constants are the published ones; plus
               uniformity and horizontal (cross-stream) tests.
  hb_draw      Langevin mean and second moment, azimuthal isotropy,
               two-site detailed balance against numerical quadrature.
  or_update    norm, s.h, involution; lattice energy conserved over sweeps;
               equivariance under global rotations and local gauge
               transformations (pins J versus J^T).
  local_field  equals minus the numerical gradient of ``energy``.
  site_field   the sum local_field evaluates after gathering a site's bonds
               and neighbours (one code path), so the same pin holds;
               neighbour is the gather's index arithmetic.
  bimodal_j9   single-bit cases, the paper's moments over all 128 bytes,
               time reversal, the isotropic limit (test_oracle_bimodal.py).
  energy       beta = 0 moments; high-temperature series to O(beta^3);
               ferromagnetic ground state.
  pt_sweep     exact acceptance rule checked against hand-made cases and
               the acceptance frequency of a two-level system.
  overlap_fourier / measure_pair   closed forms on constructed states
               (uniform, cosine-modulated, conical spiral).
  sd_residual  vanishes within error in equilibrium (statistical).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HB, OR = 0, 1
N_OBS = 9
OBS_NAMES = ("e", "e2", "q2", "q4", "q2k", "c2", "c4", "c2k", "sd")


def build(force: bool = False) -> str:
    """Compile hsg_oracle.c into liboracle.so (gcc, -O2, OpenMP, IEEE math)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", "-D_GNU_SOURCE",
               _SRC, "-o", _LIB_PATH, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # HSG_ORACLE_LIB lets the mutation tests load a deliberately broken
            # build of this oracle; normally the library next to this file.
            path = os.environ.get("HSG_ORACLE_LIB")
            if not path:
                path = build()
            lib = ctypes.CDLL(path)
            d, i32, u32, u64 = (ctypes.c_double, ctypes.c_int, ctypes.c_uint32,
                                ctypes.c_uint64)
            vp = ctypes.c_void_p
            sig = {
                "oracle_philox4x32_10": (None, [vp, vp, vp]),
                "oracle_philox4x64_10": (None, [vp, vp, vp]),
                "oracle_uniform23": (d, [u32]),
                "oracle_uniform52": (d, [u32, u32]),
                "oracle_hb_words": (None, [u64, u32, u32, u32, vp]),
                "oracle_local_field": (None, [i32, vp, vp, ctypes.c_long, vp]),
                "oracle_site_field": (None, [vp, vp, vp, vp, vp]),
                "oracle_neighbour": (ctypes.c_long, [i32, ctypes.c_long, i32, i32]),
                "oracle_energy": (d, [i32, vp, vp]),
                "oracle_hb_draw": (None, [vp, d, u32, u32, vp]),
                "oracle_or_update": (None, [vp, vp, vp]),
                "oracle_half_sweep": (None, [i32, vp, vp, i32, i32, d, u64, u32, u32]),
                "oracle_sweep": (None, [i32, vp, vp, i32, d, u64, u32, u32]),
                "oracle_pt_sweep": (None, [i32, vp, vp, vp, u64, u32, u32, vp]),
                "oracle_overlap_fourier": (None, [i32, vp, vp, vp, vp, vp, vp]),
                "oracle_measure_pair": (None, [i32, vp, vp, vp]),
                "oracle_sd_residual": (d, [i32, vp, vp, d]),
                "oracle_run": (i32, [i32, vp, i32, i32, vp, vp, vp, u64, u32, u32,
                                     vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, i32]),
                "oracle_hb_draw_batch": (None, [vp, d, u64, u32, u32, ctypes.c_long, vp]),
                "oracle_two_site_chain": (None, [vp, d, u64, u32, ctypes.c_long,
                                                 ctypes.c_long, vp, vp, vp]),
                "oracle_fields": (None, [i32, vp, vp, i32, vp]),
                "oracle_bimodal_j9": (None, [ctypes.c_long, vp, d, vp]),
                "oracle_sweep_sequential": (None, [i32, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Random numbers (Philox, Salmon et al. SC'11) and the uniform mappings
# --------------------------------------------------------------------------
def philox4x32(ctr, key) -> np.ndarray:
    """Philox4x32-10 of each counter row (uint32[...,4]) under key uint32[2]."""
    lib = _load()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    for j in range(ctr.shape[0]):
        lib.oracle_philox4x32_10(ctypes.c_void_p(ctr[j].ctypes.data), _ptr(key),
                                 ctypes.c_void_p(out[j].ctypes.data))
    return out


def philox4x64(ctr, key) -> np.ndarray:
    """Philox4x64-10 of each counter row (uint64[...,4]) under key uint64[2]."""
    lib = _load()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint64).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint64).reshape(2)
    out = np.empty_like(ctr)
    for j in range(ctr.shape[0]):
        lib.oracle_philox4x64_10(ctypes.c_void_p(ctr[j].ctypes.data), _ptr(key),
                                 ctypes.c_void_p(out[j].ctypes.data))
    return out


def uniform23(w: int) -> float:
    return _load().oracle_uniform23(int(w))


def uniform52(w0: int, w1: int) -> float:
    return _load().oracle_uniform52(int(w0), int(w1))


def hb_words(seed: int, site: int, lattice: int, t: int):
    w = np.zeros(2, dtype=np.uint32)
    _load().oracle_hb_words(seed, site, lattice, t, _ptr(w))
    return int(w[0]), int(w[1])


# --------------------------------------------------------------------------
# Couplings
# --------------------------------------------------------------------------
def bimodal_j9(bits, D: float) -> np.ndarray:
    """Bimodal couplings (Sec. II.A) from their bytes uint8 [N,3] (bit 0: sign
    of J = +-1; bits 1..6: signs of D^xx, D^yy, D^zz, D^xy, D^xz, D^yz = +-D)
    as general 3x3 matrices [N,3,9] in float64."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.empty(bits.shape + (9,), dtype=np.float64)
    _load().oracle_bimodal_j9(bits.size, _ptr(bits), float(D), _ptr(out))
    return out


def j9_from_j6(J6) -> np.ndarray:
    """Expand symmetric couplings [N,3,6] (xx,yy,zz,xy,xz,yz) to general
    3x3 matrices [N,3,9] in float64 (exact: float32 -> float64)."""
    J6 = np.asarray(J6, dtype=np.float64)
    xx, yy, zz, xy, xz, yz = (J6[..., k] for k in range(6))
    J9 = np.stack([xx, xy, xz, xy, yy, yz, xz, yz, zz], axis=-1)
    return np.ascontiguousarray(J9)


# --------------------------------------------------------------------------
# Single-site updates, field and energy
# --------------------------------------------------------------------------
def local_field(L: int, J9, s, i: int) -> np.ndarray:
    J9, s = _f64(J9), _f64(s)
    h = np.zeros(3)
    _load().oracle_local_field(L, _ptr(J9), _ptr(s), i, _ptr(h))
    return h


def site_field(Jup, Jdn, s_up, s_dn) -> np.ndarray:
    """Local field of one site from its own data: Jup[mu] the 3x3 bond to
    x+mu, Jdn[mu] the bond from x-mu, s_up[mu] / s_dn[mu] the neighbour
    spins (each [3][3] / [3][9] as arrays of shape (3, 3) or (3, 3, 3))."""
    Jup, Jdn, s_up, s_dn = _f64(Jup), _f64(Jdn), _f64(s_up), _f64(s_dn)
    h = np.zeros(3)
    _load().oracle_site_field(_ptr(Jup), _ptr(Jdn), _ptr(s_up), _ptr(s_dn), _ptr(h))
    return h


def neighbour(L: int, i: int, mu: int, sign: int) -> int:
    """Natural index of the periodic neighbour of site i along mu."""
    return int(_load().oracle_neighbour(L, int(i), mu, sign))


def fields(L: int, J9, s, colour: int) -> np.ndarray:
    """Local fields [N,3] of the sites of one colour (zeros elsewhere)."""
    J9, s = _f64(J9), _f64(s)
    h = np.zeros((L ** 3, 3))
    _load().oracle_fields(L, _ptr(J9), _ptr(s), colour, _ptr(h))
    return h


def energy(L: int, J9, s) -> float:
    J9, s = _f64(J9), _f64(s)
    return _load().oracle_energy(L, _ptr(J9), _ptr(s))


def hb_draw(h, beta: float, w0: int, w1: int) -> np.ndarray:
    h = _f64(h)
    out = np.zeros(3)
    _load().oracle_hb_draw(_ptr(h), beta, int(w0), int(w1), _ptr(out))
    return out


def hb_draw_batch(h, beta: float, seed: int, lattice: int, t: int, n: int) -> np.ndarray:
    h = _f64(h)
    out = np.zeros((n, 3))
    _load().oracle_hb_draw_batch(_ptr(h), beta, seed, lattice, t, n, _ptr(out))
    return out


def two_site_chain(J, beta: float, seed: int, lattice: int, n_skip: int, n_iter: int):
    J = _f64(J).reshape(9)
    s1 = np.array([0.0, 0.0, 1.0])
    s2 = np.array([1.0, 0.0, 0.0])
    sums = np.zeros(2)
    _load().oracle_two_site_chain(_ptr(J), beta, seed, lattice, n_skip, n_iter,
                                  _ptr(s1), _ptr(s2), _ptr(sums))
    return sums[0] / n_iter, sums[1] / n_iter


def or_update(h, s) -> np.ndarray:
    h, s = _f64(h), _f64(s)
    out = np.zeros(3)
    _load().oracle_or_update(_ptr(h), _ptr(s), _ptr(out))
    return out


def half_sweep(L: int, J9, s: np.ndarray, colour: int, kind: int, beta: float = 0.0,
               seed: int = 0, lattice: int = 0, t: int = 0) -> None:
    """In place on s (float64 [N,3], C-contiguous)."""
    assert s.dtype == np.float64 and s.flags.c_contiguous
    J9 = _f64(J9)
    _load().oracle_half_sweep(L, _ptr(J9), _ptr(s), colour, kind, beta, seed, lattice, t)


def sweep(L: int, J9, s: np.ndarray, kind: int, beta: float = 0.0, seed: int = 0,
          lattice: int = 0, t: int = 0) -> None:
    """One checkerboard sweep, in place on s (float64 [N,3])."""
    assert s.dtype == np.float64 and s.flags.c_contiguous
    J9 = _f64(J9)
    _load().oracle_sweep(L, _ptr(J9), _ptr(s), kind, beta, seed, lattice, t)


def sweep_sequential(L: int, J9, s: np.ndarray) -> None:
    """One sequential overrelaxation sweep (sites in natural order, each using
    its neighbours' current values), in place on s (float64 [N,3])."""
    assert s.dtype == np.float64 and s.flags.c_contiguous
    J9 = _f64(J9)
    _load().oracle_sweep_sequential(L, _ptr(J9), _ptr(s))


def pt_sweep(beta, E, perm: np.ndarray, seed: int, replica_set: int, t_pt: int,
             accepted: np.ndarray | None = None) -> None:
    """In place on perm (int32 [n_temps]) and accepted (int64 [n_temps-1])."""
    beta, E = _f64(beta), _f64(E)
    assert perm.dtype == np.int32 and perm.flags.c_contiguous
    acc = ctypes.c_void_p(0) if accepted is None else _ptr(accepted)
    _load().oracle_pt_sweep(len(beta), _ptr(beta), _ptr(E), _ptr(perm), seed,
                            replica_set, t_pt, acc)


def overlap_fourier(L: int, sa, sb):
    sa, sb = _f64(sa), _f64(sb)
    Q0 = np.zeros(1)
    Qk, C0, Ck = np.zeros(6), np.zeros(3), np.zeros(18)
    _load().oracle_overlap_fourier(L, _ptr(sa), _ptr(sb), _ptr(Q0), _ptr(Qk),
                                   _ptr(C0), _ptr(Ck))
    return Q0[0], Qk.reshape(3, 2), C0, Ck.reshape(3, 3, 2)


def measure_pair(L: int, sa, sb) -> np.ndarray:
    sa, sb = _f64(sa), _f64(sb)
    out = np.zeros(6)
    _load().oracle_measure_pair(L, _ptr(sa), _ptr(sb), _ptr(out))
    return out


def sd_residual(L: int, J9, s, T: float) -> float:
    J9, s = _f64(J9), _f64(s)
    return _load().oracle_sd_residual(L, _ptr(J9), _ptr(s), T)


# --------------------------------------------------------------------------
# One sample's Monte Carlo run
# --------------------------------------------------------------------------
class Sample:
    """State of one disorder sample: n_replicas x n_temps lattices sharing
    the couplings J9, with the parallel-tempering labels and accumulators.

    Lattice slot = r*n_temps + j; its global lattice id (heat-bath stream) is
    sample_index*R + slot and its replica-set id (PT stream) is
    sample_index*n_replicas + r, matching the CUDA library's numbering."""

    def __init__(self, L, J6, spins, beta, n_replicas, seed, sample_index=0):
        self.L = int(L)
        self.N = self.L ** 3
        self.beta = _f64(beta)
        self.n_temps = len(self.beta)
        self.n_replicas = int(n_replicas)
        self.R = self.n_temps * self.n_replicas
        self.J9 = j9_from_j6(J6).reshape(self.N, 3, 9)
        self.spins = _f64(spins).reshape(self.R, self.N, 3).copy()
        self.seed = int(seed)
        self.sample_index = int(sample_index)
        self.perm = np.tile(np.arange(self.n_temps, dtype=np.int32), self.n_replicas)
        self.perm += np.repeat(np.arange(self.n_replicas, dtype=np.int32) * self.n_temps,
                               self.n_temps)
        self.hb_t = np.zeros(1, dtype=np.uint32)
        self.pt_t = np.zeros(1, dtype=np.uint32)
        self.steps = np.zeros(1, dtype=np.int64)
        self.obs = np.zeros((self.n_temps, N_OBS))
        self.counts = np.zeros(self.n_temps, dtype=np.int64)
        self.accepted = np.zeros((self.n_replicas, max(self.n_temps - 1, 1)), dtype=np.int64)
        self.energies = np.zeros(self.R)

    def run(self, n_steps: int, n_or: int, measure_every: int, n_threads: int = 0) -> None:
        rc = _load().oracle_run(
            self.L, _ptr(self.J9), self.n_replicas, self.n_temps, _ptr(self.beta),
            _ptr(self.spins), _ptr(self.perm), self.seed,
            self.sample_index * self.R, self.sample_index * self.n_replicas,
            _ptr(self.hb_t), _ptr(self.pt_t), _ptr(self.steps), n_steps, n_or,
            measure_every, _ptr(self.obs), _ptr(self.counts), _ptr(self.accepted),
            _ptr(self.energies), n_threads)
        if rc != 0:
            raise MemoryError("oracle_run failed")
