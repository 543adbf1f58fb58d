"""Python binding of libhsg (include/hsg.h): Monte Carlo of the 3d
Heisenberg spin glass with random anisotropic couplings on one B300
(arXiv:1309.1599).

Argument marshalling only: every step of the Monte Carlo runs in the CUDA
kernels of ``libhsg.so``.  The binding refuses to work without that library
or without a CUDA device; there is no CPU fallback.  PyTorch is used only to
obtain the current CUDA stream.

Method names follow the C functions without the ``hsg_`` prefix.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Lattice", "HsgError", "load_library", "philox4x32_10", "library_path",
           "F32", "F16", "PLAIN", "BATCHED", "SWEEP_AUTO", "SWEEP_TWO_PASS", "NOBS",
           "OBS_NAMES"]

ABI_VERSION = 3            # HSG_VERSION of include/hsg.h
F32, F16, BIMODAL = 0, 1, 2
PLAIN, BATCHED = 0, 1
SWEEP_AUTO, SWEEP_TWO_PASS = 0, 1
NOBS = 9
OBS_NAMES = ("e", "e2", "q2", "q4", "q2k", "c2", "c4", "c2k", "sd")
_STATUS = {0: "HSG_OK", 1: "HSG_EINVAL", 2: "HSG_ENOMEM", 3: "HSG_ECUDA",
           4: "HSG_ETIMEOUT", 5: "HSG_ESTATE", 6: "HSG_EIO"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhsg.so")
_lib = None


def library_path() -> str:
    return _LIB_PATH


class HsgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("L", ctypes.POINTER(ctypes.c_int)),
                ("n_replicas", ctypes.c_int), ("n_temps", ctypes.c_int),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("coupling_prec", ctypes.c_int),
                ("layout", ctypes.c_int), ("n_or", ctypes.c_int), ("measure_every", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("timeout_cycles", ctypes.c_longlong), ("sweep_kernel", ctypes.c_int),
                ("band_rows", ctypes.c_int), ("persistent", ctypes.c_int),
                ("bimodal_D", ctypes.c_double), ("fused_groups", ctypes.c_int)]


_SIGNATURES = {
    "hsg_lattice_create": [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p)],
    "hsg_set_couplings": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_couplings": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_set_couplings_bimodal": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_set_spins_device": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_spins_device": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_couplings_bimodal": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_set_spins": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "hsg_set_spins_sample": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_spins_sample": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_spins": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "hsg_sweep_hb": [ctypes.c_void_p, ctypes.c_int],
    "hsg_sweep_or": [ctypes.c_void_p, ctypes.c_int],
    "hsg_sweep_or_sequential": [ctypes.c_void_p, ctypes.c_int],
    "hsg_energy": [ctypes.c_void_p],
    "hsg_get_energies": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_set_energies": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_pt_swap": [ctypes.c_void_p],
    "hsg_get_perm": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_set_perm": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_get_pt_accepts": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_measure": [ctypes.c_void_p],
    "hsg_run_steps": [ctypes.c_void_p, ctypes.c_int],
    "hsg_read_observables": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "hsg_reset_observables": [ctypes.c_void_p],
    "hsg_get_counters": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_set_counters": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_get_launch_count": [ctypes.c_void_p, ctypes.c_void_p],
    "hsg_get_sweep_plan": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_get_resident_plan": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hsg_autotune": [ctypes.c_void_p],
    "hsg_save": [ctypes.c_void_p, ctypes.c_char_p],
    "hsg_load": [ctypes.c_void_p, ctypes.c_char_p],
    "hsg_synchronize": [ctypes.c_void_p],
    "hsg_selftest_wait_timeout": [ctypes.c_void_p, ctypes.c_longlong],
    "hsg_philox4x32_10": [ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p],
}


def load_library():
    """Load libhsg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with "
                              "`python paper_1309_1599_b300/build.py` (needs nvcc)")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.hsg_destroy.argtypes = [ctypes.c_void_p]
        lib.hsg_destroy.restype = None
        lib.hsg_last_error.argtypes = []
        lib.hsg_last_error.restype = ctypes.c_char_p
        lib.hsg_version.argtypes = []
        lib.hsg_version.restype = ctypes.c_int
        if lib.hsg_version() != ABI_VERSION:
            raise ImportError(f"{_LIB_PATH} has ABI version {lib.hsg_version()}, this binding "
                              f"expects {ABI_VERSION}: rebuild it")
        _lib = lib
    return _lib


def _check(status: int) -> None:
    if status != 0:
        raise HsgError(status, load_library().hsg_last_error().decode())


def _ptr(a) -> ctypes.c_void_p:
    """Address of a contiguous numpy array or CPU torch tensor."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _host_f32(a, n: int, out: bool = False):
    """A contiguous float32 host buffer of n elements: a numpy array, or a
    CPU torch tensor (pinned or not).  Inputs are converted when they are
    numpy-like; output buffers must already have the right type and size.
    Raises ValueError otherwise, so that no call reads or writes past a
    caller's buffer."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.device.type != "cpu" or a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"expected a contiguous float32 CPU tensor of {n} elements")
        return a
    if out:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous and a.size == n):
            raise ValueError(f"expected a C-contiguous float32 numpy array of {n} elements")
        return a
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return a


def _device_f32(t, n: int) -> None:
    """Checks a contiguous float32 CUDA tensor of n elements (ValueError)."""
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"expected a contiguous float32 CUDA tensor of {n} elements")


def _require_gpu() -> None:
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libhsg needs a CUDA device (B300); none is visible")


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def philox4x32_10(rows) -> np.ndarray:
    """Device Philox4x32-10 of rows (c0,c1,c2,c3,k0,k1) -> uint32 [n, 4]."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32).reshape(-1, 6)
    out = np.empty((rows.shape[0], 4), dtype=np.uint32)
    _check(load_library().hsg_philox4x32_10(_ptr(rows), rows.shape[0], _ptr(out)))
    return out


class Lattice:
    """One libhsg context: S samples x n_replicas x n_temps lattices.

    ``Lattice(L, beta, n_replicas, ...)`` is hsg_lattice_create; L is an int
    or a list of per-sample sizes.  The keyword arguments are the fields of
    hsg_config in include/hsg.h: among them ``persistent`` (False/0 streaming
    steps, True/1 resident steps with one launch per lattice size, 2 all
    lattice sizes in one launch) and the tiling overrides ``band_rows`` and
    ``fused_groups`` (0 leaves both to the library and its autotuner)."""

    def __init__(self, L, beta, n_replicas=2, n_samples=None, coupling_prec=F32,
                 layout=PLAIN, n_or=8, measure_every=0, seed=1, stream=None,
                 timeout_cycles=0, sweep_kernel=SWEEP_AUTO, band_rows=0, persistent=False,
                 bimodal_D=1.0, fused_groups=0):
        lib = load_library()
        _require_gpu()
        if np.isscalar(L):
            L = [int(L)] * (1 if n_samples is None else int(n_samples))
        self.Ls = [int(x) for x in L]
        self.S = len(self.Ls)
        self.beta = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1)
        self.NT = len(self.beta)
        self.n_replicas = int(n_replicas)
        self.R = self.n_replicas * self.NT
        self.n_or = int(n_or)
        self.seed = int(seed) & (2**64 - 1)
        self._L_arr = (ctypes.c_int * self.S)(*self.Ls)
        cfg = _Config()
        cfg.n_samples = self.S
        cfg.L = self._L_arr
        cfg.n_replicas = self.n_replicas
        cfg.n_temps = self.NT
        cfg.beta = self.beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.coupling_prec = int(coupling_prec)
        cfg.layout = int(layout)
        cfg.n_or = self.n_or
        cfg.measure_every = int(measure_every)
        cfg.seed = int(seed) & (2**64 - 1)
        cfg.stream = _current_stream() if stream is None else ctypes.c_void_p(stream)
        cfg.timeout_cycles = int(timeout_cycles)
        cfg.sweep_kernel = int(sweep_kernel)
        cfg.band_rows = int(band_rows)
        cfg.persistent = int(persistent)
        cfg.bimodal_D = float(bimodal_D)
        cfg.fused_groups = int(fused_groups)
        self.coupling_prec = int(coupling_prec)
        self.bimodal_D = float(bimodal_D)
        h = ctypes.c_void_p()
        _check(lib.hsg_lattice_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._lib = lib

    # -- lifetime --------------------------------------------------------
    def destroy(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hsg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def N(self, sample: int = 0) -> int:
        return self.Ls[sample] ** 3

    # -- data ------------------------------------------------------------
    def set_couplings(self, sample: int, J6) -> None:
        """Couplings float32 [N, 3, 6] from a numpy array or a contiguous CPU
        torch tensor (pinned or not)."""
        J6 = _host_f32(J6, self.N(sample) * 18)
        _check(self._lib.hsg_set_couplings(self._h, sample, _ptr(J6)))

    def get_couplings(self, sample: int) -> np.ndarray:
        out = np.empty((self.N(sample), 3, 6), dtype=np.float32)
        _check(self._lib.hsg_get_couplings(self._h, sample, _ptr(out)))
        return out

    def set_couplings_bimodal(self, sample: int, bits) -> None:
        bits = np.ascontiguousarray(bits, dtype=np.uint8)
        if bits.size != self.N(sample) * 3:
            raise ValueError(f"expected {self.N(sample) * 3} bond bytes, got {bits.size}")
        _check(self._lib.hsg_set_couplings_bimodal(self._h, sample, _ptr(bits)))

    def get_couplings_bimodal(self, sample: int) -> np.ndarray:
        out = np.empty((self.N(sample), 3), dtype=np.uint8)
        _check(self._lib.hsg_get_couplings_bimodal(self._h, sample, _ptr(out)))
        return out

    def set_spins(self, sample: int, slot: int, s) -> None:
        s = _host_f32(s, self.N(sample) * 3)
        _check(self._lib.hsg_set_spins(self._h, sample, slot, _ptr(s)))

    def get_spins(self, sample: int, slot: int, out=None):
        if out is None:
            out = np.empty((self.N(sample), 3), dtype=np.float32)
        out = _host_f32(out, self.N(sample) * 3, out=True)
        _check(self._lib.hsg_get_spins(self._h, sample, slot, _ptr(out)))
        return out

    def set_spins_sample(self, sample: int, s) -> None:
        """Every lattice slot of a sample from host float32 [R, N, 3] (a numpy
        array or a contiguous CPU torch tensor, pinned or not)."""
        s = _host_f32(s, self.R * self.N(sample) * 3)
        _check(self._lib.hsg_set_spins_sample(self._h, sample, _ptr(s)))

    def get_spins_sample(self, sample: int, out=None):
        """Every lattice slot of a sample as host float32 [R, N, 3]."""
        if out is None:
            out = np.empty((self.R, self.N(sample), 3), dtype=np.float32)
        out = _host_f32(out, self.R * self.N(sample) * 3, out=True)
        _check(self._lib.hsg_get_spins_sample(self._h, sample, _ptr(out)))
        return out

    # -- Monte Carlo -----------------------------------------------------
    def set_spins_device(self, sample: int, slot: int, tensor) -> None:
        """From a contiguous float32 CUDA tensor [N, 3] on the context's device
        (stream-ordered, no host copy)."""
        _device_f32(tensor, self.N(sample) * 3)
        _check(self._lib.hsg_set_spins_device(self._h, sample, slot, ctypes.c_void_p(tensor.data_ptr())))

    def get_spins_device(self, sample: int, slot: int, tensor) -> None:
        """Into a contiguous float32 CUDA tensor [N, 3] (stream-ordered)."""
        _device_f32(tensor, self.N(sample) * 3)
        _check(self._lib.hsg_get_spins_device(self._h, sample, slot, ctypes.c_void_p(tensor.data_ptr())))

    def sweep_hb(self, n: int = 1) -> None:
        _check(self._lib.hsg_sweep_hb(self._h, n))

    def sweep_or(self, n: int = 1) -> None:
        _check(self._lib.hsg_sweep_or(self._h, n))

    def sweep_or_sequential(self, n: int = 1) -> None:
        _check(self._lib.hsg_sweep_or_sequential(self._h, n))

    def energy(self) -> None:
        _check(self._lib.hsg_energy(self._h))

    def get_energies(self) -> np.ndarray:
        out = np.empty((self.S, self.R), dtype=np.float64)
        _check(self._lib.hsg_get_energies(self._h, _ptr(out)))
        return out

    def set_energies(self, E) -> None:
        E = np.ascontiguousarray(E, dtype=np.float64)
        if E.size != self.S * self.R:
            raise ValueError(f"expected {self.S * self.R} energies, got {E.size}")
        _check(self._lib.hsg_set_energies(self._h, _ptr(E)))

    def pt_swap(self) -> None:
        _check(self._lib.hsg_pt_swap(self._h))

    def get_perm(self) -> np.ndarray:
        out = np.empty((self.S, self.n_replicas, self.NT), dtype=np.int32)
        _check(self._lib.hsg_get_perm(self._h, _ptr(out)))
        return out

    def set_perm(self, perm) -> None:
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        if perm.size != self.S * self.n_replicas * self.NT:
            raise ValueError(f"expected {self.S * self.n_replicas * self.NT} labels, got {perm.size}")
        _check(self._lib.hsg_set_perm(self._h, _ptr(perm)))

    def get_pt_accepts(self) -> np.ndarray:
        out = np.empty((self.S, self.n_replicas, max(self.NT - 1, 1)), dtype=np.int64)
        _check(self._lib.hsg_get_pt_accepts(self._h, _ptr(out)))
        return out

    def measure(self) -> None:
        _check(self._lib.hsg_measure(self._h))

    def run_steps(self, n: int) -> None:
        _check(self._lib.hsg_run_steps(self._h, n))

    def read_observables(self):
        obs = np.empty((self.S, self.NT, NOBS), dtype=np.float64)
        counts = np.empty((self.S, self.NT), dtype=np.int64)
        _check(self._lib.hsg_read_observables(self._h, _ptr(obs), _ptr(counts)))
        return obs, counts

    def reset_observables(self) -> None:
        _check(self._lib.hsg_reset_observables(self._h))

    def get_counters(self) -> np.ndarray:
        out = np.zeros(3, dtype=np.uint64)
        _check(self._lib.hsg_get_counters(self._h, _ptr(out)))
        return out

    def set_counters(self, hb: int, pt: int, steps: int) -> None:
        a = np.array([hb, pt, steps], dtype=np.uint64)
        _check(self._lib.hsg_set_counters(self._h, _ptr(a)))

    def get_sweep_plan(self, sample: int = 0) -> dict:
        out = np.zeros(5, dtype=np.int32)
        _check(self._lib.hsg_get_sweep_plan(self._h, sample, _ptr(out)))
        return {"fused": bool(out[0]), "band_rows": int(out[1]), "launches_per_sweep": int(out[2]),
                "groups_per_thread_or": int(out[3]), "groups_per_thread_hb": int(out[4])}

    def get_resident_plan(self, sample: int = 0) -> dict:
        out = np.zeros(6, dtype=np.int32)
        _check(self._lib.hsg_get_resident_plan(self._h, sample, _ptr(out)))
        return {"bond_residency": int(out[0]), "groups_per_item": int(out[1]), "threads": int(out[2]),
                "groups_per_cta": int(out[3]), "sets_per_cta": int(out[4]), "one_launch": bool(out[5])}

    def autotune(self) -> None:
        """Time the candidate launch shapes on this context's data and keep
        the fastest (the state is unchanged; choices are remembered for the
        process)."""
        _check(self._lib.hsg_autotune(self._h))

    def get_launch_count(self) -> int:
        out = np.zeros(1, dtype=np.uint64)
        _check(self._lib.hsg_get_launch_count(self._h, _ptr(out)))
        return int(out[0])

    def save(self, path: str) -> None:
        _check(self._lib.hsg_save(self._h, os.fsencode(path)))

    def load(self, path: str) -> None:
        _check(self._lib.hsg_load(self._h, os.fsencode(path)))

    def synchronize(self) -> None:
        _check(self._lib.hsg_synchronize(self._h))

    def selftest_wait_timeout(self, timeout_cycles: int) -> int:
        """Status of hsg_selftest_wait_timeout (4 = HSG_ETIMEOUT expected)."""
        return self._lib.hsg_selftest_wait_timeout(self._h, int(timeout_cycles))
