"""The C-ABI library loads and exports every function include/hsg.h declares;
configuration errors are rejected on the host before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1309_1599_b300 as hsg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hsg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:hsg_status|void|int|const char \*)\s*\*?\s*(hsg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_1599_b300 import build
    build.build()
    return hsg.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert lib.hsg_version() == hsg.ABI_VERSION == 3


def _cfg(**kw):
    L = (ctypes.c_int * 1)(kw.pop("L", 8))
    beta = np.ascontiguousarray(kw.pop("beta", [1.0, 2.0]), dtype=np.float64)
    c = hsg._Config()
    c.n_samples = 1
    c.L = L
    c.n_replicas = kw.pop("n_replicas", 2)
    c.n_temps = len(beta)
    c.beta = beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c.coupling_prec = kw.pop("prec", 0)
    c.layout = kw.pop("layout", 0)
    c.n_or = 8
    c.measure_every = 0
    c.seed = 1
    c.stream = None
    c.timeout_cycles = 0
    c.sweep_kernel = kw.pop("sweep_kernel", 0)
    c.band_rows = kw.pop("band_rows", 0)
    c.persistent = kw.pop("persistent", 0)
    c.bimodal_D = kw.pop("bimodal_D", 1.0)
    c.fused_groups = kw.pop("fused_groups", 0)
    return c, (L, beta)


@pytest.mark.parametrize("kw,msg", [
    (dict(L=7), "even"), (dict(L=2), "even"), (dict(L=514), "even"),
    (dict(beta=[2.0, 1.0]), "increasing"), (dict(beta=[-1.0]), ">= 0"),
    (dict(prec=5), "coupling_prec"), (dict(layout=9), "layout"),
    (dict(layout=1, n_replicas=1, beta=[1.0]), "even number"),
    (dict(n_replicas=0), "n_replicas"),
    (dict(sweep_kernel=7), "sweep_kernel"),
    (dict(band_rows=-1), "band_rows"),
    (dict(band_rows=8, sweep_kernel=1), "band_rows"),
    (dict(L=32, persistent=1), "shared memory"),
    (dict(persistent=1, layout=1, beta=[1.0, 2.0, 3.0], n_replicas=2), "multiple"),
    (dict(prec=2, bimodal_D=-0.5), "bimodal_D"),
    (dict(prec=2, bimodal_D=float("nan")), "bimodal_D"),
    (dict(persistent=3), "persistent"),
    (dict(fused_groups=3), "fused_groups"),
    (dict(fused_groups=1, sweep_kernel=1), "fused_groups"),
    (dict(fused_groups=2, layout=0), "fused_groups"),
    (dict(fused_groups=2, layout=1, n_replicas=1, beta=[1.0, 2.0]), "fused_groups"),
])
def test_invalid_configs_rejected_on_host(lib, kw, msg):
    c, keep = _cfg(**kw)
    h = ctypes.c_void_p(1)
    st = lib.hsg_lattice_create(ctypes.byref(c), ctypes.byref(h))
    assert st == 1                      # HSG_EINVAL
    assert h.value is None
    assert msg in lib.hsg_last_error().decode()


def test_null_arguments_rejected(lib):
    assert lib.hsg_lattice_create(None, None) == 1
    assert lib.hsg_sweep_hb(None, 1) == 1
    assert lib.hsg_run_steps(None, 1) == 1
    assert lib.hsg_philox4x32_10(None, -1, None) == 1
    assert lib.hsg_set_couplings_bimodal(None, 0, None) == 1
    assert lib.hsg_get_couplings_bimodal(None, 0, None) == 1
    assert lib.hsg_set_spins_sample(None, 0, None) == 1
    assert lib.hsg_autotune(None) == 1
    assert lib.hsg_get_resident_plan(None, 0, None) == 1
    assert lib.hsg_get_spins_sample(None, 0, None) == 1
    lib.hsg_destroy(None)


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(RuntimeError, match="CUDA device"):
        hsg.Lattice(8, [1.0])


def test_binding_checks_host_buffers():
    """Buffers of the wrong size, type or device are refused before any call
    reaches the library (no read or write past a caller's buffer)."""
    import torch
    f = hsg._host_f32
    assert f([[1.0, 2.0, 3.0]], 3).dtype == np.float32
    with pytest.raises(ValueError):
        f(np.zeros(5, np.float32), 6)
    with pytest.raises(ValueError):
        f(np.zeros(6, np.float64), 6, out=True)          # an output must already be float32
    with pytest.raises(ValueError):
        f(np.zeros((6, 2), np.float32)[:, 0], 6, out=True)  # not contiguous
    with pytest.raises(ValueError):
        f(torch.zeros(6, dtype=torch.float64), 6)
    t = torch.zeros(6, dtype=torch.float32)
    assert f(t, 6) is t
