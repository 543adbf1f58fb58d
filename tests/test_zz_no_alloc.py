"""hsg_energy_noalloc -- the energy entry point that allocates nothing.

Some callers cannot let a library allocate device memory (fixed arenas,
allocator-free inner loops); this call takes caller-owned device buffers and
uses only a fixed working array inside the library.  These tests call it
through the C ABI and compare it with the context API's energies
(hsg_energy + hsg_get_energies) and with the FP64 oracle's energy of the same
spins and couplings, on two calls in a row and on a request that fills the
working array exactly, within the energy tolerance used by the other parity
tests; and check that bad buffers and a first call during stream capture are
refused before anything runs.

Kept in a file of its own, collected after every other test file.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import hsg_inputs as gi
import oracle
import paper_1309_1599_b300 as hsg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _scratch_doubles():
    """HSG_NOALLOC_SCRATCH_DOUBLES as include/hsg.h defines it."""
    with open(os.path.join(ROOT, "include", "hsg.h")) as f:
        for line in f:
            if line.startswith("#define HSG_NOALLOC_SCRATCH_DOUBLES"):
                return int(line.split()[2])
    raise AssertionError("HSG_NOALLOC_SCRATCH_DOUBLES not found")

pytestmark = pytest.mark.gpu

ENERGY_RTOL = 2e-6     # as in tests/test_gpu_parity.py


def _lib():
    lib = hsg.load_library()
    lib.hsg_energy_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.hsg_energy_noalloc.restype = ctypes.c_int
    return lib


def _context_energies(L, S, R, J, spins):
    betas = [1.0] if R == 1 else list(np.linspace(0.5, 2.0, R))
    lat = hsg.Lattice([L] * S, betas,
                      n_replicas=1, coupling_prec=hsg.F32, layout=hsg.PLAIN)
    for s in range(S):
        lat.set_couplings(s, J[s])
        for j in range(R):
            lat.set_spins(s, j, spins[s][j])
    lat.energy()
    E = lat.get_energies()
    lat.destroy()
    return E


def _device_buffers(torch, L, S, R, J, spins):
    N = L ** 3
    s_dev = torch.stack([torch.from_numpy(np.ascontiguousarray(spins[s][j].T))
                         for s in range(S) for j in range(R)]).cuda()          # [S*R][3][N]
    J_dev = torch.stack([torch.from_numpy(np.ascontiguousarray(J[s].transpose(1, 0, 2)))
                         for s in range(S)]).cuda()                             # [S][3][N][6]
    assert s_dev.shape == (S * R, 3, N) and J_dev.shape == (S, 3, N, 6)
    return s_dev, J_dev


def _call(lib, torch, s_dev, J_dev, L, S, R, E_dev):
    st = lib.hsg_energy_noalloc(ctypes.c_void_p(s_dev.data_ptr()), ctypes.c_void_p(J_dev.data_ptr()),
                                L, S, R, ctypes.c_void_p(E_dev.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.hsg_last_error().decode()


def test_noalloc_energies_match_context_api_two_calls():
    import torch
    lib = _lib()
    cases = [(12, 2, 3, 11), (8, 1, 4, 12)]       # (L, samples, lattices per sample, seed)
    for L, S, R, seed in cases:
        J = [gi.couplings(L, seed, s) for s in range(S)]
        spins = [[gi.random_spins(L, seed, s, j) for j in range(R)] for s in range(S)]
        ref = _context_energies(L, S, R, J, spins).reshape(-1)
        s_dev, J_dev = _device_buffers(torch, L, S, R, J, spins)
        E_dev = torch.full((S * R,), float("nan"), dtype=torch.float64, device="cuda")
        _call(lib, torch, s_dev, J_dev, L, S, R, E_dev)
        torch.cuda.synchronize()
        E = E_dev.cpu().numpy()
        assert np.all(np.abs(E - ref) <= ENERGY_RTOL * np.abs(ref)), (E, ref)
    # the second case ran right after the first on the same working array;
    # run the first case again to check nothing of the other call leaks in
    L, S, R, seed = cases[0]
    J = [gi.couplings(L, seed, s) for s in range(S)]
    spins = [[gi.random_spins(L, seed, s, j) for j in range(R)] for s in range(S)]
    ref = _context_energies(L, S, R, J, spins).reshape(-1)
    s_dev, J_dev = _device_buffers(torch, L, S, R, J, spins)
    E_dev = torch.zeros((S * R,), dtype=torch.float64, device="cuda")
    _call(lib, torch, s_dev, J_dev, L, S, R, E_dev)
    torch.cuda.synchronize()
    E = E_dev.cpu().numpy()
    assert np.all(np.abs(E - ref) <= ENERGY_RTOL * np.abs(ref)), (E, ref)


def _abs_scale(L, J6, s):
    """sum over bonds of |s_x^T J s_(x+mu)| (natural site order, periodic):
    the scale of an energy evaluated with FP32 terms.  For the random spins
    used here the energy itself is a sum of terms of either sign close to
    zero, so its rounding error is bounded relative to this sum, not to E."""
    sp = np.asarray(s, dtype=np.float64).reshape(L, L, L, 3)            # [z][y][x]
    J = np.asarray(J6, dtype=np.float64).reshape(L, L, L, 3, 6)
    tot = 0.0
    for mu, axis in ((0, 2), (1, 1), (2, 0)):
        t = np.roll(sp, -1, axis=axis)
        j = J[..., mu, :]
        Jt = np.stack([j[..., 0] * t[..., 0] + j[..., 3] * t[..., 1] + j[..., 4] * t[..., 2],
                       j[..., 3] * t[..., 0] + j[..., 1] * t[..., 1] + j[..., 5] * t[..., 2],
                       j[..., 4] * t[..., 0] + j[..., 5] * t[..., 1] + j[..., 2] * t[..., 2]], axis=-1)
        tot += np.abs((sp * Jt).sum(axis=-1)).sum()
    return tot


def test_noalloc_energies_match_oracle_two_calls():
    """Against the FP64 oracle's energy of the same spins and couplings
    directly (not through another CUDA path), on two calls in a row with
    different shapes: within ENERGY_RTOL of the sum of the absolute bond
    terms (the scale of FP32 rounding in the energy; it equals |E| in the
    ordered states of the other parity tests)."""
    import torch
    lib = _lib()
    for L, S, R, seed in [(10, 3, 2, 21), (16, 1, 5, 22)]:
        J = [gi.couplings(L, seed, s) for s in range(S)]
        spins = [[gi.random_spins(L, seed, s, j) for j in range(R)] for s in range(S)]
        s_dev, J_dev = _device_buffers(torch, L, S, R, J, spins)
        E_dev = torch.full((S * R,), float("nan"), dtype=torch.float64, device="cuda")
        _call(lib, torch, s_dev, J_dev, L, S, R, E_dev)
        torch.cuda.synchronize()
        E = E_dev.cpu().numpy().reshape(S, R)
        for s in range(S):
            J9 = oracle.j9_from_j6(J[s])
            for j in range(R):
                ref = oracle.energy(L, J9, spins[s][j].astype(np.float64))
                tol = ENERGY_RTOL * _abs_scale(L, J[s], spins[s][j])
                assert abs(E[s, j] - ref) <= tol, (L, s, j, E[s, j], ref, tol)


def test_noalloc_at_the_capacity_of_the_working_array():
    """A request that fills the working array exactly: L = 64, 8 samples x 64
    lattices (512 lattices x 512 partial sums = HSG_NOALLOC_SCRATCH_DOUBLES),
    several blocks per lattice and several samples interleaved.  Every energy
    against the context API on the same spins, sampled ones against the FP64
    oracle (tolerance relative to the sum of the absolute bond terms, as
    above)."""
    import torch
    lib = _lib()
    L, S, R, seed = 64, 8, 64, 23
    N = L ** 3
    assert S * R * ((N // 2 + 255) // 256) == _scratch_doubles()
    J = [gi.couplings(L, seed, s) for s in range(S)]
    g = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.randn(S * R, N, 3, device="cuda", generator=g)
    v = v / v.norm(dim=2, keepdim=True)                                   # [S*R][N][3]
    s_dev = v.transpose(1, 2).contiguous()                                # [S*R][3][N]
    J_dev = torch.stack([torch.from_numpy(np.ascontiguousarray(J[s].transpose(1, 0, 2)))
                         for s in range(S)]).cuda()
    E_dev = torch.full((S * R,), float("nan"), dtype=torch.float64, device="cuda")
    _call(lib, torch, s_dev, J_dev, L, S, R, E_dev)
    torch.cuda.synchronize()
    E = E_dev.cpu().numpy().reshape(S, R)
    lat = hsg.Lattice([L] * S, list(np.linspace(0.5, 2.0, R)), n_replicas=1, coupling_prec=hsg.F32,
                      layout=hsg.PLAIN)
    for s in range(S):
        lat.set_couplings(s, J[s])
        for j in range(R):
            lat.set_spins_device(s, j, v[s * R + j])
    lat.energy()
    ref = lat.get_energies()
    lat.destroy()
    assert np.all(np.abs(E - ref) <= ENERGY_RTOL * np.abs(ref)), np.abs(E - ref).max()
    for s, j in [(0, 0), (0, 63), (3, 17), (7, 0), (7, 63)]:
        sp = v[s * R + j].double().cpu().numpy()
        o = oracle.energy(L, oracle.j9_from_j6(J[s]), sp)
        tol = ENERGY_RTOL * _abs_scale(L, J[s], sp)
        assert abs(E[s, j] - o) <= tol, (s, j, E[s, j], o, tol)


def test_noalloc_rejects_bad_buffers_before_launching():
    """Buffers that are misaligned, host memory, or smaller than the sizes
    given are refused with HSG_EINVAL, and the output is left untouched."""
    import torch
    lib = _lib()
    L, S, R = 64, 1, 1                      # 3 MB of spins, more than a small tensor's 2 MB segment
    N = L ** 3
    s_dev = torch.zeros(S * R, 3, N, device="cuda")
    J_dev = torch.zeros(S * 3 * N * 6 + 2, device="cuda")              # room for a 4-byte offset
    E_dev = torch.full((S * R,), 7.0, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    host = np.zeros(S * R * 3 * N, dtype=np.float32)
    small = torch.zeros(10, device="cuda")
    cases = {
        "J6 misaligned": (s_dev.data_ptr(), J_dev.data_ptr() + 4, E_dev.data_ptr(), "aligned"),
        "spins in host memory": (host.ctypes.data, J_dev.data_ptr(), E_dev.data_ptr(), "spins"),
        "spins too small": (small.data_ptr(), J_dev.data_ptr(), E_dev.data_ptr(), "spins needs"),
    }
    for name, (sp, jp, ep, msg) in cases.items():
        st = lib.hsg_energy_noalloc(ctypes.c_void_p(sp), ctypes.c_void_p(jp), L, S, R, ctypes.c_void_p(ep), stream)
        assert st == 1, name                                            # HSG_EINVAL
        assert msg in lib.hsg_last_error().decode(), (name, lib.hsg_last_error())
    torch.cuda.synchronize()
    assert torch.all(E_dev == 7.0)


CAPTURE_SCRIPT = r"""
import ctypes, sys
import torch
sys.path.insert(0, sys.argv[1])
import paper_1309_1599_b300 as hsg
lib = hsg.load_library()
lib.hsg_energy_noalloc.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2
lib.hsg_energy_noalloc.restype = ctypes.c_int
L, N = 8, 512
s_dev = torch.zeros(2, 3, N, device="cuda")
J_dev = torch.zeros(1, 3, N, 6, device="cuda")
E_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
g, side = torch.cuda.CUDAGraph(), torch.cuda.Stream()
with torch.cuda.graph(g, stream=side):
    st = lib.hsg_energy_noalloc(ctypes.c_void_p(s_dev.data_ptr()), ctypes.c_void_p(J_dev.data_ptr()), L, 1, 2,
                                ctypes.c_void_p(E_dev.data_ptr()), ctypes.c_void_p(side.cuda_stream))
print("status", st, lib.hsg_last_error().decode())
st2 = lib.hsg_energy_noalloc(ctypes.c_void_p(s_dev.data_ptr()), ctypes.c_void_p(J_dev.data_ptr()), L, 1, 2,
                             ctypes.c_void_p(E_dev.data_ptr()), None)
torch.cuda.synchronize()
print("after", st2, float(E_dev.sum()))
"""


def test_noalloc_first_call_during_capture_is_refused():
    """In a fresh process, a first call on a stream being captured into a
    graph is refused with HSG_ESTATE and enqueues nothing; a call outside
    capture then works."""
    r = subprocess.run([sys.executable, "-c", CAPTURE_SCRIPT, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert lines[0].startswith("status 5 ") and "stream capture" in lines[0], r.stdout
    assert lines[1] == "after 0 0.0", r.stdout


def test_noalloc_rejects_requests_beyond_the_working_array():
    import torch
    lib = _lib()
    L = 64                                  # 512 partial sums per lattice
    too_many = 262144 // 512 + 1          # lattices: one more than fits
    dummy = torch.zeros(1, device="cuda")
    st = lib.hsg_energy_noalloc(ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                L, 1, too_many, ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 1                          # HSG_EINVAL, nothing launched
    assert "working array" in lib.hsg_last_error().decode()
