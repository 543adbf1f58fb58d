"""hsg_energy_noalloc -- the energy entry point that allocates nothing.

Some callers cannot let a library allocate device memory (fixed arenas,
allocator-free inner loops); this call takes caller-owned device buffers and
uses only a fixed working array inside the library.  These tests call it
through the C ABI and compare it with the context API's energies
(hsg_energy + hsg_get_energies) on the same spins and couplings, on two calls
in a row, within the energy tolerance used by the other parity tests.

Kept in a file of its own, collected after every other test file.
"""
import ctypes

import numpy as np
import pytest

import hsg_inputs as gi
import paper_1309_1599_b300 as hsg

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
