"""Host-side logic of bench.py (no GPU): workload tables, the algorithmic
byte and flop counts the roofline uses, and the synthetic inputs."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_workload_sizes():
    for name, w in bench.WORKLOADS.items():
        Ls = bench.sample_Ls(w)
        assert len(Ls) == w["S"], name
        assert all(L % 2 == 0 and L >= 4 for L in Ls), name
    c3 = bench.sample_Ls(bench.WORKLOADS["L8x256_L12x256_R32_f16"])
    assert c3.count(8) == 256 and c3.count(12) == 256
    assert bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["L"] == 64


def test_algorithmic_bytes_and_flops():
    # spins read + written (24 B) plus 3 bonds shared by R_share lattices
    assert bench.b_alg(64, 12) == pytest.approx(24.5625)
    assert bench.b_alg(48, 12) == pytest.approx(24.75)
    assert bench.b_alg(1, 24) == pytest.approx(96.0)
    assert bench.flops_per_update(8) == pytest.approx((148 + 8 * 128) / 9)
    assert bench.flops_per_update(0) == pytest.approx(148)
    assert bench.ALU_PEAK_TFLOPS == pytest.approx(148 * 128 * 2 * 2.032e-3)


def test_make_inputs_small_mixed_workload():
    w = dict(Ls=(4, 6), S=2, n_rep=2, NT=3, Tmin=0.2, Tmax=0.8, n_or=1, measure_every=1)
    samples, J, spins, beta = bench.make_inputs(w, rank=1)
    assert samples == [2, 3]                      # rank 1 takes the next samples
    assert J[0].shape == (4 ** 3, 3, 6) and J[1].shape == (6 ** 3, 3, 6)
    assert len(spins[1]) == 6 and spins[1][0].shape == (6 ** 3, 3)
    assert np.allclose(np.linalg.norm(spins[0][0], axis=1), 1, atol=1e-6)
    assert np.all(np.diff(beta) > 0)


def test_traffic_keys_name_known_kernels():
    for (h, wname, name), v in bench.NCU_TRAFFIC.items():
        assert len(h) == 16 and v > 0 and wname in bench.WORKLOADS
        assert name.startswith("k_sweep_fused") or name.startswith("k_persistent")
    # the entries are current: each names the hash of the sources as they stand
    hashes = {bench.kernel_source_hash(), bench.kernel_source_hash(bench.RESIDENT_SOURCES)}
    assert {h for h, _, _ in bench.NCU_TRAFFIC} <= hashes


def test_single_lattice_form_gives_every_lattice_its_own_couplings():
    w = dict(L=4, S=2, n_rep=1, NT=3, Tmin=0.2, Tmax=0.8, n_or=1, measure_every=1)
    inputs = bench.make_inputs(w, rank=0)
    samples, J, spins, beta = bench.single_lattice_inputs(inputs)
    assert samples == list(range(6)) and len(J) == 6 and all(len(s) == 1 for s in spins)
    # lattice j of sample s keeps its spins and its sample's coupling values
    assert np.array_equal(spins[4][0], inputs[2][1][1]) and np.array_equal(J[4], inputs[1][1])
    assert list(beta) == [2.0]
    ws = bench.WORKLOADS[bench.SINGLE_WORKLOAD]
    wd = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert ws["S"] == wd["S"] * wd["n_rep"] * wd["NT"] and ws["n_rep"] * ws["NT"] == 1 and ws["L"] == wd["L"]
    assert ws["prec"] == "f32" and ws["layout"] == "plain"


def test_workload_forms():
    class H:
        F16, F32, PLAIN, BATCHED = 1, 0, 0, 1
    assert bench.workload_form(H, bench.WORKLOADS["L8_S1_R2_f32"]) == (H.F32, H.PLAIN)
    assert bench.workload_form(H, bench.WORKLOADS["L16_S1_R32_f32"]) == (H.F32, H.BATCHED)
    assert bench.workload_form(H, bench.WORKLOADS[bench.DEFAULT_WORKLOAD]) == (H.F16, H.BATCHED)
    assert bench.spin_bytes(bench.WORKLOADS["L8_S1_R2_f32"]) == 12 * 2 * 512
    # couplings: one set per sample, 24 B per FP32 bond and 16 B per FP16 bond as stored
    assert bench.coupling_bytes(bench.WORKLOADS["L64_S16_R1_f32_plain"]) == 16 * 3 * 24 * 64 ** 3
    assert bench.coupling_bytes(bench.WORKLOADS["L64_S8_R64_f16"]) == 8 * 3 * 16 * 64 ** 3
    assert "couplings" in bench.workload_config("L64_S16_R1_f32_plain",
                                                bench.WORKLOADS["L64_S16_R1_f32_plain"], 1)["l2"]
