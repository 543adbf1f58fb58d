"""The bench's measured paths on a small workload, so that a change to the
library or the binding cannot break the throughput, roofline and end-to-end
legs unnoticed: streaming and resident forms, the end-to-end run through the
public API, and the JSON fields they feed."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

pytestmark = pytest.mark.gpu

SMALL = dict(Ls=(8,) * 4 + (12,) * 4, S=8, n_rep=2, NT=4, Tmin=0.2, Tmax=0.8, n_or=2, measure_every=2,
             persistent=True)
STREAM = dict(L=24, S=2, n_rep=2, NT=4, Tmin=0.2, Tmax=0.8, n_or=2, measure_every=2)


@pytest.fixture()
def env(monkeypatch):
    import torch
    import paper_1309_1599_b300 as hsg
    monkeypatch.setitem(bench.WORKLOADS, "test_small", SMALL)
    monkeypatch.setitem(bench.WORKLOADS, "test_stream", STREAM)
    return hsg, torch, bench.Dist(1, 0, 0, "nccl"), bench.measured_peaks()


def test_streaming_form_and_roofline(env):
    hsg, torch, dist, peak = env
    inputs = bench.make_inputs(STREAM, 0)
    r = bench.run_form(hsg, torch, dist, "test_stream", inputs, hsg.F16, hsg.BATCHED, 2, 1, None, peak)
    r["lat"].destroy()
    roof = r["roofline"]
    assert r["value"] > 0 and r["launches"] > 0
    assert roof["bound"] == "hbm" and 0 < roof["frac"] and roof["unit"] == "GB/s"
    assert roof["tiling"]["24"]["launches_per_sweep"] in (1, 2)


def test_resident_form_and_roofline(env):
    hsg, torch, dist, peak = env
    inputs = bench.make_inputs(SMALL, 0)
    r = bench.run_form(hsg, torch, dist, "test_small", inputs, hsg.F16, hsg.BATCHED, 2, 1, None, peak,
                       persistent=True)
    roof = r["roofline"]
    assert r["value"] > 0 and roof["bound"] == "alu" and roof["launches_per_10_mcs"] >= 2
    assert set(roof["tiling"]) == {"8", "12"}


def test_end_to_end_through_the_public_api(env):
    hsg, torch, dist, peak = env
    inputs = bench.make_inputs(STREAM, 0)
    e = bench.e2e_run(hsg, torch, dist, STREAM, inputs, 2)
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
