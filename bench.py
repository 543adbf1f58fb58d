#!/usr/bin/env python
"""Throughput of the Heisenberg spin-glass Monte Carlo on one B300 (or N, as
independent replicas): spin updates/ns of the batched FP16-coupling form,
with the plain FP32 form, the bimodal one-byte-coupling forms (plain and
batched), the HBM roofline fraction of the dominant kernel, an end-to-end
figure through the public API from host buffers, and the FP64 oracle on the
host cores as a CPU baseline.

Workload (default): L = 64, 8 disorder samples per GPU, 32 temperatures evenly
spaced in [0.15, 0.75] x 2 replicas (64 lattices per sample, 512 per GPU),
Gaussian couplings quantised to FP16, FP32 spins.  One Monte Carlo step (MCS)
is 1 heat-bath sweep + 8 overrelaxation sweeps + energies + one PT sweep; the
observables are measured every 10 MCS.  One bench step = 10 MCS, so every
step runs every stage of the path.  The spins (1.6 GB per GPU) exceed L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hsg|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin updates/ns and % HBM roofline, batched FP16-coupling vs plain FP32 (1 B300)"
UNIT = "spin updates/ns"
MCS_PER_STEP = 10

# Coupling storage ("prec": "f16" unless given) and spin layout ("layout":
# "batched", two lattices per element, unless given) of each workload.
WORKLOADS = {
    "L64_S8_R64_f16": dict(L=64, S=8, n_rep=2, NT=32, Tmin=0.15, Tmax=0.75, n_or=8,
                           measure_every=10),
    # the plain method at L=8: one sample, 2 replicas at T = 0.5, FP32
    # couplings, one lattice per element, observables every step (no PT)
    "L8_S1_R2_f32": dict(L=8, S=1, n_rep=2, NT=1, Tmin=0.5, Tmax=0.5, n_or=8, measure_every=1,
                         prec="f32", layout="plain"),
    # one L=16 sample with PT over 16 temperatures in [0.15, 0.75] x 2
    # replicas, FP32 couplings, observables every 10 steps
    "L16_S1_R32_f32": dict(L=16, S=1, n_rep=2, NT=16, Tmin=0.15, Tmax=0.75, n_or=8,
                           measure_every=10, prec="f32"),
    "L32_S64_R48_f16": dict(L=32, S=64, n_rep=2, NT=24, Tmin=0.15, Tmax=0.75, n_or=8,
                            measure_every=10),
    # the plain single-lattice form at L=64: 512 samples of one lattice each at
    # T = 0.5, FP32 couplings of their own (no two lattices share a coupling
    # read), one lattice per element; the default run builds it from its own
    # inputs (each lattice with its own copy of its sample's couplings)
    "L64_S512_R1_f32_plain": dict(L=64, S=512, n_rep=1, NT=1, Tmin=0.5, Tmax=0.5, n_or=8, measure_every=10,
                                  prec="f32", layout="plain"),
    # profiling size of the plain single-lattice form: 16 lattices of L=64,
    # each with FP32 couplings of its own (302 MB of couplings, above L2)
    "L64_S16_R1_f32_plain": dict(L=64, S=16, n_rep=1, NT=1, Tmin=0.5, Tmax=0.5, n_or=8, measure_every=10,
                                 prec="f32", layout="plain"),
    # profiling size: 512 lattices of L=32 (201 MB of spins, above L2)
    "L32_S8_R64_f16": dict(L=32, S=8, n_rep=2, NT=32, Tmin=0.15, Tmax=0.75, n_or=8,
                           measure_every=10),
    # profiling size of the L=64 tiling: one sample, 64 lattices (201 MB of spins)
    "L64_S1_R64_f16": dict(L=64, S=1, n_rep=2, NT=32, Tmin=0.15, Tmax=0.75, n_or=8,
                           measure_every=10),
    # many small lattices of mixed L, every replica set resident in shared
    # memory (4 replicas x 8 temperatures per sample), both sizes in one
    # launch per stretch of steps
    "L8x256_L12x256_R32_f16": dict(Ls=(8,) * 256 + (12,) * 256, S=512, n_rep=4, NT=8, Tmin=0.2,
                                   Tmax=0.8, n_or=8, measure_every=10, persistent=2),
    # mid-size lattices: a replica set (393 KB) is larger than shared memory,
    # so each CTA holds one lattice group for one step and PT runs between
    "L16_S512_R32_f16": dict(L=16, S=512, n_rep=2, NT=16, Tmin=0.15, Tmax=0.75, n_or=8,
                             measure_every=10, persistent=True),
}
DEFAULT_WORKLOAD = "L64_S8_R64_f16"
# the plain single-lattice form timed beside the default workload
SINGLE_WORKLOAD = "L64_S512_R1_f32_plain"
# the small- and mid-size-lattice workloads summarised in every run of another workload
SMALL_WORKLOAD = "L8x256_L12x256_R32_f16"
MID_WORKLOAD = "L16_S512_R32_f16"

# DRAM bytes per launch of the dominant kernel from an ncu capture, keyed by a
# hash of the device sources that kernel is built from (stale -> null), the
# workload and the kernel.
FUSED_SOURCES = ("kernels.cuh", "fused.cuh", "philox.cuh")
RESIDENT_SOURCES = ("kernels.cuh", "persistent.cuh", "philox.cuh")
NCU_TRAFFIC = {
    # the L=64 overrelaxation sweep in 8-row bands: 387.9 MB for one sample of
    # 64 lattices, x8 samples
    ("e85d062003519016", "L64_S8_R64_f16", "k_sweep_fused<OR,2,f16> (bands of 8 rows)"): 3103438848,
    # the same sweep of the plain FP32 form (one lattice per element): 418.2 MB
    # for one sample, x8 samples; the 64 lattices of a sample read their
    # shared couplings through L2, so this is far below the 96 B per update
    # that lattices with couplings of their own move
    ("e85d062003519016", "L64_S8_R64_f16", "k_sweep_fused<OR,1,f32> (bands of 8 rows)"): 3345754112,
    # the plain single-lattice form (FP32 couplings of its own per lattice):
    # 365.0 MB read + 42.2 MB written for 16 lattices (97.1 B per update
    # against the algorithmic 96), x32 for the 512 lattices timed beside the
    # default workload
    ("e85d062003519016", "L64_S16_R1_f32_plain", "k_sweep_fused<OR,1,f32> (bands of 8 rows)"): 407172608,
    ("e85d062003519016", "L64_S512_R1_f32_plain", "k_sweep_fused<OR,1,f32> (bands of 8 rows)"): 13029523456,
    # the L=32 overrelaxation sweep: one launch of 64 samples x 48 lattices
    ("e85d062003519016", "L32_S64_R48_f16", "k_sweep_fused<OR,2,f16> (bands of 8 rows)"): 2644966144,
    # the resident steps of 256 x L=8 + 256 x L=12 samples, both sizes in one
    # launch of 10 MCS: 249.3 MB read + 163.8 MB written
    ("629648d1f094eef9", "L8x256_L12x256_R32_f16",
     "k_persistent_pair<2,f16> (10 MCS per launch, both lattice sizes in one launch)"): 413147648,
}


def sample_Ls(w):
    """Linear size of each sample of the workload."""
    return list(w["Ls"]) if "Ls" in w else [w["L"]] * w["S"]


def workload_form(hsg, w):
    """(coupling storage, spin layout) of the workload's own form."""
    prec = {"f16": hsg.F16, "f32": hsg.F32}[w.get("prec", "f16")]
    layout = hsg.PLAIN if w.get("layout") == "plain" else hsg.BATCHED
    return prec, layout


def spin_bytes(w):
    return 12 * w["n_rep"] * w["NT"] * sum(L ** 3 for L in sample_Ls(w))


def coupling_bytes(w):
    """Device bytes of the workload's couplings (one set per sample: 16 B per
    bond for FP16 as stored, 24 B for FP32)."""
    per_bond = 16 if w.get("prec", "f16") == "f16" else 24
    return 3 * per_bond * sum(L ** 3 for L in sample_Ls(w))


def kernel_source_hash(files=FUSED_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1309_1599_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# Peak of the FP32 pipe: 148 SMs x 128 FP32 lanes x 2 flops (FMA) x 2032 MHz.
ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# Algorithmic FP32 flops per site update: the local field is 18 FMA per bond
# direction pair (6 3x3 matrix-vector products = 54 FMA = 108 flops); an
# overrelaxation adds h.h, h.s, the ratio and s' = c h - s (20 flops), a
# heat-bath draw the kappa, inverse-CDF and rotation arithmetic (40 flops,
# transcendentals counted once each).
FLOPS_OR, FLOPS_HB = 128, 148


def flops_per_update(n_or: int) -> float:
    return (FLOPS_HB + n_or * FLOPS_OR) / (1 + n_or)


def b_alg(R_share: int, bond_bytes: int) -> float:
    """Algorithmic bytes per site update: each spin (12 B) read and written
    once per sweep, each bond's bond_bytes read once per sweep for all
    R_share lattices that share it (3 bonds per site)."""
    return 2 * 12 + 3 * bond_bytes / R_share


# ----------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, world, rank, local, backend):
        import torch
        self.world, self.rank, self.local = world, rank, local
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist
        self.torch = torch

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64,
                              device="cuda" if self.torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------
# inputs
# ----------------------------------------------------------------------------
def make_inputs(w, rank, seed=1, n_samples=None):
    """Seeded inputs of this rank's samples (the first n_samples of them if
    given)."""
    import hsg_inputs as gi
    Ls, S, R = sample_Ls(w), w["S"], w["n_rep"] * w["NT"]
    samples = [rank * S + s for s in range(S if n_samples is None else min(S, n_samples))]
    J = [gi.couplings(Ls[s], seed, sg, precision=w.get("prec", "f16")) for s, sg in enumerate(samples)]
    spins = [[gi.random_spins(Ls[s], seed, sg, j) for j in range(R)] for s, sg in enumerate(samples)]
    beta = gi.linear_betas(w["Tmin"], w["Tmax"], w["NT"])
    return samples, J, spins, beta


def single_lattice_inputs(inputs):
    """The default workload's lattices as samples of one lattice each (at
    T = 0.5), each given its own device copy of its sample's couplings: the
    same values, but every lattice reads its couplings from an address of its
    own, as lattices with distinct couplings do."""
    samples, J, spins, beta = inputs
    flat = [(s, j) for s in range(len(samples)) for j in range(len(spins[s]))]
    return (list(range(len(flat))), [J[s] for s, _ in flat], [[spins[s][j]] for s, j in flat],
            np.array([1.0 / 0.5]))


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# the hsg arm
# ----------------------------------------------------------------------------
# Magnitude of the anisotropy of the bimodal forms (the paper uses 0.5 and 1).
BIMODAL_D = 1.0


def philox_key(rank: int) -> int:
    """Random-number key of a rank's context: the contexts of different ranks
    number their samples from 0, so distinct keys keep the replicas'
    random streams independent."""
    return 1 + rank


def build_lattice(hsg, w, samples, J, spins, beta, prec, layout, seed=1, band_rows=0,
                  persistent=False, key=1, fused_groups=0):
    import hsg_inputs as gi
    Ls = sample_Ls(w)
    lat = hsg.Lattice(Ls, beta, n_replicas=w["n_rep"], coupling_prec=prec,
                      layout=layout, n_or=w["n_or"], measure_every=w["measure_every"], seed=key,
                      band_rows=band_rows, persistent=persistent, bimodal_D=BIMODAL_D,
                      fused_groups=fused_groups)
    for s in range(len(samples)):
        if prec == hsg.BIMODAL:
            lat.set_couplings_bimodal(s, gi.bimodal_bits(Ls[s], seed, samples[s]))
        else:
            lat.set_couplings(s, J[s])
        lat.set_spins_sample(s, np.stack(spins[s]))
    if band_rows == 0 and fused_groups == 0:
        lat.autotune()                 # launch shapes timed on this data, outside any timed region
    return lat


def time_steps(lat, steps, torch, dist, sampler=None):
    """Device time of `steps` bench steps (10 MCS each), CUDA events on the
    stream the library launches on, barrier + synchronize on both sides."""
    stream = torch.cuda.current_stream()
    dist.barrier()
    torch.cuda.synchronize()
    l0 = lat.get_launch_count()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lat.run_steps(MCS_PER_STEP)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    dist.barrier()
    ms = e0.elapsed_time(e1)
    return ms, lat.get_launch_count() - l0, clocks


def time_or_kernel(lat, torch, n_calls=4, sweeps=8):
    """Average duration of one overrelaxation sweep-kernel launch (the
    dominant kernel: one fused sweep, or one colour half-sweep), from CUDA
    events around sweep_or calls on the library's stream."""
    stream = torch.cuda.current_stream()
    lat.sweep_or(sweeps)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_calls):
        lat.sweep_or(sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    per_sweep = lat.get_sweep_plan(0)["launches_per_sweep"]
    return e0.elapsed_time(e1) / (n_calls * per_sweep * sweeps)


def time_persistent_kernel(hsg, w, inputs, torch, n_calls=3, mode=1):
    """Device time of the resident steps for 10 whole MCS without
    measurement, from CUDA events on the library's stream: one launch per
    distinct L plus a counter bump of ~2 us, or, where replica sets span
    several CTAs, per MCS one launch per L, the PT sweep and the bump.
    With mode 2 both lattice sizes share one launch.
    Returns (ms per 10 MCS, launches per 10 MCS)."""
    samples, J, spins, beta = inputs
    wk = dict(w, measure_every=0)
    lat = build_lattice(hsg, wk, samples, J, spins, beta, hsg.F16, hsg.BATCHED, persistent=mode)
    stream = torch.cuda.current_stream()
    lat.run_steps(MCS_PER_STEP)
    torch.cuda.synchronize()
    l0 = lat.get_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_calls):
        lat.run_steps(MCS_PER_STEP)
    e1.record(stream)
    torch.cuda.synchronize()
    n_kernels = (lat.get_launch_count() - l0) // n_calls
    lat.destroy()
    return e0.elapsed_time(e1) / n_calls, n_kernels


def time_sequential_or(hsg, w, inputs, torch, n_calls=3):
    """Sequential overrelaxation sweeps (App. A.1, sites in natural order,
    executed by hyperplanes x+y+z) of the whole workload: updates/ns and ms
    per sweep, CUDA events on the library's stream."""
    samples, J, spins, beta = inputs
    lat = build_lattice(hsg, w, samples, J, spins, beta, hsg.F16, hsg.BATCHED)
    stream = torch.cuda.current_stream()
    lat.sweep_or_sequential(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_calls):
        lat.sweep_or_sequential(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n_calls
    upd = lat.R * sum(L ** 3 for L in sample_Ls(w))
    lat.destroy()
    return {"value": round(upd / (ms * 1e6), 3), "unit": UNIT, "ms_per_sweep": round(ms, 4),
            "kernel": "k_sweep_or_seq<2,f16> (hyperplanes x+y+z, one lattice pair per CTA)"}


def run_form(hsg, torch, dist, wname, inputs, prec, layout, steps, warmup, sampler, peak, band_rows=0,
             persistent=False, fused_groups=0):
    w = WORKLOADS[wname]
    samples, J, spins, beta = inputs
    lat = build_lattice(hsg, w, samples, J, spins, beta, prec, layout, band_rows=band_rows,
                        persistent=persistent, key=philox_key(dist.rank), fused_groups=fused_groups)
    R = lat.R
    n_sites = sum(L ** 3 for L in sample_Ls(w))
    # the autotuned launch shapes, one entry per lattice size
    first = {L: s for s, L in reversed(list(enumerate(sample_Ls(w))))}
    tiling = {str(L): (lat.get_resident_plan(s) if persistent else lat.get_sweep_plan(s))
              for L, s in sorted(first.items())}
    for _ in range(warmup):
        lat.run_steps(MCS_PER_STEP)
    torch.cuda.synchronize()
    ms, launches, clocks = time_steps(lat, steps, torch, dist, sampler)
    ms_max = dist.max(ms)
    updates_rank = R * n_sites * (1 + w["n_or"]) * MCS_PER_STEP * steps
    value = updates_rank * dist.world / (ms_max * 1e6)
    if persistent:
        lat.destroy()
        k_ms, n_kernels = time_persistent_kernel(hsg, w, inputs, torch, mode=int(persistent))
        upd = R * n_sites * (1 + w["n_or"]) * MCS_PER_STEP
        fpu = flops_per_update(w["n_or"])
        achieved = upd * fpu / (k_ms * 1e-3) / 1e12
        vname = 2 if layout == hsg.BATCHED else 1
        # replica sets that span several CTAs run one MCS per launch, PT between
        split = any(t["groups_per_cta"] * vname < w["NT"] for t in tiling.values())
        one_launch = any(t.get("one_launch") for t in tiling.values())
        n_res = (1 if one_launch else len(tiling)) * (MCS_PER_STEP if split else 1)
        kname = (f"k_persistent<{vname},f16> (1 MCS per launch, parts of replica sets, PT kernel between)" if split
                 else f"k_persistent_pair<{vname},f16> ({MCS_PER_STEP} MCS per launch, both lattice sizes in one launch)"
                 if one_launch
                 else f"k_persistent<{vname},f16> ({MCS_PER_STEP} MCS per launch, one launch per L)")
        roof = {"bound": "alu", "kernel": kname,
                "achieved": round(achieved, 2), "peak": round(ALU_PEAK_TFLOPS, 2),
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x 2032 MHz",
                "unit": "TFLOP/s", "frac": round(achieved / ALU_PEAK_TFLOPS, 4),
                "flops_per_update": round(fpu, 2), "launch_ms": round(k_ms / n_res, 4),
                "launches_per_10_mcs": n_kernels, "ms_per_10_mcs": round(k_ms, 4),
                "updates_per_ns_kernel": round(upd / (k_ms * 1e6), 2),
                "traffic": None, "tiling": tiling}
        # DRAM bytes of the resident launches of 10 MCS
        roof["traffic"] = NCU_TRAFFIC.get((kernel_source_hash(RESIDENT_SOURCES), wname, roof["kernel"]))
        return dict(value=value, ms_per_step=ms_max / steps, launches=launches, clocks=clocks,
                    roofline=roof, lat=None)
    or_ms = time_or_kernel(lat, torch)
    bond_bytes = {hsg.F16: 12, hsg.F32: 24, hsg.BIMODAL: 1}[prec]
    r_share = R if layout == hsg.BATCHED else 1
    balg = b_alg(r_share, bond_bytes)
    plan = lat.get_sweep_plan(0)
    # updates per launch: every site (fused sweep) or half of them (half-sweep)
    upd_launch = R * n_sites // plan["launches_per_sweep"]
    bytes_launch = upd_launch * balg
    achieved = bytes_launch / (or_ms * 1e-3) / 1e9
    vname = 2 if layout == hsg.BATCHED else 1
    pname = {hsg.F16: "f16", hsg.F32: "f32", hsg.BIMODAL: "bimodal"}[prec]
    gps = ", 2 lattice groups per thread" if plan.get("groups_per_thread_or", 1) == 2 else ""
    kname = (f"k_sweep_fused<OR,{vname},{pname}> (bands of {plan['band_rows']} rows{gps})" if plan["fused"]
             else f"k_sweep_half<OR,{vname},{pname}>")
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": round(achieved, 1), "peak": peak[0], "peak_source": peak[1],
            "unit": "GB/s", "frac": round(achieved / peak[0], 4),
            "b_alg_bytes_per_update": round(balg, 4),
            "bytes_per_launch": int(bytes_launch), "launch_ms": round(or_ms, 4),
            "updates_per_ns_roofline": round(peak[0] / balg, 2),
            "traffic": None, "tiling": tiling}
    key = (kernel_source_hash(), wname, roof["kernel"])
    if key in NCU_TRAFFIC:
        roof["traffic"] = NCU_TRAFFIC[key]
    out = dict(value=value, ms_per_step=ms_max / steps, launches=launches, clocks=clocks,
               roofline=roof, lat=lat)
    return out


def e2e_run(hsg, torch, dist, w, inputs, steps):
    """Whole job through the public API from pinned host buffers: couplings and
    initial spins host->device, `steps` bench steps each followed by a read of
    the observables (the step's result) to the host, and the final spins
    device->host.  Wall time around it, synchronised."""
    samples, J, spins, beta = inputs
    Ls, S = sample_Ls(w), len(samples)
    prec, layout = workload_form(hsg, w)
    lat = hsg.Lattice(Ls, beta, n_replicas=w["n_rep"], coupling_prec=prec,
                      layout=layout, n_or=w["n_or"], measure_every=w["measure_every"],
                      persistent=w.get("persistent", False), seed=philox_key(dist.rank))
    R, n_sites = lat.R, sum(L ** 3 for L in Ls)
    lat.autotune()                     # the shapes tuned for this workload (remembered)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    J_h = [pin(j) for j in J]
    s_h = [pin(np.stack(row)) for row in spins]            # [R][N][3] per sample
    out_h = [torch.empty((R, Ls[s] ** 3, 3), dtype=torch.float32).pin_memory() for s in range(S)]
    lat.run_steps(1)                   # capture graphs outside the timed region
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for s in range(S):
        lat.set_couplings(s, J_h[s])
        lat.set_spins_sample(s, s_h[s])
    for _ in range(steps):
        lat.run_steps(MCS_PER_STEP)
        obs, counts = lat.read_observables()
    for s in range(S):
        lat.get_spins_sample(s, out=out_h[s])
    torch.cuda.synchronize()
    dt = dist.max(time.perf_counter() - t0)
    lat.destroy()
    updates = R * n_sites * (1 + w["n_or"]) * MCS_PER_STEP * steps * dist.world
    h2d = sum(x.numel() * 4 for x in J_h) + R * n_sites * 12
    d2h = (obs.nbytes + counts.nbytes) * steps + R * n_sites * 12
    return {"value": updates / (dt * 1e9), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / steps), "d2h_bytes_per_step": int(d2h / steps),
            "wall_s": round(dt, 3)}


# ----------------------------------------------------------------------------
# the oracle on the host cores
# ----------------------------------------------------------------------------
def oracle_sample_run(w, inputs, n_mcs, threads):
    """The FP64 oracle on one sample (R lattices) of the workload for n_mcs
    Monte Carlo steps; returns (updates, seconds)."""
    import oracle
    samples, J, spins, beta = inputs
    L = sample_Ls(w)[0]
    smp = oracle.Sample(L, J[0], np.stack(spins[0]), beta, w["n_rep"], 1,
                        sample_index=samples[0])
    t0 = time.perf_counter()
    smp.run(n_mcs, w["n_or"], w["measure_every"], n_threads=threads)
    dt = time.perf_counter() - t0
    return smp.R * L ** 3 * (1 + w["n_or"]) * n_mcs, dt


def cpu_baseline(w, inputs, budget_s=15.0):
    threads = os.cpu_count() or 1
    ups, dt = oracle_sample_run(w, inputs, 1, threads)
    n = 1
    while dt < budget_s / 3 and n < 4096:
        more = max(1, int(n * (budget_s / max(dt, 1e-3) - 1)))
        u2, d2 = oracle_sample_run(w, inputs, more, threads)
        ups, dt, n = ups + u2, dt + d2, n + more
    cq = "FP16-quantised" if w.get("prec", "f16") == "f16" else "FP32"
    return {"value": ups / (dt * 1e9), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} MCS of 1 sample ({w['n_rep'] * w['NT']} lattices of L={sample_Ls(w)[0]}, "
                      f"{cq} couplings as FP64), OpenMP over lattices, "
                      f"{dt:.1f} s"}


def oracle_error(hsg, w, inputs):
    """Error of the GPU form against the FP64 oracle on sample 0 of the
    workload (the couplings as stored, the oracle computing in FP64 on the
    identical values), per stage:
      * one overrelaxation sweep from an identical state: the largest spin
        difference over four sampled lattices (trajectories under identical
        streams separate only over many sweeps, so this is the per-sweep
        arithmetic error);
      * after one Monte Carlo step, the fused energies against the oracle's
        energy of the same spins, and one measurement of every observable
        against the oracle's measurement of the same spins and labels: the
        largest difference over the temperatures relative to the largest
        magnitude of that observable.
    Part of the CPU-baseline leg (the oracle on the timed sample).  The
    long-run averages are compared statistically by the GPU test suite."""
    import oracle
    samples, J, spins, beta = inputs
    L = sample_Ls(w)[0]
    N, NT, n_rep = L ** 3, w["NT"], w["n_rep"]
    prec, layout = workload_form(hsg, w)
    lat = hsg.Lattice([L], beta, n_replicas=n_rep, coupling_prec=prec, layout=layout,
                      n_or=w["n_or"], measure_every=0, seed=1)
    lat.set_couplings(0, J[0])
    lat.set_spins_sample(0, np.stack(spins[0]))
    J9 = oracle.j9_from_j6(J[0])
    R = lat.R
    before = lat.get_spins_sample(0).astype(np.float64)
    lat.sweep_or(1)
    after = lat.get_spins_sample(0)
    ds = 0.0
    for j in sorted({0, 1, R // 2, R - 1}):
        ref = np.ascontiguousarray(before[j])
        oracle.sweep(L, J9, ref, oracle.OR)
        ds = max(ds, float(np.abs(after[j] - ref).max()))
    lat.run_steps(1)
    lat.reset_observables()
    lat.measure()
    obs, _ = lat.read_observables()
    E, perm = lat.get_energies(), lat.get_perm()
    st = lat.get_spins_sample(0).astype(np.float64)
    lat.destroy()
    ref = np.zeros((NT, hsg.NOBS))
    e_err = 0.0
    for k in range(NT):
        for r in range(n_rep):
            slot = perm[0, r, k]
            e = oracle.energy(L, J9, st[slot])
            e_err = max(e_err, abs(E[0, slot] - e) / abs(e))
            ref[k, 0] += e / N
            ref[k, 1] += (e / N) ** 2
            ref[k, 8] += oracle.sd_residual(L, J9, st[slot], 1 / beta[k])
        for pr in range(n_rep // 2):
            ref[k, 2:8] += oracle.measure_pair(L, st[perm[0, 2 * pr, k]], st[perm[0, 2 * pr + 1, k]])
    rel = {}
    for j, name in enumerate(oracle.OBS_NAMES):
        scale = float(np.abs(ref[:, j]).max())
        if j >= 2 and j < 8 and n_rep < 2:
            continue
        rel[name] = float(f"{np.abs(obs[0, :, j] - ref[:, j]).max() / scale:.3g}") if scale > 0 else None
    return {"sample": f"sample 0 ({R} lattices of L={L}, {w.get('prec', 'f16').upper()} couplings)",
            "or_sweep_max_abs_ds": float(f"{ds:.3g}"),
            "energy_max_rel_diff": float(f"{e_err:.3g}"),
            "measurement_max_rel_diff": rel}


def workload_config(name, w, world):
    """The `config` object of the JSON line: the workload and its shape."""
    persistent = w.get("persistent", False)
    return {"workload": name,
            "L": w["L"] if "L" in w else sorted(set(sample_Ls(w))),
            "samples_per_gpu": w["S"],
            "lattices_per_sample": w["n_rep"] * w["NT"], "n_temps": w["NT"],
            "T_range": [w["Tmin"], w["Tmax"]], "n_or": w["n_or"],
            "couplings": ("gaussian, FP16-quantised" if w.get("prec", "f16") == "f16" else
                          "gaussian, FP32"),
            "layout": w.get("layout", "batched"),
            "step": f"{MCS_PER_STEP} MCS (HB + {w['n_or']} OR + PT each) + 1 measurement",
            "l2": ("no flush: spins stay in shared memory within a launch; "
                   f"the whole set ({spin_bytes(w) / 1e6:.0f} MB per GPU) exceeds L2" if persistent else
                   "no flush: spins per GPU exceed L2 (126 MB)" if spin_bytes(w) > 126e6 else
                   f"no flush: spins and couplings per GPU ({(spin_bytes(w) + coupling_bytes(w)) / 1e6:.0f} MB) "
                   "exceed L2 (126 MB)" if spin_bytes(w) + coupling_bytes(w) > 126e6 else
                   f"no flush: the whole state ({spin_bytes(w) / 1e3:.0f} KB of spins) stays in L2 in any "
                   "run of this size; the workload is latency-bound and not graded against HBM"),
            "resident": bool(persistent),
            **({"resident_launches": "both lattice sizes in one launch per stretch of steps"}
               if persistent == 2 else {}),
            "parallelism": f"replicas x{world} (independent samples per GPU)"}


def reference_arm(args, w, world, rank, local):
    if rank != 0:
        return 0
    inputs = make_inputs(w, 0, n_samples=1)
    threads = os.cpu_count() or 1
    times, ups = [], 0
    for i in range(args.warmup + args.steps):
        u, dt = oracle_sample_run(w, inputs, 1, threads)
        if i >= args.warmup:
            times.append(dt)
            ups += u
    total = sum(times)
    value = ups / (total * 1e9)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args.workload, w, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                             "sample": f"each step: 1 MCS of sample 0 ({w['n_rep'] * w['NT']} lattices "
                                       f"of L={sample_Ls(w)[0]}), a bounded sample of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hsg", choices=["hsg", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run")
    ap.add_argument("--no-bimodal", action="store_true", help="skip the bimodal-coupling forms")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the summary of the small-lattice workload (resident steps)")
    ap.add_argument("--band-rows", type=int, default=0,
                    help="rows per CTA band of the fused sweep (0: library choice)")
    ap.add_argument("--fused-groups", type=int, default=0,
                    help="lattice groups per thread of the fused sweeps (0: library choice)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, w, world, rank, local)

    import torch
    import paper_1309_1599_b300 as hsg
    torch.cuda.set_device(local)
    dist = Dist(world, rank, local, "nccl")
    peak = measured_peaks()
    inputs = make_inputs(w, rank)

    sampler = ClockSampler(local)
    persistent = w.get("persistent", False)
    wprec, wlayout = workload_form(hsg, w)
    # the plain FP32 and bimodal comparisons and the small- and mid-lattice
    # summaries go with the streaming FP16 batched workloads
    f16_streaming = (wprec == hsg.F16 and wlayout == hsg.BATCHED and not persistent)
    batched = run_form(hsg, torch, dist, args.workload, inputs, wprec, wlayout, args.steps,
                       args.warmup, sampler, peak, band_rows=args.band_rows, persistent=persistent,
                       fused_groups=args.fused_groups)
    if batched["lat"] is not None:
        batched["lat"].destroy()
    streaming = None
    sequential = None
    joint = None
    if persistent:
        sequential = time_sequential_or(hsg, w, inputs, torch)
        if persistent == 2:
            # the same resident steps with one launch per lattice size
            joint = run_form(hsg, torch, dist, args.workload, inputs, wprec, wlayout, args.steps, args.warmup, None,
                             peak, persistent=1)
        # the same workload through the streaming kernels, for comparison
        streaming = run_form(hsg, torch, dist, args.workload, inputs, hsg.F16, hsg.BATCHED, args.steps,
                             args.warmup, None, peak)
        streaming["lat"].destroy()
    plain = single = None
    if not args.no_plain and f16_streaming:
        plain = run_form(hsg, torch, dist, args.workload, inputs, hsg.F32, hsg.PLAIN, args.steps,
                         args.warmup, None, peak)
        plain["lat"].destroy()
        if args.workload == DEFAULT_WORKLOAD:
            single = run_form(hsg, torch, dist, SINGLE_WORKLOAD, single_lattice_inputs(inputs), hsg.F32,
                              hsg.PLAIN, args.steps, args.warmup, None, peak)
            single["lat"].destroy()
    bimodal = {}
    if not args.no_bimodal and f16_streaming:
        for key, layout in (("bimodal_plain", hsg.PLAIN), ("bimodal_batched", hsg.BATCHED)):
            r = run_form(hsg, torch, dist, args.workload, inputs, hsg.BIMODAL, layout, args.steps, args.warmup,
                         None, peak)
            r["lat"].destroy()
            bimodal[key] = {"value": round(r["value"], 3), "ms_per_step": round(r["ms_per_step"], 3),
                            "D": BIMODAL_D, "roofline": r["roofline"], "gpu_launches": r["launches"]}
    small = mid = None
    if not args.no_small and f16_streaming:
        # many small lattices: resident steps against the streaming kernels,
        # and the sequential overrelaxation sweep, on the same inputs
        ws = WORKLOADS[SMALL_WORKLOAD]
        inputs_s = make_inputs(ws, rank)
        k = max(2, args.steps // 2)
        res = run_form(hsg, torch, dist, SMALL_WORKLOAD, inputs_s, hsg.F16, hsg.BATCHED, k, args.warmup, None, peak,
                       persistent=ws["persistent"])
        one = run_form(hsg, torch, dist, SMALL_WORKLOAD, inputs_s, hsg.F16, hsg.BATCHED, k, args.warmup, None, peak,
                       persistent=1)
        strm = run_form(hsg, torch, dist, SMALL_WORKLOAD, inputs_s, hsg.F16, hsg.BATCHED, k, args.warmup, None, peak)
        strm["lat"].destroy()
        small = {"workload": SMALL_WORKLOAD, "steps": k,
                 "resident": {"value": round(res["value"], 3), "ms_per_step": round(res["ms_per_step"], 3),
                              "roofline": res["roofline"], "gpu_launches": res["launches"]},
                 "resident_per_size": {"value": round(one["value"], 3), "ms_per_step": round(one["ms_per_step"], 3),
                                       "roofline": one["roofline"], "gpu_launches": one["launches"]},
                 "streaming_f16": {"value": round(strm["value"], 3),
                                   "ms_per_step": round(strm["ms_per_step"], 3)},
                 "resident_over_streaming": round(res["value"] / strm["value"], 3),
                 "sequential_or_sweep": time_sequential_or(hsg, ws, inputs_s, torch)}
        del inputs_s
        # mid-size lattices: parts of replica sets resident, PT between launches
        wm = WORKLOADS[MID_WORKLOAD]
        inputs_m = make_inputs(wm, rank)
        res = run_form(hsg, torch, dist, MID_WORKLOAD, inputs_m, hsg.F16, hsg.BATCHED, k, args.warmup, None, peak,
                       persistent=True)
        strm = run_form(hsg, torch, dist, MID_WORKLOAD, inputs_m, hsg.F16, hsg.BATCHED, k, args.warmup, None, peak)
        strm["lat"].destroy()
        mid = {"workload": MID_WORKLOAD, "steps": k,
               "resident": {"value": round(res["value"], 3), "ms_per_step": round(res["ms_per_step"], 3),
                            "roofline": res["roofline"], "gpu_launches": res["launches"]},
               "streaming_f16": {"value": round(strm["value"], 3), "ms_per_step": round(strm["ms_per_step"], 3),
                                 "roofline": strm["roofline"]},
               "resident_over_streaming": round(res["value"] / strm["value"], 3)}
        del inputs_m
    e2e = None if args.no_e2e else e2e_run(hsg, torch, dist, w, inputs, args.steps)
    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, inputs)
        err = oracle_error(hsg, w, inputs)
    if rank == 0:
        line = {"metric": METRIC, "value": round(batched["value"], 3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(batched["ms_per_step"], 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.workload, w, world),
                "roofline": batched["roofline"], "gpu_launches": batched["launches"],
                "clocks": batched["clocks"], "e2e": e2e, "cpu_baseline": cpu}
        if err is not None:
            line["oracle_error"] = err
        if plain is not None:
            line["plain_fp32"] = {"value": round(plain["value"], 3),
                                  "ms_per_step": round(plain["ms_per_step"], 3),
                                  "roofline": plain["roofline"], "gpu_launches": plain["launches"],
                                  "note": "one lattice per element, but the lattices of a sample share "
                                          "their couplings through L2 (traffic well below the algorithmic "
                                          "96 B per update), so frac is not an HBM-roofline fraction; "
                                          "plain_fp32_single is the single-lattice form"}
            line["batched_over_plain"] = round(batched["value"] / plain["value"], 3)
        if single is not None:
            line["plain_fp32_single"] = {"value": round(single["value"], 3),
                                         "ms_per_step": round(single["ms_per_step"], 3),
                                         "workload": SINGLE_WORKLOAD,
                                         "roofline": single["roofline"], "gpu_launches": single["launches"]}
            line["batched_over_plain_single"] = round(batched["value"] / single["value"], 3)
        line.update(bimodal)
        if streaming is not None:
            line["streaming_f16"] = {"value": round(streaming["value"], 3),
                                     "ms_per_step": round(streaming["ms_per_step"], 3),
                                     "roofline": streaming["roofline"],
                                     "gpu_launches": streaming["launches"]}
            line["resident_over_streaming"] = round(batched["value"] / streaming["value"], 3)
        if sequential is not None:
            line["sequential_or_sweep"] = sequential
        if joint is not None:
            line["resident_per_size"] = {"value": round(joint["value"], 3),
                                         "ms_per_step": round(joint["ms_per_step"], 3),
                                         "roofline": joint["roofline"], "gpu_launches": joint["launches"]}
        if small is not None:
            line["small_lattices"] = small
        if mid is not None:
            line["mid_lattices"] = mid
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
