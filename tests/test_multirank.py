"""The multi-rank path on the CPU (two gloo ranks): independent replicas --
each rank runs its own samples with its own random-number key, the timing is
the maximum over ranks, and the reference arm prints on rank 0 only."""
import argparse
import contextlib
import io
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_env() == (world, rank, rank)
    d = bench.Dist(world, rank, rank, "gloo")
    res = {"max": d.max(float(rank + 1))}
    d.barrier()
    w = dict(Ls=(4, 6), S=2, n_rep=2, NT=2, Tmin=0.3, Tmax=0.9, n_or=1, measure_every=1)
    samples, J, spins, beta = bench.make_inputs(w, rank)
    res["samples"] = samples
    res["J0"] = float(J[0].sum())
    res["key"] = bench.philox_key(rank)
    args = argparse.Namespace(steps=1, warmup=0, workload="tiny")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        res["rc"] = bench.reference_arm(args, w, world, rank, rank)
    res["printed"] = buf.getvalue()
    d.barrier()
    d.close()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_run_independent_replicas(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["max"] == r[1]["max"] == 2.0                 # max over ranks
    assert r[0]["samples"] == [0, 1] and r[1]["samples"] == [2, 3]
    assert r[0]["J0"] != r[1]["J0"]                         # different disorder
    assert r[0]["key"] != r[1]["key"]                       # independent streams
    assert r[0]["rc"] == r[1]["rc"] == 0
    line = json.loads(r[0]["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert r[1]["printed"] == ""                            # rank 0 alone prints
