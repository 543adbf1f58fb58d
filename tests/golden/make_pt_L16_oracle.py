"""Writes tests/golden/pt_L16_oracle.json (FP32-stored couplings) or, with
--f16, tests/golden/pt_L16_f16_oracle.json (the same Gaussian draws rounded
once to FP16, the values the FP16-coupling GPU form stores): block averages
of independent FP64 oracle chains on the parallel-tempering workload (L=16,
the couplings of disorder sample 0, 16 temperatures evenly spaced in
[0.15, 0.75] x 2 replicas, 20000 steps of one heat-bath + 8 overrelaxation
sweeps + one PT sweep, observables every 10 steps).  Chain c starts from the
random spins of generator sample c and uses the random streams of sample
index c, as chain c of the GPU test does.  Calls only the oracle and the
seeded input generator.

    python tests/golden/make_pt_L16_oracle.py [--f16]     # 8 chains in parallel
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

L, N_T, N_REP, SEED, N_CHAINS = 16, 16, 2, 1, 8
STEPS, BLOCK, MEASURE_EVERY, N_OR = 20000, 1000, 10, 8


def chain(args):
    c, precision = args
    import numpy as np

    import hsg_inputs as gi
    import oracle
    beta = gi.linear_betas(0.15, 0.75, N_T)
    J6 = gi.couplings(L, SEED, 0, precision=precision)
    spins = gi.random_spins_batch(L, SEED, c, N_T * N_REP)
    smp = oracle.Sample(L, J6, spins, beta, N_REP, SEED, sample_index=c)
    blocks = []
    t0 = time.time()
    for b in range(STEPS // BLOCK):
        smp.obs[:] = 0
        smp.counts[:] = 0
        smp.run(BLOCK, N_OR, MEASURE_EVERY, n_threads=max(1, os.cpu_count() // N_CHAINS))
        obs = smp.obs.copy()
        n = smp.counts[:, None].astype(float)
        mean = np.empty_like(obs)
        mean[:, 0:2] = obs[:, 0:2] / (n * N_REP)          # per lattice
        mean[:, 2:8] = obs[:, 2:8] / (n * (N_REP // 2))   # per pair
        mean[:, 8] = obs[:, 8] / (n[:, 0] * N_REP)
        blocks.append(mean.tolist())
        print(f"chain {c} block {b} done at {time.time() - t0:.0f} s", flush=True)
    return blocks, smp.accepted.tolist()


def main():
    precision = "f16" if "--f16" in sys.argv else "f32"
    ctx = mp.get_context("spawn")
    with ctx.Pool(N_CHAINS) as pool:
        res = pool.map(chain, [(c, precision) for c in range(N_CHAINS)])
    import oracle
    out = {"L": L, "n_temps": N_T, "n_replicas": N_REP, "seed": SEED, "steps": STEPS,
           "block_steps": BLOCK, "measure_every": MEASURE_EVERY, "n_or": N_OR,
           "T_range": [0.15, 0.75], "couplings": precision, "observables": list(oracle.OBS_NAMES),
           "chains": [r[0] for r in res], "pt_accepted": [r[1] for r in res]}
    name = "pt_L16_f16_oracle.json" if precision == "f16" else "pt_L16_oracle.json"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main()
