"""Writes tests/golden/workload2_128holes_fp64_1000sweeps.json from the oracle
alone (oracle.sampler and the seeded inputs of mockgen; nothing of the CUDA
library).

The 128^3 workload with 40 holes (32 shells, seed 2, one chain, FP64) asks for
1000 sweeps matched draw for draw.  The oracle needs about half a second per
sweep at this size, too slow to run inside the GPU test, so this script runs
it once and stores, after sweeps 300 and 1000, the chain's P(k) and its field s
at 2048 voxels drawn (seeded) without replacement.  The GPU test sweeps the
same chain 1000 times and compares at both checkpoints.

    python tests/golden/make_workload2_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import mockgen  # noqa: E402
from oracle import sampler  # noqa: E402

OUT = os.path.join(HERE, "workload2_128holes_fp64_1000sweeps.json")
CHECKPOINTS = (300, 1000)
N_SAMPLE = 2048
SAMPLE_SEED = 12345


def main():
    w = mockgen.workload(2)
    m = w.mocks[0]
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, m.n_bins)
    seed = w.seeds[0]
    ch = sampler.Chains(prob, seed=seed, chain_ids=[0])
    M = int(np.prod(m.shape))
    vox = np.sort(np.random.default_rng(SAMPLE_SEED).choice(M, N_SAMPLE, replace=False))
    out = {"workload": w.name, "seed": seed, "chain": 0, "n_bins": m.n_bins, "grid": m.n,
           "made_by": "tests/golden/make_workload2_golden.py (oracle.sampler.Chains, FP64 numpy)",
           "sample_voxels": [int(v) for v in vox], "checkpoints": {}}
    done = 0
    t0 = time.time()
    for cp in CHECKPOINTS:
        ch.sweep(cp - done)
        done = cp
        s = ch.s[0].reshape(-1)
        out["checkpoints"][str(cp)] = {"P": [float(x) for x in ch.P[0]],
                                       "s_sample": [float(x) for x in s[vox]],
                                       "s_norm": float(np.linalg.norm(s))}
        print(f"sweep {cp}: {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
