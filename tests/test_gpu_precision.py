"""Precision form: the FP32 path (FP32 FFTs and draws, FP64 shell sums and
inverse-gamma parameters) against the FP64 path, which matches the oracle to
1e-12, on the 256^3 workload with the same seeds: chains 0 and 15 over 200
sweeps.  Reported: relative L2 error of each chain's running mean of s and of
its mean P(k) over sweeps 21..200, and the worst per-sweep errors; bounded here
by the per-sweep FP32 tolerance 2e-5.
"""
import json

import numpy as np
import pytest

import mockgen

from gpu_helpers import gpu_sampler, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def test_fp32_against_fp64_over_200_sweeps(capsys):
    need_gpu()
    w = mockgen.workload(3)
    m = w.mocks[0]
    S = 200
    report = {}
    with gpu_sampler(m, m.n_bins, 3, 32, n_chains=16) as g32, gpu_sampler(m, m.n_bins, 3, 64, n_chains=1,
                                                                                  chain_id0=0) as g0, \
            gpu_sampler(m, m.n_bins, 3, 64, n_chains=1, chain_id0=15) as g15:
        ms32 = {0: 0.0, 15: 0.0}
        ms64 = {0: 0.0, 15: 0.0}
        mp32 = {0: 0.0, 15: 0.0}
        mp64 = {0: 0.0, 15: 0.0}
        worst_s, worst_p = 0.0, 0.0
        for sw in range(1, S + 1):
            g32.sweep(1)
            g0.sweep(1)
            g15.sweep(1)
            if sw % 10 and sw != 1:
                continue
            for c, g64 in ((0, g0), (15, g15)):
                s32, s64 = g32.read_s(c).astype(np.float64), g64.read_s(0)
                p32, p64 = g32.read_pk(c), g64.read_pk(0)
                worst_s = max(worst_s, rel_l2(s32, s64))
                worst_p = max(worst_p, rel_l2(p32, p64))
                if sw > 20:
                    ms32[c] = ms32[c] + s32
                    ms64[c] = ms64[c] + s64
                    mp32[c] = mp32[c] + p32
                    mp64[c] = mp64[c] + p64
        for c in (0, 15):
            report[f"chain{c}_mean_s_rel_l2"] = rel_l2(ms32[c], ms64[c])
            report[f"chain{c}_mean_P_rel_l2"] = rel_l2(mp32[c], mp64[c])
        report["worst_sample_s_rel_l2"] = worst_s
        report["worst_sample_P_rel_l2"] = worst_p
    with capsys.disabled():
        print("\nprecision report " + json.dumps(report))
    assert worst_s <= 2e-5 and worst_p <= 2e-5, report
