"""Precision form: the FP32 path (FP32 FFTs and draws, FP64 shell sums and
inverse-gamma parameters) against the FP64 path, which matches the oracle to
1e-12, on the 256^3 workload with the same seeds: chains 0 and 15 over 200
sweeps (bounded by the per-sweep FP32 tolerance 2e-5) and over the
configuration's 2000 sweeps (bounded against the Monte-Carlo standard error of
the posterior means).  Reported: relative L2 error of each chain's mean of s and
of its mean P(k), and the worst per-sweep errors.
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


def test_fp32_against_fp64_over_2000_sweeps(capsys):
    """The 256^3 configuration's full length: 16 FP32 chains and FP64 chains 0
    and 15 on the same seeds, 2000 sweeps, every 10th state recorded on the
    device (mean and variance maps of s, P(k) trace).  Past the first few
    hundred sweeps the two trajectories drift apart like a random walk (the
    chain does not contract the per-sweep rounding in its slow directions), so
    the bar is on what the samples are for: the difference between the FP32 and
    FP64 posterior means (of s and of P(k)) must stay below 1 % of the
    Monte-Carlo standard error of those means, sd / sqrt(records) per voxel or
    shell (the number of records bounds the effective sample size from above,
    so this is conservative).  Also reported: relative L2 of the means and the
    worst single-sweep error at every 100th sweep."""
    need_gpu()
    w = mockgen.workload(3)
    m = w.mocks[0]
    S, every = 2000, 10
    report = {"sweeps": S, "record_every": every}
    with gpu_sampler(m, m.n_bins, 3, 32, n_chains=16, record_every=every) as g32, \
            gpu_sampler(m, m.n_bins, 3, 64, n_chains=1, chain_id0=0, record_every=every) as g0, \
            gpu_sampler(m, m.n_bins, 3, 64, n_chains=1, chain_id0=15, record_every=every) as g15:
        worst_s, worst_p = 0.0, 0.0
        for blk in range(S // 100):
            g32.sweep(100)
            g0.sweep(100)
            g15.sweep(100)
            for c, g64 in ((0, g0), (15, g15)):
                worst_s = max(worst_s, rel_l2(g32.read_s(c).astype(np.float64), g64.read_s(0)))
                worst_p = max(worst_p, rel_l2(g32.read_pk(c), g64.read_pk(0)))
        for c, g64 in ((0, g0), (15, g15)):
            st32 = g32.read_stats(c, maps=True)
            st64 = g64.read_stats(0, maps=True)
            nrec = st64["records"]
            assert st32["records"] == nrec == S // every
            dmean = np.linalg.norm(st32["mean"] - st64["mean"])
            se_s = np.sqrt(st64["var"].sum() / nrec)
            tr32, tr64 = g32.pk_trace(c), g64.pk_trace(0)
            nb = st64["n_b"] > 0
            dP = np.linalg.norm(tr32.mean(0)[nb] - tr64.mean(0)[nb])
            se_P = np.sqrt((tr64[:, nb].var(0, ddof=1) / nrec).sum())
            report[f"chain{c}_mean_s_rel_l2"] = dmean / np.linalg.norm(st64["mean"])
            report[f"chain{c}_mean_P_rel_l2"] = dP / np.linalg.norm(tr64.mean(0)[nb])
            report[f"chain{c}_mean_s_diff_over_mc_se"] = dmean / se_s
            report[f"chain{c}_mean_P_diff_over_mc_se"] = dP / se_P
        report["worst_sample_s_rel_l2"] = worst_s
        report["worst_sample_P_rel_l2"] = worst_p
    with capsys.disabled():
        print("\nprecision report 2000 sweeps " + json.dumps(report))
    for c in (0, 15):
        assert report[f"chain{c}_mean_s_diff_over_mc_se"] <= 0.01, report
        assert report[f"chain{c}_mean_P_diff_over_mc_se"] <= 0.01, report
        assert report[f"chain{c}_mean_s_rel_l2"] <= 2e-4 and report[f"chain{c}_mean_P_rel_l2"] <= 2e-4, report
