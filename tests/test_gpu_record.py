"""Recorded samples and the posterior mean and variance maps built from them.

With record_every = r > 0, every r-th sweep's state is a sample: the library
keeps FP64 sums of s and s^2 per voxel (a sample is added inside the next
sweep's pass YZ, or by a separate pass when the sums are read first, the state
is replaced, or the schedule is the persistent one) and reports
mean = S1/n, var = (S2 - S1 mean)/(n - 1).  Checked against the oracle's
samples (numpy mean and var with ddof = 1 of the same draws):

* record_every = 3, reads in between that find a sample still pending (at 9
  sweeps) and none (at 10): nothing is added twice or lost (FP64, 1e-12).
* The FP32 path (the sums are FP64 of the FP32 samples): within the FP32
  field tolerance.
* The persistent schedule (the samples added right after each sweep).
* Alternating plain and mixing sweeps (both sweep kinds carry the record).
* set_s with a sample pending adds the old state first.
* The sums formed inside the sweep and by the separate pass agree bit for bit
  (FP64 sums, and the double-float pairs of FP32 samples), also where pass YZ
  splits its planes over thread-block clusters (128^3, 192^3, 256^3).
"""
import numpy as np
import pytest

import mockgen
from oracle import mixing as mx

from gpu_helpers import TOL, gpu_sampler, need_gpu, oracle_chains

pytestmark = pytest.mark.gpu


def samples(orc, sweeps, every, chain=0):
    xs = []
    for k in range(1, sweeps + 1):
        orc.sweep(1)
        if k % every == 0:
            xs.append(orc.s[chain].copy())
    return np.array(xs)


def check(st, xs, atol):
    n = len(xs)
    assert st["records"] == n
    np.testing.assert_allclose(st["mean"].reshape(xs.shape[1:]), xs.mean(axis=0), rtol=0, atol=atol)
    np.testing.assert_allclose(st["var"].reshape(xs.shape[1:]), xs.var(axis=0, ddof=1), rtol=0, atol=10 * atol)


def test_reads_between_sweeps_add_every_sample_once():
    need_gpu()
    m = mockgen.make_mock(16, seed=71, n_bins=4, sigma_n=0.3)
    orc = oracle_chains(m, 4, 5, [0])
    with gpu_sampler(m, 4, 5, 64, record_every=3) as g:
        g.sweep(9)
        st9 = g.read_stats(0, maps=True)  # sample 9 still pending: added by the read
        g.sweep(1)
        st10 = g.read_stats(0, maps=True)  # nothing pending
        g.sweep(11)
        st21 = g.read_stats(0, maps=True)  # sample 21 pending
    xs = samples(orc, 21, 3)
    check(st9, xs[:3], 1e-12)
    check(st10, xs[:3], 1e-12)
    check(st21, xs, 1e-12)


def test_fp32_sums():
    need_gpu()
    m = mockgen.make_mock(24, seed=72, n_bins=6, sigma_n=0.3)
    orc = oracle_chains(m, 6, 6, [0])
    with gpu_sampler(m, 6, 6, 32, record_every=1) as g:
        g.sweep(12)
        st = g.read_stats(0, maps=True)
    xs = samples(orc, 12, 1)
    scale = np.abs(xs).max()
    check(st, xs, 4 * TOL[32] * scale)


def test_persistent_schedule_records_after_each_sweep():
    need_gpu()
    from paper_1402_1763_gb300 import Sampler
    m = mockgen.make_mock(16, seed=73, n_bins=4, sigma_n=0.3)
    orc = oracle_chains(m, 4, 7, [0, 1])
    with Sampler.batch([m.n], [m.L], [m.N], [m.R], [m.d], [4], [7], precision=64, n_chains=2,
                       persistent=True, record_every=2) as g:
        assert g.schedule()["persistent"]
        g.sweep(8)
        st0, st1 = g.read_stats(0, maps=True), g.read_stats(1, maps=True)
    xs = []
    for k in range(1, 9):
        orc.sweep(1)
        if k % 2 == 0:
            xs.append(orc.s.copy())
    xs = np.array(xs)
    check(st0, xs[:, 0], 1e-12)
    check(st1, xs[:, 1], 1e-12)


def test_alternating_mixing_sweeps_record():
    need_gpu()
    from oracle import sampler
    m = mockgen.make_mock(16, seed=74, n_bins=4, sigma_n=0.3)
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, 4)
    orc = mx.AlternatingChains(prob, seed=8, chain_ids=[0])
    with gpu_sampler(m, 4, 8, 64, record_every=1, mixing=2) as g:
        g.sweep(10)
        st = g.read_stats(0, maps=True)
    check(st, samples(orc, 10, 1), 1e-12)


def test_set_s_adds_the_pending_sample_first():
    need_gpu()
    m = mockgen.make_mock(16, seed=75, n_bins=4, sigma_n=0.3)
    orc = oracle_chains(m, 4, 9, [0])
    xs = samples(orc, 4, 2)
    with gpu_sampler(m, 4, 9, 64, record_every=2) as g:
        g.sweep(4)  # samples 2 and 4; 4 pending
        g.set_s(0, np.zeros(m.shape))
        st = g.read_stats(0, maps=True)
    check(st, xs, 1e-12)


@pytest.mark.parametrize("n,precision,cluster", [(24, 64, 0), (24, 32, 0), (128, 32, 2), (192, 64, 2),
                                               (256, 32, 4), (256, 32, 2)])
def test_fused_and_separate_sums_agree_bit_for_bit(n, precision, cluster):
    """Also in the cluster forms of pass YZ, whose record mode finds each
    voxel's sums through the CTA's rank in the cluster."""
    need_gpu()
    m = mockgen.make_mock(n, seed=76, n_bins=6, sigma_n=0.3)
    with gpu_sampler(m, 6, 10, precision, record_every=1, yz_cluster=cluster) as a, \
            gpu_sampler(m, 6, 10, precision, record_every=1, yz_cluster=cluster) as b:
        for _ in range(6):
            a.sweep(1)
            a.read_stats(0, maps=True)  # every sample added by the separate pass
        b.sweep(6)  # samples 1..5 added inside the next sweep, 6 by the read
        sa, sb = a.read_stats(0, maps=True), b.read_stats(0, maps=True)
    assert sa["records"] == sb["records"] == 6
    np.testing.assert_array_equal(sa["mean"], sb["mean"])
    np.testing.assert_array_equal(sa["var"], sb["var"])
