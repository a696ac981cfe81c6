"""Batching form: chains of uneven grid sizes advanced by one persistent kernel
launch per sweep (captured in a CUDA graph), the autotuner, and the bounded
waits of the persistent kernel.

* A mixed batch (16^3, 24^3, 48^3; FP64 and FP32) in one persistent launch
  matches independent oracle chains draw for draw.
* The full batching workload (16 x 64^3 + 16 x 96^3 + 16 x 128^3, each with
  its own data, FP32) in one persistent launch per sweep: sampled chains of
  each size against the oracle.
* The tuner leaves the chains untouched and picks a valid schedule.
* A wait budget of one cycle makes the x tiles give up on their y/z planes:
  the device reports MG_ETIMEOUT (sticky) and nothing faults or hangs.
* 70 chains on one data set (more than one launch holds) match the oracle on
  both sides of the split.
* mg_read_pk_all returns every chain's P(k) in one transfer, equal to the
  per-chain reads, with zero padding for the chains with fewer shells.
"""
import numpy as np
import pytest

import mockgen

from gpu_helpers import TOL, check_elementwise, need_gpu, oracle_chains, rel_l2

pytestmark = pytest.mark.gpu


def batch(mocks, seeds, precision, **kw):
    from paper_1402_1763_gb300 import Sampler
    return Sampler.batch([m.n for m in mocks], [m.L for m in mocks], [m.N for m in mocks],
                         [m.R for m in mocks], [m.d for m in mocks], [m.n_bins for m in mocks], seeds,
                         precision=precision, **kw)


def mixed():
    mocks = [mockgen.make_mock(n, seed=500 + n, n_bins=b, sigma_n=sg)
             for n, b, sg in ((16, 4, 0.1), (24, 6, 0.5), (48, 12, 0.1))]
    return mocks, [21, 22, 23]


@pytest.mark.parametrize("precision", [64, 32])
def test_persistent_mixed_batch_matches_oracle(precision):
    need_gpu()
    mocks, seeds = mixed()
    with batch(mocks, seeds, precision, n_chains=2, persistent=True) as g:
        assert g.schedule()["persistent"]
        g.sweep(3)
        for gi, m in enumerate(mocks):
            orc = oracle_chains(m, m.n_bins, seeds[gi], [0, 1])
            orc.sweep(3)
            for c in range(2):
                sg, pg = g.read_s(2 * gi + c), g.read_pk(2 * gi + c)
                es = rel_l2(sg, orc.s[c])
                ep = rel_l2(pg, orc.P[c])
                assert es <= TOL[precision] and ep <= TOL[precision], (gi, c, es, ep)
                check_elementwise(precision, sg, orc.s[c], pg, orc.P[c], f"persistent batch n={m.n} chain {c}")


def test_batching_workload_one_persistent_launch_per_sweep():
    need_gpu()
    w = mockgen.workload(4)
    with batch(w.mocks, w.seeds, 32, persistent=True) as g:
        assert g.schedule() == {"sizes": [64, 96, 128], "yz_cluster": [1, 1, 1], "persistent": True}
        g.sweep(2)
        for c in (0, 15, 16, 31, 32, 47):
            m = w.mocks[c]
            orc = oracle_chains(m, m.n_bins, w.seeds[c], [0])
            orc.sweep(2)
            sg, pg = g.read_s(c), g.read_pk(c)
            es = rel_l2(sg, orc.s[0])
            ep = rel_l2(pg, orc.P[0])
            assert es <= TOL[32] and ep <= TOL[32], (c, es, ep)
            check_elementwise(32, sg, orc.s[0], pg, orc.P[0], f"batching workload chain {c}")
        assert g.sweep_count == 2


def test_tuner_keeps_chains_and_picks_a_schedule():
    need_gpu()
    mocks, seeds = mixed()
    with batch(mocks, seeds, 32, n_chains=2) as g:
        g.sweep(2)
        before = [g.read_s(c) for c in range(6)]
        pk = [g.read_pk(c) for c in range(6)]
        g.tune(3)
        sch = g.schedule()
        assert sch["sizes"] == [16, 24, 48] and all(c == 1 for c in sch["yz_cluster"])
        for c in range(6):
            assert np.array_equal(g.read_s(c), before[c]) and np.array_equal(g.read_pk(c), pk[c])
        assert g.sweep_count == 2
        g.sweep(1)
        for gi, m in enumerate(mocks):
            orc = oracle_chains(m, m.n_bins, seeds[gi], [0, 1])
            orc.sweep(3)
            assert rel_l2(g.read_s(2 * gi), orc.s[0]) <= TOL[32]


def test_autotune_option_on_the_256_grid():
    need_gpu()
    from paper_1402_1763_gb300 import Sampler
    m = mockgen.make_mock(256, seed=3, n_bins=64)
    with Sampler.single(256, m.L, m.N, m.R, m.d, 64, 3, precision=32, n_chains=2, autotune=True) as g:
        sch = g.schedule()
        assert sch["sizes"] == [256] and sch["yz_cluster"][0] in (2, 4, 8) and not sch["persistent"]
        assert g.sweep_count == 0


def test_wait_budget_exhaustion_is_reported():
    need_gpu()
    from paper_1402_1763_gb300 import MG_ETIMEOUT, MgError
    mocks, seeds = mixed()
    g = batch(mocks, seeds, 64, n_chains=2, persistent=True, timeout_cycles=1)
    try:
        g.sweep(1)
        with pytest.raises(MgError) as e:
            g.sync()
        assert e.value.status == MG_ETIMEOUT
        with pytest.raises(MgError) as e2:
            g.sweep(1)
        assert e2.value.status == MG_ETIMEOUT
    finally:
        g.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_more_chains_than_one_launch_holds(precision):
    """70 chains of one data set: the passes are issued in launches of at most
    64 chains each; chains on both sides of the split match the oracle."""
    need_gpu()
    from gpu_helpers import gpu_sampler
    m = mockgen.make_mock(16, seed=70, n_bins=4)
    follow = [0, 63, 64, 69]
    orc = oracle_chains(m, 4, 31, follow)
    orc.sweep(2)
    with gpu_sampler(m, 4, 31, precision, n_chains=70) as g:
        g.sweep(2)
        for k, c in enumerate(follow):
            assert rel_l2(g.read_s(c), orc.s[k]) <= TOL[precision]
            assert rel_l2(g.read_pk(c), orc.P[k]) <= TOL[precision]


def test_read_pk_all_matches_per_chain_reads():
    need_gpu()
    mocks, seeds = mixed()
    with batch(mocks, seeds, 32, n_chains=2) as g:
        g.sweep(3)
        allp = g.read_pk_all()
        B1 = max(m.n_bins for m in mocks) + 1
        assert allp.shape == (6, B1)
        for c in range(6):
            p = g.read_pk(c)
            np.testing.assert_array_equal(allp[c, :p.size], p)
            assert np.all(allp[c, p.size:] == 0.0)
        g.sweep(1)
        again = np.full((6, B1), np.nan)
        g.read_pk_all(again)
        assert np.array_equal(again[0, :5], g.read_pk(0)) and not np.array_equal(again, allp)
