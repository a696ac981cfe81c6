"""The recorded P(k) trace and its summaries on the device (correlation length
of the paper's efficiency analysis, posterior quantiles), through the C ABI.

* With record_every = 1 the trace holds P after every sweep: checked against
  mg_read_pk read after each single sweep (bit-exact), for plain and mixing
  sweeps, FP64 and FP32.
* mg_pk_acf and mg_pk_quantiles against the oracle's definitions applied to
  the trace read back (relative 1e-12; correlation lengths equal).
* With record_every = 3 only every third sweep is recorded.
* mg_pk_rhat over the chains against the oracle's Gelman-Rubin definition.
* Over-dispersed starts (start_dispersion > 0): the starting P of every chain
  and the chains after a few sweeps match the oracle.
* Invalid lags and quantiles, and summaries without records, are MG_EINVAL.
"""
import numpy as np
import pytest

import mockgen

from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def sampler(precision, record_every, mixing=0, n=16):
    from paper_1402_1763_gb300 import Sampler
    m = mockgen.make_mock(n, seed=6, n_bins=6, sigma_n=0.5)
    return Sampler.single(m.n, m.L, m.N, m.R, m.d, 6, 9, precision=precision, n_chains=2,
                          record_every=record_every, mixing=mixing)


@pytest.mark.parametrize("precision,mixing", [(64, 0), (32, 0), (64, 2)])
def test_trace_acf_and_quantiles(precision, mixing):
    need_gpu()
    from oracle import summary
    with sampler(precision, 1, mixing) as g:
        seen = [[], []]
        for _ in range(300):
            g.sweep(1)
            for c in range(2):
                seen[c].append(g.read_pk(c))
        for c in range(2):
            tr = g.pk_trace(c)
            assert tr.shape == (300, 7)
            np.testing.assert_array_equal(tr, np.array(seen[c]))
            acf, nc = g.pk_acf(40, c)
            acf_o, nc_o = summary.acf(tr, 40)
            np.testing.assert_allclose(acf, acf_o, rtol=1e-12, atol=1e-12)
            np.testing.assert_array_equal(nc, nc_o)
            q = [0.025, 0.16, 0.5, 0.84, 0.975, 0.0, 1.0]
            np.testing.assert_allclose(g.pk_quantiles(q, c), summary.quantiles(tr, q), rtol=1e-12, atol=0)


@pytest.mark.parametrize("mixing", [0, 1])
def test_rhat_across_chains(mixing):
    need_gpu()
    from oracle import summary
    from paper_1402_1763_gb300 import Sampler
    m = mockgen.make_mock(16, seed=6, n_bins=6, sigma_n=0.5)
    with Sampler.single(m.n, m.L, m.N, m.R, m.d, 6, 9, precision=64, n_chains=4, record_every=1,
                        mixing=mixing) as g:
        g.sweep(120)
        traces = [g.pk_trace(c) for c in range(4)]
        for burn in (0, 40):
            np.testing.assert_allclose(g.pk_rhat(0, 4, burn), summary.rhat(traces, burn), rtol=1e-12)
        np.testing.assert_allclose(g.pk_rhat(1, 2, 10), summary.rhat(traces[1:3], 10), rtol=1e-12)


def test_over_dispersed_starts():
    need_gpu()
    from oracle import sampler as sp
    from paper_1402_1763_gb300 import Sampler
    from gpu_helpers import rel_l2
    m = mockgen.make_mock(16, seed=6, n_bins=6, sigma_n=0.5)
    prob = sp.make_problem(m.shape, m.L, m.N, m.R, m.d, 6)
    orc = sp.Chains(prob, seed=9, chain_ids=[0, 1, 2], start_dispersion=1.5)
    with Sampler.single(m.n, m.L, m.N, m.R, m.d, 6, 9, precision=64, n_chains=3, start_dispersion=1.5) as g:
        for c in range(3):
            np.testing.assert_allclose(g.read_pk(c), orc.P[c], rtol=1e-14)
        orc.sweep(4)
        g.sweep(4)
        for c in range(3):
            assert rel_l2(g.read_pk(c), orc.P[c]) <= 1e-12 and rel_l2(g.read_s(c), orc.s[c]) <= 1e-12


def test_record_every_three():
    need_gpu()
    with sampler(32, 3) as g:
        seen = []
        for k in range(1, 31):
            g.sweep(1)
            if k % 3 == 0:
                seen.append(g.read_pk(1))
        np.testing.assert_array_equal(g.pk_trace(1), np.array(seen))


def test_summary_argument_checks():
    need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MgError
    with sampler(32, 0) as g:
        g.sweep(2)
        with pytest.raises(MgError) as e:
            g.pk_acf(1)
        assert e.value.status == MG_EINVAL
        with pytest.raises(MgError) as e:
            g.pk_quantiles([0.5])
        assert e.value.status == MG_EINVAL
    with sampler(32, 1) as g:
        g.sweep(5)
        with pytest.raises(MgError) as e:
            g.pk_acf(5)
        assert e.value.status == MG_EINVAL
        with pytest.raises(MgError) as e:
            g.pk_quantiles([1.5])
        assert e.value.status == MG_EINVAL
