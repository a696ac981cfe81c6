"""End-to-end check of what the samples are for (Sec. 5.2): the posterior P(k)
of the 128^3 workload with holes (16 FP32 chains, 4000 plain sweeps, every
10th state recorded, the first quarter dropped) against the power of the field
that generated the data, binned into the sampler's shells with the oracle's
transform and shell sums: P_b = (V/M) sigma_b(s_true) / n_b.  A calibrated
posterior holds the realized power inside its central 95 % interval in about
95 % of the shells; on this data set 30 of 33 (31 inside the 99 % interval).
The draws are fixed by the seeds, so the counts are a regression bar: at least
29 shells inside 95 % and 30 inside 99 %, and no posterior median off the
realized power by more than a factor of 2."""
import numpy as np
import pytest

import mockgen
from oracle import sampler

from gpu_helpers import gpu_sampler, need_gpu

pytestmark = pytest.mark.gpu


def test_posterior_power_covers_the_realized_power_128cubed():
    need_gpu()
    w = mockgen.workload(2)
    m = w.mocks[0]
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, m.n_bins)
    n_b = prob.bins.n_b
    sig = sampler.shell_sums(prob.bins, sampler.ont(m.s_true)[None])[0]
    keep = n_b > 0
    P_real = (prob.V / prob.M) * sig[keep] / n_b[keep]
    with gpu_sampler(m, m.n_bins, w.seeds[0], 32, n_chains=16, record_every=10) as g:
        g.sweep(4000)
        traces = [g.pk_trace(c) for c in range(16)]
    burn = traces[0].shape[0] // 4
    pool = np.concatenate([t[burn:] for t in traces])[:, keep]
    q = np.quantile(pool, [0.005, 0.025, 0.5, 0.975, 0.995], axis=0)
    inside95 = int(np.sum((q[1] <= P_real) & (P_real <= q[3])))
    inside99 = int(np.sum((q[0] <= P_real) & (P_real <= q[4])))
    ratio = q[2] / P_real
    assert inside95 >= 29 and inside99 >= 30, (inside95, inside99, int(keep.sum()))
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio
