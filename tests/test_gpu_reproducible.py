"""Bit-for-bit reproducibility: two contexts made from the same inputs and seeds
give identical fields and P(k) after the same sweeps.  Every sum in the library
runs in a fixed order (segmented warp scans, per-tile and per-shell combines in
index order), the tau bound is an integer minimum, and every draw is a function
of its Philox counter, so nothing may depend on scheduling: checked for the
plain sweep at 256^3 (clusters of 4, the benchmark's launch form) and 32^3, the
persistent batch schedule, and mixing sweeps, in FP64 and FP32."""
import numpy as np
import pytest

import mockgen

from gpu_helpers import gpu_sampler, need_gpu

pytestmark = pytest.mark.gpu


def states(g, chains):
    return [(g.read_s(c).copy(), g.read_pk(c).copy()) for c in chains]


def same(a, b):
    for (s1, p1), (s2, p2) in zip(a, b):
        assert np.array_equal(s1, s2) and np.array_equal(p1, p2)


@pytest.mark.parametrize("n,precision,n_chains,sweeps", [(32, 64, 2, 6), (32, 32, 2, 6), (256, 32, 16, 3)])
def test_plain_sweeps_are_bitwise_reproducible(n, precision, n_chains, sweeps):
    need_gpu()
    m = mockgen.make_mock(n, seed=61 + n, n_bins=8 if n == 32 else 64)
    runs = []
    for _ in range(2):
        with gpu_sampler(m, m.n_bins, 17, precision, n_chains=n_chains) as g:
            g.sweep(sweeps)
            runs.append(states(g, [0, n_chains - 1]))
    same(*runs)


@pytest.mark.parametrize("precision", [64, 32])
def test_persistent_batch_and_mixing_are_bitwise_reproducible(precision):
    need_gpu()
    from paper_1402_1763_gb300 import Sampler
    mocks = [mockgen.make_mock(n, seed=700 + n, n_bins=b) for n, b in ((16, 4), (24, 6))]
    runs = []
    for _ in range(2):
        with Sampler.batch([m.n for m in mocks], [m.L for m in mocks], [m.N for m in mocks],
                           [m.R for m in mocks], [m.d for m in mocks], [m.n_bins for m in mocks], [31, 32],
                           precision=precision, n_chains=2, persistent=True) as g:
            g.sweep(4)
            runs.append(states(g, [0, 3]))
    same(*runs)
    m = mockgen.make_mock(32, seed=77, n_bins=8)
    runs = []
    for _ in range(2):
        with gpu_sampler(m, 8, 19, precision, n_chains=2, mixing=2) as g:
            g.sweep(5)
            runs.append(states(g, [0, 1]))
    same(*runs)
