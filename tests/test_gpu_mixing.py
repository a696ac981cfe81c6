"""Mixing sweeps (Sec. 3.3, Alg. 3 on k-shells) on the GPU against the oracle,
draw for draw, through the C ABI.

* 32^3 (the 32^3 workload's data and shells) over 6 sweeps, 2 chains, FP64
  and FP32; 64^3 (column-pair draw path) and 48^3 (single-column path).
* The 128^3 workload with holes, FP64, 2 sweeps.
* The 256^3 workload in the benchmark's launch form (16 FP32 chains, C = 4),
  chains 0 and 15 after one sweep.
* Per sweep: relative L2 of s and P within the parity tolerances, and the
  shells' acceptance flags identical.
* Alternating sweeps (mixing = 2: plain on even sweep counts, mixing on odd),
  32^3, FP64 and FP32, 6 sweeps.
* mixing with persistent is MG_EUNSUPPORTED, with fix_P MG_EINVAL.
"""
import numpy as np
import pytest

import mockgen

from gpu_helpers import TOL, check_elementwise, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def oracle_mixing(mock, n_bins, seed, chain_ids, mixing=1):
    from oracle import mixing as mx, sampler
    prob = sampler.make_problem(mock.shape, mock.L, mock.N, mock.R, mock.d, n_bins)
    cls = mx.MixingChains if mixing == 1 else mx.AlternatingChains
    return cls(prob, seed=seed, chain_ids=chain_ids)


def gpu_mixing(mock, n_bins, seed, precision, n_chains, mixing=1, **kw):
    from paper_1402_1763_gb300 import Sampler
    return Sampler.single(mock.n, mock.L, mock.N, mock.R, mock.d, n_bins, seed, precision=precision,
                          n_chains=n_chains, mixing=mixing, **kw)


def compare(mock, n_bins, seed, precision, sweeps, follow, n_chains, mixing=1, **kw):
    orc = oracle_mixing(mock, n_bins, seed, follow, mixing)
    worst = []
    with gpu_mixing(mock, n_bins, seed, precision, n_chains, mixing, **kw) as g:
        for sw in range(sweeps):
            orc.sweep(1)
            g.sweep(1)
            for k, c in enumerate(follow):
                sg, pg = g.read_s(c), g.read_pk(c)
                es = rel_l2(sg, orc.s[k])
                ep = rel_l2(pg, orc.P[k])
                check_elementwise(precision, sg, orc.s[k], pg, orc.P[k], f"mixing n={mock.n} sweep {sw} chain {c}")
                st = g.read_stats(c)
                if mixing == 1 or sw % 2 == 1:
                    assert np.array_equal(st["chi_b"], orc.last_X[k]), (sw, c, "acceptance flags differ")
                assert es <= TOL[precision] and ep <= TOL[precision], (sw, c, es, ep)
                worst.append((es, ep))
            assert g.sweep_count == sw + 1
    return worst


@pytest.mark.parametrize("precision", [64, 32])
def test_mixing_32cubed_matches_oracle(precision):
    need_gpu()
    m = mockgen.make_mock(32, seed=1, n_bins=16)
    compare(m, 16, 1, precision, 6, [0, 1], 2)


@pytest.mark.parametrize("n,precision", [(64, 64), (64, 32), (48, 64), (48, 32)])
def test_mixing_draw_paths(n, precision):
    need_gpu()
    m = mockgen.make_mock(n, seed=40 + n, n_bins=n // 4, sigma_n=0.5)
    compare(m, n // 4, 7, precision, 3, [0, 1], 2)


def test_mixing_128cubed_holes_fp64():
    need_gpu()
    w = mockgen.workload(2)
    m = w.mocks[0]
    compare(m, m.n_bins, 2, 64, 2, [0], 1)


def test_mixing_256cubed_benchmark_form():
    need_gpu()
    w = mockgen.workload(3)
    m = w.mocks[0]
    compare(m, m.n_bins, 3, 32, 1, [0, 15], 16, yz_cluster=4)


@pytest.mark.parametrize("precision", [64, 32])
def test_alternating_sweeps_match_oracle(precision):
    need_gpu()
    m = mockgen.make_mock(32, seed=1, n_bins=16)
    compare(m, 16, 1, precision, 6, [0, 1], 2, mixing=2)


def test_mixing_option_checks():
    need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MG_EUNSUPPORTED, MgError
    m = mockgen.make_mock(16, seed=2, n_bins=4)
    with pytest.raises(MgError) as e:
        gpu_mixing(m, 4, 1, 32, 1, persistent=True)
    assert e.value.status == MG_EUNSUPPORTED
    with pytest.raises(MgError) as e:
        gpu_mixing(m, 4, 1, 32, 1, fix_P=True)
    assert e.value.status == MG_EINVAL
    with pytest.raises(MgError) as e:
        gpu_mixing(m, 4, 1, 32, 1, mixing=3)
    assert e.value.status == MG_EINVAL
