"""GPU vs oracle, draw for draw on the same seeds, through the C ABI.

Bars (relative L2 of each chain's field s and of its P, after each checkpoint):
1e-12 for the FP64 path, 2e-5 for the FP32 path; Philox words bit-exact.
Sizes cover a single tile, several tiles and non-power-of-two (ragged) lengths
(12, 24, 48, 96 have a radix-3 factor), the 32^3 workload over 200 sweeps and
the 128^3 workload with holes over 100 (FP64), and the 256^3 workload in the
launch configuration the benchmark uses.
"""
import numpy as np
import pytest

import mockgen
from oracle import philox as ph
from oracle import sampler

from gpu_helpers import TOL, check_elementwise, compare_run, gpu_sampler, need_gpu, oracle_chains, rel_l2

pytestmark = pytest.mark.gpu


def test_philox_words_bit_exact():
    torch = need_gpu()
    from paper_1402_1763_gb300 import mg_philox
    n = 1 << 16
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    for seed, c0, c1, c2, c3 in ((1, 0, 0, 0, 0), (0xDEADBEEFCAFEF00D, 2 ** 32 - 1000, 7, 3, 1),
                                 (2 ** 63 + 5, 123456, 2 ** 32 - 1, 15, 2)):
        mg_philox(seed, c0, c1, c2, c3, n, out.data_ptr())
        got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
        idx = (np.arange(n, dtype=np.uint64) + c0) & 0xFFFFFFFF
        want = np.stack(ph.philox4x32_10(idx, c1, c2, c3, seed), axis=1)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("precision", [64, 32])
def test_workload_32cubed_draw_for_draw(precision):
    need_gpu()
    w = mockgen.workload(1)
    m = w.mocks[0]
    res = compare_run(m, m.n_bins, 1, precision, [1, 2, 5, 20, 200])
    for cp, es, ep in res:
        assert es <= TOL[precision] and ep <= TOL[precision], (cp, es, ep)


@pytest.mark.parametrize("n", [8, 12, 16, 24, 48, 64, 96])
@pytest.mark.parametrize("precision", [64, 32])
def test_grid_sizes_draw_for_draw(n, precision):
    need_gpu()
    m = mockgen.make_mock(n, seed=100 + n, n_bins=max(2, n // 4))
    res = compare_run(m, m.n_bins, 7 + n, precision, [1, 3], n_chains=2)
    for cp, es, ep in res:
        assert es <= TOL[precision] and ep <= TOL[precision], (n, cp, es, ep)


@pytest.mark.parametrize("precision,cluster", [(64, 0), (32, 1), (32, 2)])
def test_workload_128cubed_holes(precision, cluster):
    need_gpu()
    w = mockgen.workload(2)
    m = w.mocks[0]
    res = compare_run(m, m.n_bins, 2, precision, [1, 3], yz_cluster=cluster)
    for cp, es, ep in res:
        assert es <= TOL[precision] and ep <= TOL[precision], (cp, es, ep)


def test_workload_128cubed_holes_fp64_over_100_sweeps():
    """The 128^3 FP64 workload with holes, draw for draw over 100 sweeps
    (checkpoints 10, 30, 100): the FP64 bar holds as the chain moves."""
    need_gpu()
    w = mockgen.workload(2)
    m = w.mocks[0]
    res = compare_run(m, m.n_bins, 2, 64, [10, 30, 100])
    for cp, es, ep in res:
        assert es <= TOL[64] and ep <= TOL[64], (cp, es, ep)


@pytest.mark.parametrize("precision,cluster", [(64, 2), (32, 1), (32, 2)])
def test_grid_192_draw_for_draw(precision, cluster):
    """192^3 (192 = 16 x 12: a radix-3 factor in every axis) in each cluster
    size built for it: FP32 with 1 and 2 CTAs per plane, FP64 with 2."""
    need_gpu()
    m = mockgen.make_mock(192, seed=192, n_bins=48)
    n_chains = 2 if precision == 32 else 1
    res = compare_run(m, 48, 13, precision, [1, 2], n_chains=n_chains, yz_cluster=cluster)
    for cp, es, ep in res:
        assert es <= TOL[precision] and ep <= TOL[precision], (cp, es, ep)


@pytest.mark.parametrize("precision,cluster", [(32, 2), (32, 4), (32, 8), (64, 4)])
def test_workload_256cubed_sampled_chains(precision, cluster):
    """Full-size 256^3 grid in the benchmark's launch form (16 chains in one
    launch for FP32); the oracle follows chains 0 and 15 for two sweeps."""
    need_gpu()
    w = mockgen.workload(3)
    m = w.mocks[0]
    n_chains = 16 if precision == 32 else 1
    follow = [0, n_chains - 1] if n_chains > 1 else [0]
    orc = oracle_chains(m, m.n_bins, 3, follow)
    with gpu_sampler(m, m.n_bins, 3, precision, n_chains=n_chains, yz_cluster=cluster) as g:
        for sw in (1, 2):
            orc.sweep(1)
            g.sweep(1)
            for k, c in enumerate(follow):
                sg, pg = g.read_s(c), g.read_pk(c)
                es = rel_l2(sg, orc.s[k])
                ep = rel_l2(pg, orc.P[k])
                assert es <= TOL[precision] and ep <= TOL[precision], (sw, c, es, ep)
                check_elementwise(precision, sg, orc.s[k], pg, orc.P[k], f"256^3 C={cluster} sweep {sw} chain {c}")


def test_batch_of_mixed_sizes_matches_independent_oracles():
    need_gpu()
    from paper_1402_1763_gb300 import Sampler
    mocks = [mockgen.make_mock(n, seed=300 + n, n_bins=b, sigma_n=s)
             for n, b, s in ((16, 4, 0.1), (24, 6, 0.5), (32, 8, 0.1))]
    seeds = [11, 12, 13]
    with Sampler.batch([m.n for m in mocks], [m.L for m in mocks], [m.N for m in mocks],
                       [m.R for m in mocks], [m.d for m in mocks], [m.n_bins for m in mocks], seeds,
                       precision=64, n_chains=2) as g:
        g.sweep(3)
        for gi, m in enumerate(mocks):
            orc = oracle_chains(m, m.n_bins, seeds[gi], [0, 1])
            orc.sweep(3)
            for c in range(2):
                sg, pg = g.read_s(2 * gi + c), g.read_pk(2 * gi + c)
                es = rel_l2(sg, orc.s[c])
                ep = rel_l2(pg, orc.P[c])
                assert es <= 1e-12 and ep <= 1e-12, (gi, c, es, ep)
                check_elementwise(64, sg, orc.s[c], pg, orc.P[c], f"batch n={m.n} chain {c}")


def test_fixed_P_and_explicit_edges_and_tau_scale():
    need_gpu()
    m = mockgen.make_mock(32, seed=41, n_bins=5)
    kf = 2 * np.pi / m.L
    edges = kf * np.array([0.5, 2.1, 4.5, 7.3, 11.2, 20.0])  # no edge on an |m| value
    P0 = np.linspace(2.0, 0.5, 6) * m.L ** 3 / m.n ** 3
    res = compare_run(m, 5, 9, 64, [1, 4], k_edges=edges, P0=P0, fix_P=True, tau_scale=0.7)
    for cp, es, ep in res:
        assert es <= 1e-12 and ep == 0.0, (cp, es, ep)


def test_set_s_read_s_round_trip_and_resume():
    need_gpu()
    m = mockgen.make_mock(24, seed=51, n_bins=6)
    rng = np.random.default_rng(0)
    s0 = rng.standard_normal(m.shape)
    with gpu_sampler(m, 6, 5, 64) as g:
        g.set_s(0, s0)
        assert rel_l2(g.read_s(0), s0) <= 1e-14
        g.sweep(6)
        s6, p6 = g.read_s(0), g.read_pk(0)
    with gpu_sampler(m, 6, 5, 64) as a:
        a.sweep(3)
        s3, p3, k3 = a.read_s(0), a.read_pk(0), a.sweep_count
    assert k3 == 3
    with gpu_sampler(m, 6, 5, 64) as b:
        b.set_s(0, s0)
        b.sweep(3)
        mid_s, mid_p = b.read_s(0), b.read_pk(0)
    with gpu_sampler(m, 6, 5, 64) as r:
        r.set_s(0, mid_s)
        r.set_pk(0, mid_p)
        r.sweep_count = 3
        r.sweep(3)
        assert rel_l2(r.read_s(0), s6) <= 1e-12
        assert rel_l2(r.read_pk(0), p6) <= 1e-12


def test_chain_statistics_match_oracle_running_moments():
    need_gpu()
    m = mockgen.make_mock(16, seed=61, n_bins=4)
    orc = oracle_chains(m, 4, 3, [0])
    xs = []
    for _ in range(30):
        orc.sweep(1)
        xs.append(orc.s[0].copy())
    xs = np.array(xs)
    with gpu_sampler(m, 4, 3, 64, record_every=1) as g:
        g.sweep(30)
        st = g.read_stats(0, maps=True)
    assert st["records"] == 30 and st["sweeps"] == 30
    np.testing.assert_allclose(st["mean"].reshape(m.shape), xs.mean(axis=0), atol=1e-12)
    np.testing.assert_allclose(st["var"].reshape(m.shape), xs.var(axis=0, ddof=1), atol=1e-11)
    np.testing.assert_array_equal(st["n_b"], orc.prob.bins.n_b)
    np.testing.assert_allclose(st["sigma_b"], orc.last_sig[0], rtol=1e-12)
    np.testing.assert_allclose(st["chi_b"], orc.last_X[0], rtol=1e-12)
    assert st["tau"] == orc.prob.tau


def test_invalid_inputs_are_rejected():
    need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MG_EUNSUPPORTED, MgError
    m = mockgen.make_mock(16, seed=71, n_bins=4)
    with pytest.raises(MgError) as e:
        gpu_sampler(m.__class__(16, m.L, m.N, np.zeros(m.shape), m.d, m.s_true, 4, 1, 0.1), 4, 1, 64)
    assert e.value.status == MG_EINVAL
    badN = m.N.copy()
    badN[m.R > 0] = -1.0
    with pytest.raises(MgError) as e:
        gpu_sampler(m.__class__(16, m.L, badN, m.R, m.d, m.s_true, 4, 1, 0.1), 4, 1, 64)
    assert e.value.status == MG_EINVAL
    badR = m.R.copy()
    badR[0, 0, 0] = -0.5
    with pytest.raises(MgError) as e:
        gpu_sampler(m.__class__(16, m.L, m.N, badR, m.d, m.s_true, 4, 1, 0.1), 4, 1, 64)
    assert e.value.status == MG_EINVAL
    with pytest.raises(MgError) as e:
        gpu_sampler(m, 0, 1, 64)
    assert e.value.status == MG_EINVAL
    m20 = mockgen.make_mock(20, seed=1, n_bins=4)
    with pytest.raises(MgError) as e:
        gpu_sampler(m20, 4, 1, 64)
    assert e.value.status == MG_EUNSUPPORTED
    with pytest.raises(MgError) as e:
        gpu_sampler(m, 4, 1, 64, yz_cluster=4)
    assert e.value.status == MG_EUNSUPPORTED
    with gpu_sampler(m, 4, 1, 64) as g:
        with pytest.raises(MgError):
            g.read_pk(5)
        with pytest.raises(MgError):
            g.set_pk(0, -np.ones(5))


def test_single_observed_voxel_and_zero_sweeps():
    need_gpu()
    m = mockgen.make_mock(8, seed=81, n_bins=2)
    R = np.zeros(m.shape)
    R[3, 4, 5] = 0.9
    N = np.ones(m.shape)
    d = np.zeros(m.shape)
    d[3, 4, 5] = 1.3
    mm = m.__class__(8, m.L, N, R, d, m.s_true, 2, 1, 0.1)
    res = compare_run(mm, 2, 4, 64, [0, 1, 4])
    for cp, es, ep in res:
        assert es <= 1e-12 and ep <= 1e-12, (cp, es, ep)


@pytest.mark.parametrize("n,precision,checkpoints", [(32, 64, [1, 3, 10]), (32, 32, [1, 3, 10]),
                                                     (256, 32, [1, 2])])
def test_largest_shell_count(n, precision, checkpoints):
    """254 shells, the most the shell table holds: at 32^3 most shells are
    narrower than the spacing of |m| (empty shells held, one-mode shells
    drawing u = G^2); at 256^3 the per-warp shell sums take 32 KB of pass X's
    shared memory, two CTAs per SM instead of three."""
    need_gpu()
    m = mockgen.make_mock(n, seed=91 + n, n_bins=254)
    res = compare_run(m, 254, 5, precision, checkpoints)
    for cp, es, ep in res:
        assert es <= TOL[precision] and ep <= TOL[precision], (n, cp, es, ep)


@pytest.mark.parametrize("precision", [64, 32])
def test_new_data_mid_chain(precision):
    """mg_set_data replaces the data d of a running chain (the messenger
    constants c = gamma d and their packed rows are rebuilt, b and tau stay):
    3 sweeps on d, then 5 on d' = 0.7 d + 0.2 R, against the oracle whose
    problem is rebuilt on d' at the same point."""
    need_gpu()
    m = mockgen.make_mock(32, seed=57, n_bins=8)
    d2 = 0.7 * m.d + 0.2 * m.R
    orc = oracle_chains(m, 8, 6, [0, 1])
    with gpu_sampler(m, 8, 6, precision, n_chains=2) as g:
        for sweeps, data_after in ((3, True), (5, False)):
            orc.sweep(sweeps)
            g.sweep(sweeps)
            for c in (0, 1):
                sg, pg = g.read_s(c), g.read_pk(c)
                es = rel_l2(sg, orc.s[c])
                ep = rel_l2(pg, orc.P[c])
                assert es <= TOL[precision] and ep <= TOL[precision], (sweeps, c, es, ep)
                check_elementwise(precision, sg, orc.s[c], pg, orc.P[c], f"set_data sweep {sweeps} chain {c}")
            if data_after:
                g.set_data(0, d2)
                orc.prob = sampler.make_problem(m.shape, m.L, m.N, m.R, d2, 8)


@pytest.mark.parametrize("n,precision,cluster", [(256, 32, 4), (256, 32, 2), (256, 64, 4), (192, 64, 2),
                                               (128, 32, 2)])
def test_set_s_read_s_round_trip_in_cluster_forms(n, precision, cluster):
    """set_s runs pass YZ in its load mode and read_s in its materialise mode;
    in the cluster forms both go through the exchange between the CTAs of a
    plane.  A field set and read back is unchanged up to the transforms'
    rounding (FP64 1e-14, FP32 1e-6 relative L2), the chain then sweeps on,
    and resuming from a saved state reproduces the same sweeps."""
    need_gpu()
    m = mockgen.make_mock(n, seed=53, n_bins=8)
    s0 = np.random.default_rng(1).standard_normal(m.shape)
    tol_rt = 1e-14 if precision == 64 else 1e-6
    with gpu_sampler(m, 8, 5, precision, yz_cluster=cluster) as g:
        g.set_s(0, s0)
        assert rel_l2(g.read_s(0), s0) <= tol_rt
        g.sweep(2)
        mid_s, mid_p = g.read_s(0), g.read_pk(0)
        g.sweep(1)
        s3, p3 = g.read_s(0), g.read_pk(0)
    with gpu_sampler(m, 8, 5, precision, yz_cluster=cluster) as r:
        r.set_s(0, mid_s)
        r.set_pk(0, mid_p)
        r.sweep_count = 2
        r.sweep(1)
        assert rel_l2(r.read_s(0), s3) <= TOL[precision] and rel_l2(r.read_pk(0), p3) <= TOL[precision]


def test_workload_128cubed_holes_fp64_over_1000_sweeps():
    """The 128^3 FP64 workload with holes draw for draw over its full 1000
    sweeps, against the oracle's chain stored by
    tests/golden/make_workload2_golden.py (the oracle takes ~0.5 s per sweep at
    this size): P(k) and s at 2048 sampled voxels after sweeps 300 and 1000,
    relative L2 within the FP64 bar 1e-12."""
    import json
    import os
    need_gpu()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "workload2_128holes_fp64_1000sweeps.json")
    with open(path) as f:
        ref = json.load(f)
    w = mockgen.workload(2)
    m = w.mocks[0]
    assert ref["workload"] == w.name and ref["seed"] == w.seeds[0]
    vox = np.asarray(ref["sample_voxels"])
    with gpu_sampler(m, m.n_bins, w.seeds[0], 64) as g:
        done = 0
        for cp in sorted(int(k) for k in ref["checkpoints"]):
            g.sweep(cp - done)
            done = cp
            want = ref["checkpoints"][str(cp)]
            s = g.read_s(0).reshape(-1)
            pg = g.read_pk(0)
            es = rel_l2(s[vox], want["s_sample"])
            ep = rel_l2(pg, want["P"])
            en = abs(np.linalg.norm(s) / want["s_norm"] - 1.0)
            assert es <= TOL[64] and ep <= TOL[64] and en <= TOL[64], (cp, es, ep, en)
            check_elementwise(64, s[vox], np.asarray(want["s_sample"]), pg, np.asarray(want["P"]),
                              f"128^3 holes, 1000-sweep record, sweep {cp}")


@pytest.mark.parametrize("precision", [64, 32])
def test_shell_chi_square_variates_match_oracle(precision):
    """The chi-square variate of each shell (Alg. 2 on shells, drawn once per
    shell in FP64 in both precision forms) against the oracle's draws, sweep by
    sweep: a shell holding one self-conjugate mode (n_b = 1: u = G^2, Alg. 2
    literally), a large shell (Marsaglia-Tsang) and an empty overflow shell
    (held)."""
    need_gpu()
    from paper_1402_1763_gb300 import Sampler
    n, L = 8, 1.0
    kc = 2 * np.pi * np.sqrt(3 * (n // 2) ** 2)  # |k| of the corner mode (n/2, n/2, n/2)
    edges = np.array([0.0, kc - 0.1, kc + 0.1])
    rng = np.random.default_rng(19)
    R = np.ones((n, n, n))
    N = np.full((n, n, n), 0.5)
    d = rng.standard_normal((n, n, n))
    prob = sampler.make_problem((n, n, n), L, N, R, d, 2, k_edges=edges)
    assert list(prob.bins.n_b) == [n ** 3 - 2, 1, 0]
    orc = sampler.Chains(prob, seed=23, chain_ids=[0, 1])
    with Sampler.single(n, L, N, R, d, 2, 23, precision=precision, n_chains=2, k_edges=edges) as g:
        for _ in range(6):
            orc.sweep(1)
            g.sweep(1)
            for c in range(2):
                st = g.read_stats(c)
                np.testing.assert_array_equal(st["n_b"], prob.bins.n_b)
                np.testing.assert_allclose(st["chi_b"][:2], orc.last_X[c][:2], rtol=1e-12)
                assert st["chi_b"][2] == 0.0  # empty shell: nothing drawn, P held
                assert rel_l2(g.read_pk(c), orc.P[c]) <= TOL[precision]
