"""The hand-written CUDA adjoint of K fixed-P sweeps (differentiation form),
through the C ABI and the torch.autograd binding.

* 16^3 copy, FP64 and FP32: loss and gradients against torch FP64 autograd of
  the oracle's sweep (relative L2: 1e-10 for FP64, 1e-4 for FP32).
* Full 128^3 FP32 workload (32 shells, K = 8, seeded weights): gradients
  against central finite differences with h = 1e-3, evaluated with the FP64
  library on the same GPU, in every non-empty log P shell and along random
  directions in d; the chain state, P and sweep counter are unchanged after
  the call; the autograd binding returns the same gradients.
* The work buffers kept between calls: a call after calls with a smaller K
  (the checkpoints grow) and on another chain returns bit for bit what the
  same call returns in a fresh context.
"""
import numpy as np
import pytest

import mockgen
from oracle import adjoint as oadj
from oracle import sampler

from gpu_helpers import gpu_sampler, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def copy_problem(n, n_bins, seed):
    m = mockgen.make_mock(n, seed=seed, n_bins=n_bins)
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, n_bins)
    rng = np.random.default_rng(seed)
    logP = np.log(prob.V / prob.M) + rng.uniform(-1.0, 1.0, size=n_bins + 1)
    w = mockgen.mode_weights(n, seed)
    return m, prob, logP, w


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_adjoint_16cubed_against_torch_autograd(precision, tol):
    need_gpu()
    m, prob, logP, w = copy_problem(16, 8, 5)
    K = 8
    L0, gl0, gd0 = oadj.loss_and_gradients(prob, logP, m.d, w, K, seed=5)
    with gpu_sampler(m, 8, 5, precision) as g:
        L, gl, gd = g.adjoint(0, K, logP, w)
    assert abs(L - L0) <= tol * abs(L0)
    assert rel_l2(gl, gl0) <= tol, rel_l2(gl, gl0)
    assert rel_l2(gd, gd0) <= tol, rel_l2(gd, gd0)


def test_adjoint_128cubed_fp32_against_central_differences():
    need_gpu()
    w5 = mockgen.workload(5)
    m = w5.mocks[0]
    nb, K, h = m.n_bins, 8, 1e-3
    wts = mockgen.mode_weights(m.n, 5)
    V, M = m.L ** 3, m.n ** 3
    logP = np.log(V / M) + np.random.default_rng(9).uniform(-1.0, 1.0, size=nb + 1)
    with gpu_sampler(m, nb, 5, 32) as g32, gpu_sampler(m, nb, 5, 64) as g64:
        g32.sweep(2)
        g64.sweep(2)
        s_before, p_before, k_before = g32.read_s(0), g32.read_pk(0), g32.sweep_count
        L, gl, gd = g32.adjoint(0, K, logP, wts)
        assert np.array_equal(g32.read_s(0), s_before)
        assert np.array_equal(g32.read_pk(0), p_before) and g32.sweep_count == k_before
        n_b = g32.read_stats(0)["n_b"]
        L64 = g64.adjoint(0, K, logP, wts)[0]
        assert abs(L - L64) <= 1e-4 * abs(L64)

        def loss(lp, d=None):
            if d is not None:
                g64.set_data(0, d)
            return g64.adjoint(0, K, lp, wts)[0]

        for b in range(nb + 1):
            e = np.zeros(nb + 1)
            e[b] = h
            fd = (loss(logP + e) - loss(logP - e)) / (2 * h)
            if n_b[b] == 0:
                assert gl[b] == 0.0
                continue
            assert abs(gl[b] - fd) <= 2e-3 * abs(fd) + 1e-6 * abs(L), (b, gl[b], fd)
        rng = np.random.default_rng(3)
        for _ in range(2):
            u = rng.standard_normal(m.shape) * (m.R > 0)
            fd = (loss(logP, m.d + h * u) - loss(logP, m.d - h * u)) / (2 * h)
            g64.set_data(0, m.d)
            assert abs((gd * u).sum() - fd) <= 2e-3 * abs(fd), ((gd * u).sum(), fd)


def test_adjoint_256cubed_cluster_forms_agree():
    """At 256^3 the FP32 adjoint's y/z pass runs in thread-block clusters, its
    planes split over 4 (or 2) CTAs that exchange through distributed shared
    memory, a path the smaller grids above (one CTA per plane) do not take.
    The adjoint arithmetic they share is checked above; here the two cluster
    forms must give the same loss and gradients."""
    need_gpu()
    w = mockgen.workload(3)
    m = w.mocks[0]
    nb, K = m.n_bins, 2
    wts = mockgen.mode_weights(m.n, 5)
    V, M = m.L ** 3, m.n ** 3
    logP = np.log(V / M) + np.random.default_rng(11).uniform(-1.0, 1.0, size=nb + 1)
    out = {}
    for c in (4, 2):
        with gpu_sampler(m, nb, 3, 32, yz_cluster=c) as g:
            g.sweep(1)
            out[c] = g.adjoint(0, K, logP, wts)
    (L4, gl4, gd4), (L2, gl2, gd2) = out[4], out[2]
    assert np.isfinite(L4) and np.all(np.isfinite(gl4)) and np.all(np.isfinite(gd4))
    assert abs(L4 - L2) <= 1e-6 * abs(L2), (L4, L2)
    assert rel_l2(gl4, gl2) <= 1e-5 and rel_l2(gd4, gd2) <= 1e-5, (rel_l2(gl4, gl2), rel_l2(gd4, gd2))


def test_adjoint_128cubed_cluster_matches_single_cta():
    """At 128^3 the FP32 y/z pass is built both with one CTA per plane (the form
    checked against central differences above) and with clusters of 2: the
    adjoint must agree between them."""
    need_gpu()
    w5 = mockgen.workload(5)
    m = w5.mocks[0]
    nb, K = m.n_bins, 8
    wts = mockgen.mode_weights(m.n, 5)
    V, M = m.L ** 3, m.n ** 3
    logP = np.log(V / M) + np.random.default_rng(9).uniform(-1.0, 1.0, size=nb + 1)
    out = {}
    for c in (1, 2):
        with gpu_sampler(m, nb, 5, 32, yz_cluster=c) as g:
            g.sweep(2)
            out[c] = g.adjoint(0, K, logP, wts)
    (L1, gl1, gd1), (L2, gl2, gd2) = out[1], out[2]
    assert abs(L1 - L2) <= 1e-6 * abs(L1), (L1, L2)
    assert rel_l2(gl2, gl1) <= 1e-5 and rel_l2(gd2, gd1) <= 1e-5, (rel_l2(gl2, gl1), rel_l2(gd2, gd1))


def test_autograd_binding_returns_the_adjoint():
    torch = need_gpu()
    from paper_1402_1763_gb300.autograd import gibbs_loss
    m, prob, logP, w = copy_problem(16, 8, 6)
    with gpu_sampler(m, 8, 6, 64) as g:
        L_ref, gl_ref, gd_ref = g.adjoint(0, 4, logP, w)
        lp = torch.tensor(logP, requires_grad=True)
        d = torch.tensor(m.d, requires_grad=True)
        L = gibbs_loss(lp, d, g, 0, 4, w)
        L.backward()
    assert float(L.detach()) == L_ref
    np.testing.assert_array_equal(lp.grad.numpy(), gl_ref)
    np.testing.assert_array_equal(d.grad.numpy(), gd_ref)


def test_adjoint_buffers_reused_across_calls():
    need_gpu()
    m, prob, logP, w = copy_problem(16, 8, 7)
    with gpu_sampler(m, 8, 7, 64, n_chains=2) as fresh:
        L0, gl0, gd0 = fresh.adjoint(0, 5, logP, w)
    with gpu_sampler(m, 8, 7, 64, n_chains=2) as g:
        g.adjoint(0, 2, logP, w)
        g.adjoint(1, 3, logP[::-1].copy(), w)
        L, gl, gd = g.adjoint(0, 5, logP, w)
    assert L == L0
    np.testing.assert_array_equal(gl, gl0)
    np.testing.assert_array_equal(gd, gd0)
