"""Pins of the autograd oracle of the differentiation workload, and of the
adjoint recursion the CUDA library implements.

* The torch forward map equals the numpy oracle's fixed-P chain.
* Its autograd gradients equal central finite differences of the numpy oracle
  (a separate code path) in log P and along random directions in d.
* The transposes used by the hand-written adjoint, for the unitary real DFT F
  and its inverse F^-1 on stored modes with dof weights w (2 inside, 1 on the
  kz = 0 and n/2 planes):  F^T lam = F^-1(lam / w)  and  (F^-1)^T mu = w F mu.
* The resulting recursion, mu_{k-1} = F(b F^-1(a mu_k)), dL/dd += gamma
  F^-1(a mu_k), dL/dlogP_b += sum_{j in b} w_j (1 - a) Re(conj mu_j (a t_hat_j
  + sd xi_j / 2)), written out in numpy, reproduces the autograd gradients.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import mockgen  # noqa: E402
from oracle import adjoint, sampler  # noqa: E402


def problem(n=8, seed=3, n_bins=4):
    m = mockgen.make_mock(n, seed=seed, n_bins=n_bins)
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, n_bins)
    rng = np.random.default_rng(seed)
    logP = np.log(prob.V / prob.M) + rng.uniform(-0.5, 0.5, size=n_bins + 1)
    w = mockgen.mode_weights(n, seed)
    return m, prob, logP, w


def numpy_loss(prob, logP, d, w, K, seed):
    p2 = sampler.Problem(prob.shape, prob.L, prob.N, prob.R, d, prob.bins, prob.tau)
    ch = sampler.Chains(p2, seed=seed, chain_ids=[0], P0=np.exp(logP), fix_P=True)
    s_hat = None
    for k in range(K):
        g, z0, z1 = sampler.sweep_draws(p2.shape, seed, k, [0])
        ch.s, _, s_hat, _, _ = sampler.gibbs_sweep(p2, ch.s, ch.P, g, z0, z1, None, fix_P=True)
    return float((w * np.abs(s_hat[0]) ** 2).sum()), ch.s[0]


def test_torch_forward_equals_numpy_oracle():
    m, prob, logP, w = problem()
    L_np, s_np = numpy_loss(prob, logP, m.d, w, 3, seed=5)
    L_t = float(adjoint.chain_loss(prob, torch.tensor(logP), torch.tensor(m.d), w, 3, seed=5))
    assert L_t == pytest.approx(L_np, rel=1e-13)


def test_autograd_equals_finite_differences_of_numpy_oracle():
    m, prob, logP, w = problem()
    K, seed = 3, 5
    L, gl, gd = adjoint.loss_and_gradients(prob, logP, m.d, w, K, seed)
    h = 1e-5
    for b in range(len(logP)):
        if prob.bins.n_b[b] == 0:
            assert gl[b] == 0.0
            continue
        e = np.zeros_like(logP)
        e[b] = h
        fd = (numpy_loss(prob, logP + e, m.d, w, K, seed)[0] - numpy_loss(prob, logP - e, m.d, w, K, seed)[0]) / (2 * h)
        assert gl[b] == pytest.approx(fd, rel=1e-6, abs=1e-8 * abs(L))
    rng = np.random.default_rng(1)
    for _ in range(3):
        u = rng.standard_normal(m.shape) * (m.R > 0)
        fd = (numpy_loss(prob, logP, m.d + h * u, w, K, seed)[0]
              - numpy_loss(prob, logP, m.d - h * u, w, K, seed)[0]) / (2 * h)
        assert (gd * u).sum() == pytest.approx(fd, rel=1e-6)


def dof_weights(shape):
    nz = shape[2]
    w = np.full((shape[0], shape[1], nz // 2 + 1), 2.0)
    w[:, :, 0] = 1.0
    w[:, :, nz // 2] = 1.0
    return w


def test_transposes_of_the_orthonormal_transform():
    shape = (6, 4, 8)
    rng = np.random.default_rng(2)
    s = rng.standard_normal(shape)
    lam = rng.standard_normal((6, 4, 5)) + 1j * rng.standard_normal((6, 4, 5))
    wd = dof_weights(shape)
    F = lambda x: sampler.ont(x[None])[0]
    Finv = lambda x: sampler.ont_inv(x[None], shape)[0]
    ip = lambda u, v: float(np.sum(u.real * v.real + u.imag * v.imag))
    assert ip(F(s), lam) == pytest.approx(ip(s, Finv(lam / wd)), rel=1e-12)
    mu = rng.standard_normal(shape)
    assert ip(Finv(lam), mu) == pytest.approx(ip(lam, wd * F(mu)), rel=1e-12)


def hand_adjoint(prob, logP, d, w, K, seed):
    """The adjoint recursion of the CUDA library, in numpy FP64."""
    shape = prob.shape
    M, T = prob.M, prob.tau
    Nt = sampler.augmented_noise(prob.N, prob.R, T)
    obs = prob.R > 0
    den = np.where(obs, T * prob.R ** 2 + Nt, 1.0)
    b = np.where(obs, Nt / den, 1.0)
    gamma = np.where(obs, T * prob.R / den, 0.0)
    S = prob.S_hat(np.exp(logP))[0]
    a = S / (S + T)
    sd = np.sqrt(S * T / (S + T))
    wd = dof_weights(shape)
    F = lambda x: sampler.ont(x[None])[0]
    Finv = lambda x: sampler.ont_inv(x[None], shape)[0]
    p2 = sampler.Problem(prob.shape, prob.L, prob.N, prob.R, d, prob.bins, T)
    # forward, keeping every sweep's input s and its t_hat, xi
    s = np.zeros(shape)
    keep = []
    for k in range(K):
        g, z0, z1 = sampler.sweep_draws(shape, seed, k, [0])
        t = sampler.messenger_draw(s, d, prob.N, prob.R, T, g[0])
        th = F(t)
        xi = sampler.mode_noise(prob.bins, z0, z1)[0]
        sh = a * th + sd * xi
        keep.append((th, xi))
        s = Finv(sh)
    L = float((w * np.abs(sh) ** 2).sum())
    mu = 2 * w * sh / wd
    gl = np.zeros_like(logP)
    gd = np.zeros(shape)
    idx = prob.bins.bin_of
    for k in range(K - 1, -1, -1):
        th, xi = keep[k]
        contrib = wd * (1 - a) * (np.conj(mu) * (a * th + 0.5 * sd * xi)).real
        gl += np.bincount(idx[idx >= 0], weights=contrib[idx >= 0], minlength=len(logP))
        lam_t = Finv(a * mu)
        gd += gamma * lam_t
        mu = F(b * lam_t)
    return L, gl, gd


def test_hand_adjoint_recursion_equals_autograd():
    m, prob, logP, w = problem(n=8, seed=7, n_bins=5)
    K, seed = 4, 0
    L, gl, gd = adjoint.loss_and_gradients(prob, logP, m.d, w, K, seed)
    Lh, glh, gdh = hand_adjoint(prob, logP, m.d, w, K, seed)
    assert Lh == pytest.approx(L, rel=1e-13)
    np.testing.assert_allclose(glh, gl, rtol=1e-10, atol=1e-10 * np.abs(gl).max())
    np.testing.assert_allclose(gdh, gd, rtol=1e-10, atol=1e-10 * np.abs(gd).max())
