"""Gradients of a fixed-P chain of sweeps by torch FP64 autograd (CPU).

ORACLE — test infrastructure only (see ``oracle/sampler.py``).  The forward
map re-expresses, in torch ops, exactly the oracle's fixed-P sweep (Sec. 3.1,
Alg. 1: messenger draw, orthonormal transform, signal draw, inverse transform)
with the noise held fixed (the same Philox normals ``sampler.sweep_draws``
produces).  The loss of the differentiation workload is
    L = sum_j w_j |s_hat_K,j|^2
over the stored modes of the K-th sample; gradients are taken with respect to
log P (per shell) and the data d.  torch's autograd provides the derivatives;
nothing here states an adjoint by hand.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sampler


def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64)


def sweep_fixed_P(prob: sampler.Problem, s, logP, d, g, z0, z1):
    """One sweep with P = exp(logP) fixed and explicit noise; torch FP64.

    s: (M,) field; logP: (B+1,); d: data; g: messenger normals; z0, z1: the
    mode normals that build xi.  Returns (s_new, s_hat).
    """
    shape = prob.shape
    M = prob.M
    T = prob.tau
    N = _t(prob.N)
    R = _t(prob.R)
    Nt = torch.clamp(N - R * T * R, min=0.0)
    obs = R ** 2 > 0
    denom = torch.where(obs, T * R ** 2 + Nt, torch.ones_like(R))
    mu = torch.where(obs, T / denom * R * d + Nt / denom * s, s)
    var = torch.where(obs, T * Nt / denom, torch.full_like(R, T))
    t = mu + torch.sqrt(var) * g
    t_hat = torch.fft.rfftn(t, dim=(-3, -2, -1)) / np.sqrt(M)
    idx = torch.as_tensor(np.where(prob.bins.bin_of >= 0, prob.bins.bin_of, 0))
    dc = torch.as_tensor(prob.bins.bin_of < 0)
    S = (M / prob.V) * torch.exp(logP[idx])
    S = torch.where(dc, torch.zeros_like(S), S)
    a = S / (S + T)
    v = S * T / (S + T)
    sd = torch.where(dc, torch.zeros_like(v), torch.sqrt(torch.where(dc, torch.ones_like(v), v)))
    xi = torch.as_tensor(sampler.mode_noise(prob.bins, z0, z1))
    s_hat = a * t_hat + sd * xi
    s_new = torch.fft.irfftn(s_hat, s=shape, dim=(-3, -2, -1)) * np.sqrt(M)
    return s_new, s_hat


def chain_loss(prob, logP, d, w, K, seed, chain_id=0, sweep0=0, s0=None):
    """L(logP, d) after K fixed-P sweeps from s0 (default 0), noise of sweeps
    sweep0 .. sweep0+K-1 of chain ``chain_id``."""
    s = torch.zeros(prob.shape, dtype=torch.float64) if s0 is None else _t(s0)
    s_hat = None
    for k in range(K):
        g, z0, z1 = sampler.sweep_draws(prob.shape, seed, sweep0 + k, [chain_id])
        s, s_hat = sweep_fixed_P(prob, s, logP, d, _t(g[0]), z0[0], z1[0])
    return (_t(w) * (s_hat.real ** 2 + s_hat.imag ** 2)).sum()


def loss_and_gradients(prob, logP, d, w, K, seed, chain_id=0, sweep0=0, s0=None):
    """(L, dL/dlogP, dL/dd) as numpy FP64."""
    lp = _t(logP).clone().requires_grad_(True)
    dd = _t(d).clone().requires_grad_(True)
    L = chain_loss(prob, lp, dd, w, K, seed, chain_id, sweep0, s0)
    gl, gd = torch.autograd.grad(L, (lp, dd))
    return float(L.detach()), gl.numpy(), gd.numpy()
