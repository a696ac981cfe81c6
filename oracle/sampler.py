"""Plain FP64 CPU messenger Gibbs sampler (Jasche & Lavaux 2014).

ORACLE — test infrastructure only.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline use it.  It shares no code with the CUDA library: it is numpy in FP64,
written from the paper's equations in the order the paper gives them.

Conventions (where the paper leaves them open, these are the readings taken):

* Grid n = (nx, ny, nz), side L = (Lx, Ly, Lz), M = nx*ny*nz voxels, V = Lx*Ly*Lz.
  Voxel index i = (ix*ny + iy)*nz + iz (z fastest).  Arrays have shape
  (chains, nx, ny, nz).
* The orthonormal transform ("ONT", Sec. 3.1, Alg. 1) is the unitary real DFT
  s_hat = rfftn(s) / sqrt(M).  Stored modes have shape (nx, ny, nz//2 + 1) and
  index j = (kx*ny + ky)*(nz//2 + 1) + kz.  Because the transform is unitary the
  messenger covariance is the same in both bases: T_hat = T = tau (the remark
  after the t-conditional in Sec. 3.1).
* Signal covariance S_hat_k = (M / V) P(bin(k)), and S_hat = 0 at k = 0.
* Random draws: Philox4x32-10 keyed by the seed with counter
  (index, sweep, chain, stream) (``oracle.philox``): the messenger normals
  (stream 0), the modes' complex noise (stream 1, two modes per call) and one
  chi-square variate per shell (stream 5); see ``sweep_draws`` and
  ``chi2_shell_draws``.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import philox as ph
from .bins import BinTable, make_bins


# --------------------------------------------------------------------------
# Sec. 2: the messenger covariance T = tau * 1 and the augmented noise N~.
# --------------------------------------------------------------------------

def messenger_tau(N, R, tau_scale: float = 1.0) -> float:
    """tau per Sec. 2: 0 < tau <= [(R^-1)^T N R^-1]_i for all observed i.

    For a diagonal response R the bound is N_i / R_i^2; the paper takes the
    minimum over the observed domain (R_i > 0).  ``tau_scale`` in (0, 1] scales
    it down so that N~ stays strictly positive everywhere.
    """
    obs = R > 0
    if not np.any(obs):
        raise ValueError("no observed voxel (R > 0 nowhere)")
    return float(tau_scale * np.min(N[obs] / R[obs] ** 2))


def augmented_noise(N, R, tau: float):
    """N~ = N - R^T T R (Sec. 2), elementwise for diagonal N, R and T = tau.

    At the voxel(s) where tau meets its bound N~ is zero in exact arithmetic;
    the rounded difference can come out an ulp below zero, so it is clamped at
    zero (N~ must not be negative, Sec. 2).
    """
    return np.maximum(N - R * tau * R, 0.0)


# --------------------------------------------------------------------------
# Sec. 3.1 / Alg. 1, first loop: the messenger draw t | s, d.
# --------------------------------------------------------------------------

def messenger_moments(s, d, N, R, tau: float):
    """Mean and variance of t_i | s_i, d_i (Sec. 3.1, the two piecewise
    formulas for mu^t and (sigma^t)^2).

    Observed voxels (R_i^2 > 0):
        mu   = T R d / (T R^2 + N~) + N~ s / (T R^2 + N~)
        var  = T N~ / (T R^2 + N~)
    Unobserved voxels: mu = s, var = T.
    """
    T = tau
    Nt = augmented_noise(N, R, tau)
    obs = R ** 2 > 0
    denom = np.where(obs, T * R ** 2 + Nt, 1.0)
    mu = np.where(obs, T / denom * R * d + Nt / denom * s, s)
    var = np.where(obs, T * Nt / denom, T)
    return mu, var


def messenger_draw(s, d, N, R, tau: float, g):
    """t_i = mu^t_i + sqrt((sigma^t_i)^2) G_i (Alg. 1, first loop)."""
    mu, var = messenger_moments(s, d, N, R, tau)
    return mu + np.sqrt(var) * g


# --------------------------------------------------------------------------
# The orthonormal transform (Sec. 3.1; Alg. 1 "ONT").
# --------------------------------------------------------------------------

def ont(x):
    """Unitary real DFT over the last three axes: rfftn(x) / sqrt(M)."""
    shape = x.shape[-3:]
    M = shape[0] * shape[1] * shape[2]
    return np.fft.rfftn(x, axes=(-3, -2, -1)) / np.sqrt(M)


def ont_inv(xh, shape):
    """Inverse of ``ont``: irfftn(xh) * sqrt(M) for a real grid of ``shape``."""
    M = shape[0] * shape[1] * shape[2]
    return np.fft.irfftn(xh, s=shape, axes=(-3, -2, -1)) * np.sqrt(M)


# --------------------------------------------------------------------------
# Sec. 3.1 / Alg. 1, second loop: the signal draw s_hat | t_hat, S_hat.
# --------------------------------------------------------------------------

def mode_moments(t_hat, S_hat, T_hat: float):
    """mu = S/(S + T) t_hat and var = S T/(S + T) per mode (Sec. 3.1)."""
    mu = S_hat / (S_hat + T_hat) * t_hat
    var = S_hat * T_hat / (S_hat + T_hat)
    return mu, var


def mode_noise(bins: BinTable, z0, z1):
    """Complex unit noise xi per stored mode of a real field.

    Interior modes (0 < kz < nz/2): xi = (z0 + i z1)/sqrt(2).  On the kz = 0 and
    kz = nz/2 planes both k and -k are stored; of each pair the member with
    the smaller key ky*nx + kx (so the row 0 < ky < ny/2, or, in the rows
    ky = 0 and ny/2, the smaller kx) is canonical and draws
    (z0 + i z1)/sqrt(2) from its own normals, its partner takes the complex
    conjugate of that same value.  Self-conjugate modes (k = -k) are real:
    xi = z0.  This keeps s_hat the transform of a real field while every
    full-grid dof has unit variance.  (With the pairing of ``sweep_draws``, a
    row ky of an edge plane and its partner row ny - ky then take all their
    noise from the calls of one of the two rows.)
    """
    zc = (z0 + 1j * z1) / np.sqrt(2.0)
    flat_c = zc.reshape(zc.shape[:-3] + (-1,))
    flat_r = z0.reshape(z0.shape[:-3] + (-1,))
    part = bins.partner.reshape(-1)
    own = np.arange(part.size)
    nx, ny, nz = bins.shape
    nh = nz // 2 + 1

    def key(j):  # ky * nx + kx of stored index j = (kx * ny + ky) * nh + kz
        return ((j // nh) % ny) * nx + j // (ny * nh)

    xi = flat_c.copy()
    plane = bins.edge_plane.reshape(-1)
    selfc = plane & (part == own)
    lower = plane & (key(part) < key(own))
    xi[..., selfc] = flat_r[..., selfc]
    xi[..., lower] = np.conj(flat_c[..., part[lower]])
    return xi.reshape(zc.shape)


def signal_draw(t_hat, S_hat, T_hat: float, xi):
    """s_hat_i = mu_i + sqrt(var_i) G_i (Alg. 1, second loop)."""
    mu, var = mode_moments(t_hat, S_hat, T_hat)
    return mu + np.sqrt(var) * xi


# --------------------------------------------------------------------------
# Sec. 3.2 / Alg. 2 on k-shells: the covariance draw P | s.
# --------------------------------------------------------------------------

def shell_sums(bins: BinTable, s_hat):
    """sigma_b = sum_{j in b} w_j |s_hat_j|^2 over the stored modes of shell b
    (w_j its dof weight).  The DC mode belongs to no shell.  Shape (chains, B+1).
    """
    B1 = bins.n_bins + 1
    idx = bins.bin_of.reshape(-1)
    w = bins.weight.reshape(-1).astype(np.float64)
    keep = idx >= 0
    C = s_hat.shape[0]
    sig = np.zeros((C, B1))
    a2 = (np.abs(s_hat) ** 2).reshape(C, -1)
    for c in range(C):
        sig[c] = np.bincount(idx[keep], weights=(w * a2[c])[keep], minlength=B1)
    return sig


# Marsaglia & Tsang (2000), "A simple method for generating gamma variables",
# ACM TOMS 26(3): for shape alpha >= 1 with d = alpha - 1/3, c = 1/sqrt(9 d),
# x a unit normal and v = (1 + c x)^3, the value d v is accepted when v > 0 and
# ln U < x^2/2 + d - d v + d ln v (U uniform); accepted values are Gamma(alpha, 1).
CHI2_MAX_ATTEMPTS = 64


def chi2_shell_draws(n_b, seed: int, sweep: int, chain_ids: Sequence[int]):
    """X_b ~ chi^2_{n_b} for every shell b and chain (the chi-square variate of
    Alg. 2 on shells, drawn once per shell), shape (chains, B+1).

    Random numbers: Philox stream 5, attempt k of shell b uses the call
    (b + 256 k, sweep, chain, 5).
      n_b = 1:  X = z^2, z the first Box-Muller normal of call (b, sweep, chain, 5)
                (Alg. 2 literally: u = G^2).
      n_b >= 2: X = 2 Gamma(n_b / 2) by Marsaglia & Tsang with alpha = n_b/2 >= 1:
                attempt k takes x = the first Box-Muller normal of words (w0, w1)
                and U = U(w2); the first accepted attempt gives X = 2 d v.
      n_b = 0, or no acceptance in 64 attempts: nan (the shell keeps its P).
    """
    n_b = np.asarray(n_b, dtype=np.int64)
    B1 = n_b.size
    C = len(chain_ids)
    X = np.full((C, B1), np.nan)
    for ci, cid in enumerate(chain_ids):
        for b in range(B1):
            nb = int(n_b[b])
            if nb == 0:
                continue
            if nb == 1:
                w = ph.philox4x32_10(np.uint64(b), sweep, cid, ph.STREAM_CHI2, seed)
                z = float(ph.box_muller(w[0], w[1])[0])
                X[ci, b] = z * z
                continue
            alpha = 0.5 * nb
            d = alpha - 1.0 / 3.0
            c = 1.0 / np.sqrt(9.0 * d)
            for k in range(CHI2_MAX_ATTEMPTS):
                w = ph.philox4x32_10(np.uint64(b + 256 * k), sweep, cid, ph.STREAM_CHI2, seed)
                x = float(ph.box_muller(w[0], w[1])[0])
                v = 1.0 + c * x
                if v <= 0.0:
                    continue
                v = v * v * v
                u = float(ph.uniform_open0(w[2]))
                if np.log(u) < 0.5 * x * x + d - d * v + d * np.log(v):
                    X[ci, b] = 2.0 * d * v
                    break
    return X


def covariance_draw(sig, X, n_b, P_prev, V: float, M: int):
    """Inverse-gamma draw of each shell's power (Sec. 3.2, Alg. 2).

    With Jeffreys' prior 1/S_b and the Gaussian likelihood of the n_b real
    degrees of freedom in shell b, S_b | s ~ InvGamma(n_b/2, sigma_b/2), i.e.
    S_b = sigma_b / X_b with X_b ~ chi^2_{n_b}; for n_b = 1 this is exactly
    Alg. 2 (u = G^2, S = |s|^2/u).  P_b = (V/M) S_b.  Empty shells, and shells
    whose sigma_b or X_b is not positive and finite, keep their previous value.
    """
    P = np.array(P_prev, dtype=np.float64, copy=True)
    ok = (np.broadcast_to(n_b > 0, P.shape) & np.isfinite(X) & (X > 0)
          & np.isfinite(sig) & (sig > 0))
    P[ok] = (V / M) * sig[ok] / X[ok]
    return P


# --------------------------------------------------------------------------
# Random draws for one sweep (Philox keyed by seed; Sec. 3.4's per-core RNGs).
# --------------------------------------------------------------------------

def sweep_draws(shape, seed: int, sweep: int, chain_ids: Sequence[int]):
    """The unit normals one sweep's messenger and signal draws consume, per chain.

    Messenger: voxel i uses call (i // 4, sweep, chain, 0), normal number i % 4.
    Modes: the stored modes kx and nx - kx at the same (ky, kz) share one call,
    that of the stored index j' = (kx'*ny + ky)*(nz//2 + 1) + kz with
    kx' = min(kx, nx - kx); the member with kx <= nx/2 takes the normals
    (z0, z1) of words (w0, w1), the other (z2, z3) of words (w2, w3).
    Returns g (chains, nx, ny, nz) and z0, z1 (chains, nx, ny, nz//2+1): the two
    normals behind each stored mode's complex noise (``mode_noise``).
    """
    nx, ny, nz = shape
    M = nx * ny * nz
    nh = nz // 2 + 1
    hx = nx // 2
    cid = np.asarray(list(chain_ids), dtype=np.uint64)
    C = cid.size
    calls = np.arange((M + 3) // 4, dtype=np.uint64)[None, :]
    n4 = ph.normals4(calls, sweep, cid[:, None], ph.STREAM_MESSENGER, seed)
    g = np.stack(n4, axis=-1).reshape(C, -1)[:, :M].reshape((C, nx, ny, nz))
    kxp = np.arange(hx + 1, dtype=np.uint64)[:, None, None]
    jp = (kxp * np.uint64(ny) + np.arange(ny, dtype=np.uint64)[None, :, None]) * np.uint64(nh) \
        + np.arange(nh, dtype=np.uint64)[None, None, :]
    zz = ph.normals4(jp[None], sweep, cid[:, None, None, None], ph.STREAM_MODES, seed)
    z0 = np.empty((C, nx, ny, nh))
    z1 = np.empty((C, nx, ny, nh))
    z0[:, :hx + 1] = zz[0]
    z1[:, :hx + 1] = zz[1]
    hi = np.arange(hx + 1, nx)
    z0[:, hi] = zz[2][:, nx - hi]
    z1[:, hi] = zz[3][:, nx - hi]
    return g, z0, z1


# --------------------------------------------------------------------------
# The problem and the chain driver.
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Inputs of the joint problem Pi(s, S | d) with d = R s + eps (Sec. 2)."""

    shape: tuple
    L: tuple
    N: np.ndarray
    R: np.ndarray
    d: np.ndarray
    bins: BinTable
    tau: float

    @property
    def M(self) -> int:
        return int(np.prod(self.shape))

    @property
    def V(self) -> float:
        return float(np.prod(self.L))

    def S_hat(self, P):
        """S_hat per stored mode for each chain's P (chains, B+1): (M/V) P[bin];
        zero at the DC mode."""
        P = np.atleast_2d(P)
        idx = self.bins.bin_of
        S = (self.M / self.V) * P[:, np.where(idx >= 0, idx, 0)]
        S[:, idx < 0] = 0.0
        return S


def make_problem(shape, L, N, R, d, n_bins: int, k_edges=None,
                 tau_scale: float = 1.0) -> Problem:
    shape = tuple(int(v) for v in shape)
    L = tuple(float(v) for v in (L if np.ndim(L) else (L, L, L)))
    N = np.asarray(N, dtype=np.float64).reshape(shape)
    R = np.asarray(R, dtype=np.float64).reshape(shape)
    d = np.asarray(d, dtype=np.float64).reshape(shape)
    bins = make_bins(shape, L, n_bins, k_edges)
    tau = messenger_tau(N, R, tau_scale)
    return Problem(shape, L, N, R, d, bins, tau)


def gibbs_sweep(prob: Problem, s, P, g, z0, z1, X, fix_P: bool = False):
    """One Gibbs sweep with explicit noise: Alg. 1 then Alg. 2 (Sec. 3.2: the
    sequential iteration of the two samples the joint posterior).

    s: (C, nx, ny, nz), P: (C, B+1), X: (C, B+1) chi-square variates (unused
    with fix_P).  Returns (s_new, P_new, s_hat, sig, X).  The map is affine in
    (s, noise) for fixed P.
    """
    t = messenger_draw(s, prob.d, prob.N, prob.R, prob.tau, g)
    t_hat = ont(t)
    xi = mode_noise(prob.bins, z0, z1)
    s_hat = signal_draw(t_hat, prob.S_hat(P), prob.tau, xi)
    s_new = ont_inv(s_hat, prob.shape)
    sig = shell_sums(prob.bins, s_hat)
    if fix_P:
        P_new = np.array(P, dtype=np.float64, copy=True)
    else:
        P_new = covariance_draw(sig, X, prob.bins.n_b, P, prob.V, prob.M)
    return s_new, P_new, s_hat, sig, X


class Chains:
    """A batch of chains on one problem, driven by Philox draws.

    State: s (C, nx, ny, nz) starting at 0, P (C, B+1) starting flat at
    S_hat = 1 unless P0 is given, sweep counter starting at 0.
    """

    def __init__(self, prob: Problem, seed: int, chain_ids: Sequence[int],
                 P0: Optional[np.ndarray] = None, fix_P: bool = False, start_dispersion: float = 0.0):
        self.prob = prob
        self.seed = int(seed)
        self.chain_ids = list(chain_ids)
        C = len(self.chain_ids)
        B1 = prob.bins.n_bins + 1
        self.s = np.zeros((C,) + prob.shape)
        if P0 is None:
            P0 = np.full(B1, prob.V / prob.M)
        self.P = np.tile(np.asarray(P0, dtype=np.float64).reshape(1, B1), (C, 1))
        if start_dispersion > 0.0:
            # over-dispersed starts (Sec. 3.4): P_b * exp(sigma z_b), z_b from
            # Philox call (b, 0, chain, 2)
            b = np.arange(B1, dtype=np.uint64)[None, :]
            cid = np.asarray(self.chain_ids, dtype=np.uint64)[:, None]
            w = ph.philox4x32_10(b, 0, cid, ph.STREAM_START, self.seed)
            z = ph.box_muller(w[0], w[1])[0]
            self.P = self.P * np.exp(start_dispersion * z)
        self.fix_P = fix_P
        self.sweeps_done = 0
        self.last_sig = None
        self.last_X = None

    def sweep(self, n: int = 1):
        for _ in range(n):
            g, z0, z1 = sweep_draws(self.prob.shape, self.seed, self.sweeps_done, self.chain_ids)
            X = chi2_shell_draws(self.prob.bins.n_b, self.seed, self.sweeps_done, self.chain_ids)
            self.s, self.P, _, self.last_sig, self.last_X = gibbs_sweep(
                self.prob, self.s, self.P, g, z0, z1, X, self.fix_P)
            self.sweeps_done += 1
        return self
