"""The mixing sampler of Sec. 3.3 (Alg. 3) on k-shells, FP64.

ORACLE — test infrastructure only (see ``oracle/sampler.py``).

Sec. 3.3 samples the signal and its covariance jointly given the messenger
field, after the change of coordinates s_hat = sqrt(S_hat) x_hat.  Written out
for a shell b of n_b real degrees of freedom c (stored mode j counted with its
dof weight w_j) with Jeffreys' prior 1/S_b, unitary transform and T_hat = tau:

* x_j | S_b, t_hat is Gaussian with mean sqrt(S) t_hat_j / (S + tau) and
  variance tau / (S + tau) per dof (completing the square in the two Gaussian
  factors; the paper's printed mean carries an extra factor tau).  With the
  complex unit noise xi of the plain sampler this is x_j = s_hat_j / sqrt(S)
  for the plain signal draw s_hat_j = a t_hat_j + sd xi_j.
* u_b = sqrt(S_b) | x, t_hat has density proportional to
      u^-1 exp(-B (u - A/B)^2 / (2 tau)),   u > 0,
  A = sum_j w_j Re(conj(x_j) t_hat_j),  B = sum_j w_j |x_j|^2:
  the prior 1/S, the Jacobian S^(n_b/2) of s -> x and the normalisation
  S^(-n_b/2) of the signal prior leave S^-1, and dS = 2u du turns it into u^-1
  (the paper's printed factors sqrt(S) and u^2 do not follow from its own
  change of coordinates).
* Metropolis-Hastings with the independence proposal u' ~ N(A/B, tau/B)
  truncated to u' > 0 (Alg. 3) then accepts with probability min(1, u/u').
* s_hat_j = u_b x_j for the new u_b, and s = ONT^-1(s_hat).

For one dof per shell these are Alg. 3's per-element steps.

Random numbers (Philox stream 4): attempt k of shell b uses the call
(b + 256 k, sweep, chain, 4), k < 64.  The truncated normal is drawn for
a = -mu/sigma <= 1/2 by plain rejection (z = the first Box-Muller normal of
words (w0, w1); keep if z > a) and for a > 1/2 by Robert's (1995) exponential
rejection (lambda = (a + sqrt(a^2 + 4))/2; z = a - ln(U(w0))/lambda; keep if
U(w1) <= exp(-(z - lambda)^2 / 2)); u' = mu + sigma z.  The acceptance
uniform is U(w3) of attempt 0.  If no attempt succeeds (probability far below
1e-8) the shell keeps its value.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import philox as ph
from . import sampler as sp

STREAM_MIXING = ph.STREAM_MIXING
MAX_ATTEMPTS = 64
ROBERT_FROM = 0.5


def truncated_normal_positive(mu: float, sigma: float, words) -> Optional[float]:
    """A draw from N(mu, sigma^2) restricted to (0, inf), from the attempt
    words ``words[k] = (w0, w1, w2, w3)`` (k = 0, 1, ...); None if every attempt
    is rejected."""
    a = -mu / sigma
    if a <= ROBERT_FROM:
        for w in words:
            z = float(ph.box_muller(w[0], w[1])[0])
            if z > a:
                return mu + sigma * z
        return None
    lam = 0.5 * (a + np.sqrt(a * a + 4.0))
    for w in words:
        z = a - float(np.log(ph.uniform_open0(w[0]))) / lam
        if float(ph.uniform_open0(w[1])) <= float(np.exp(-0.5 * (z - lam) ** 2)):
            return mu + sigma * z
    return None


class AttemptWords:
    """The Philox calls of shell b's proposal: item k is attempt k's four
    words (call (b + 256 k, sweep, chain, 4)); computed on first use."""

    def __init__(self, seed: int, sweep: int, chain: int, b: int):
        self.key = (int(seed), int(sweep), int(chain), int(b))
        self.cache = {}

    def __len__(self):
        return MAX_ATTEMPTS

    def __getitem__(self, k: int):
        if not 0 <= k < MAX_ATTEMPTS:
            raise IndexError(k)
        if k not in self.cache:
            seed, sweep, chain, b = self.key
            w = ph.philox4x32_10(np.uint64(b + 256 * k), sweep, chain, STREAM_MIXING, seed)
            self.cache[k] = tuple(int(x) for x in w)
        return self.cache[k]


def attempt_words(seed: int, sweep: int, chain: int, b: int):
    """Shell b's proposal words for this sweep and chain (lazily computed)."""
    return AttemptWords(seed, sweep, chain, b)


def shell_update(u: float, A: float, B: float, tau: float, words):
    """One Metropolis-Hastings update of u = sqrt(S_b) (Alg. 3 on a shell).

    Returns (u_new, accepted)."""
    if not (B > 0.0 and np.isfinite(A) and np.isfinite(B)):
        return u, False
    mu = A / B
    sigma = np.sqrt(tau / B)
    up = truncated_normal_positive(mu, sigma, words)
    if up is None:
        return u, False
    alpha = float(ph.uniform_open0(words[0][3]))
    if alpha * up < u:
        return up, True
    return u, False


def mixing_sweep(prob: sp.Problem, s, P, g, z0, z1, seed: int, sweep: int,
                 chain_ids: Sequence[int]):
    """One sweep: the messenger draw (Alg. 1, first loop), then Alg. 3 on the
    shells.  g, z0, z1 are the messenger and mode normals of ``sampler.
    sweep_draws`` (the same words the plain sweep uses).  Returns
    (s_new, P_new, s_hat, sigma, accepted)."""
    bins = prob.bins
    tau = prob.tau
    t = sp.messenger_draw(s, prob.d, prob.N, prob.R, tau, g)
    t_hat = sp.ont(t)
    xi = sp.mode_noise(bins, z0, z1)
    S = prob.S_hat(P)
    x = np.sqrt(S) * t_hat / (S + tau) + np.sqrt(tau / (S + tau)) * xi
    B1 = bins.n_bins + 1
    idx = bins.bin_of.reshape(-1)
    w = bins.weight.reshape(-1).astype(np.float64)
    keep = idx >= 0
    C = s.shape[0]
    xr = x.reshape(C, -1)
    tr = t_hat.reshape(C, -1)
    P_new = np.array(P, dtype=np.float64, copy=True)
    acc = np.zeros((C, B1))
    S_new = (prob.M / prob.V) * P_new
    for c in range(C):
        A = np.bincount(idx[keep], weights=(w * np.real(np.conj(xr[c]) * tr[c]))[keep], minlength=B1)
        Bs = np.bincount(idx[keep], weights=(w * np.abs(xr[c]) ** 2)[keep], minlength=B1)
        for b in range(B1):
            if bins.n_b[b] == 0:
                continue
            u0 = np.sqrt(S_new[c, b])
            u1, ok = shell_update(u0, A[b], Bs[b], tau,
                                  attempt_words(seed, sweep, chain_ids[c], b))
            S_new[c, b] = u1 * u1
            acc[c, b] = 1.0 if ok else 0.0
    P_new = (prob.V / prob.M) * S_new
    S_mode = prob.S_hat(P_new)
    s_hat = np.sqrt(S_mode) * x
    s_new = sp.ont_inv(s_hat, prob.shape)
    sig = np.zeros((C, B1))
    a2 = (np.abs(s_hat) ** 2).reshape(C, -1)
    for c in range(C):
        sig[c] = np.bincount(idx[keep], weights=(w * a2[c])[keep], minlength=B1)
    return s_new, P_new, s_hat, sig, acc


class MixingChains(sp.Chains):
    """Chains advanced by mixing sweeps (messenger draw + Alg. 3); same start
    and random streams as ``sampler.Chains``."""

    def sweep(self, n: int = 1):
        for _ in range(n):
            g, z0, z1 = sp.sweep_draws(self.prob.shape, self.seed, self.sweeps_done, self.chain_ids)
            self.s, self.P, _, self.last_sig, self.last_X = mixing_sweep(
                self.prob, self.s, self.P, g, z0, z1, self.seed, self.sweeps_done, self.chain_ids)
            self.sweeps_done += 1
        return self


class AlternatingChains(sp.Chains):
    """Chains whose sweeps alternate: a sweep with an even sweep count is a
    plain sweep (Alg. 1 + Alg. 2), one with an odd count a mixing sweep."""

    def sweep(self, n: int = 1):
        for _ in range(n):
            g, z0, z1 = sp.sweep_draws(self.prob.shape, self.seed, self.sweeps_done, self.chain_ids)
            if self.sweeps_done % 2 == 0:
                X = sp.chi2_shell_draws(self.prob.bins.n_b, self.seed, self.sweeps_done, self.chain_ids)
                self.s, self.P, _, self.last_sig, self.last_X = sp.gibbs_sweep(
                    self.prob, self.s, self.P, g, z0, z1, X)
            else:
                self.s, self.P, _, self.last_sig, self.last_X = mixing_sweep(
                    self.prob, self.s, self.P, g, z0, z1, self.seed, self.sweeps_done, self.chain_ids)
            self.sweeps_done += 1
        return self
