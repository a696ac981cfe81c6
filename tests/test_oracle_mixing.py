"""Pins of the mixing sampler oracle (Sec. 3.3, Alg. 3 on k-shells).

* The truncated-normal proposal (plain rejection for a <= 1/2, Robert's
  exponential rejection above) against scipy's truncnorm, in both branches.
* The x draw: sqrt(S) x equals the plain sampler's signal draw s_hat on the
  same noise (so x is the exact conditional of Sec. 3.1 rescaled).
* The Metropolis-Hastings update of u = sqrt(S_b) leaves the conditional
  u^-1 exp(-B (u - A/B)^2 / (2 tau)) invariant: many independent chains of the
  update alone against the CDF of that density by quadrature.  A planted
  mistake (the printed acceptance (u'/u)^2, or accepting every proposal)
  fails the same check.
* Whole sweeps: on a tiny fully observed grid with constant noise N the
  marginal posterior of each shell's S_b is known in closed form up to
  normalisation, S^-1 (S + N)^(-n_b/2) exp(-D_b / (2 (S + N))) with D_b the
  dof-weighted data power of the shell; the final P of many independent mixing
  chains (and, as a cross-check, of plain chains) matches it.

The conditional of u is improper at u -> 0 (its density is finite times u^-1
there, as is the Jeffreys posterior of S_b at S_b -> 0); every case here is in
the regime where that tail carries a negligible weight (A^2 / (2 B tau) >= 50,
high signal to noise), where it is the distribution the samplers must reach.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import mixing as mx
from oracle import philox as ph
from oracle import sampler as sp


@pytest.mark.parametrize("a", [-1.5, 0.0, 0.45, 0.55, 1.5, 4.0])
def test_truncated_normal_matches_scipy(a):
    z = np.array([mx.truncated_normal_positive(-a, 1.0, mx.attempt_words(21, d, 2, 7)) for d in range(3000)])
    z = z + a  # u' = mu + sigma z with mu = -a, sigma = 1
    assert np.all(z > a)
    assert stats.kstest(z, stats.truncnorm(a, np.inf).cdf).pvalue > 1e-3


def test_x_draw_is_the_plain_draw_over_sqrt_S():
    rng = np.random.default_rng(3)
    shape = (6, 6, 6)
    prob = sp.make_problem(shape, 6.0, np.full(shape, 0.3), np.ones(shape),
                           rng.normal(size=shape), 3)
    P = np.array([[0.7, 1.3, 0.4, 2.0]]) * prob.V / prob.M
    g, z0, z1 = sp.sweep_draws(shape, 5, 0, [0])
    t_hat = sp.ont(sp.messenger_draw(np.zeros((1,) + shape), prob.d, prob.N, prob.R, prob.tau, g))
    xi = sp.mode_noise(prob.bins, z0, z1)
    S = prob.S_hat(P)
    s_hat = sp.signal_draw(t_hat, S, prob.tau, xi)
    x = np.sqrt(S) * t_hat / (S + prob.tau) + np.sqrt(prob.tau / (S + prob.tau)) * xi
    keep = prob.bins.bin_of >= 0
    np.testing.assert_allclose((np.sqrt(S) * x)[:, keep], s_hat[:, keep], rtol=1e-13, atol=1e-13)


def u_conditional_cdf(A, B, tau):
    mu, sig = A / B, np.sqrt(tau / B)
    u = np.linspace(max(mu - 20 * sig, 1e-12), mu + 20 * sig, 400001)
    lp = -np.log(u) - B * (u - mu) ** 2 / (2 * tau)
    f = np.exp(lp - lp.max())
    c = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(u))])
    c /= c[-1]
    return lambda v: np.interp(v, u, c)


def run_updates(update, A, B, tau, chains=1200, steps=12):
    """Independent chains of one update rule started at A/B; final states."""
    u = np.full(chains, A / B)
    for k in range(steps):
        for c in range(chains):
            u[c] = update(u[c], A, B, tau, mx.attempt_words(17, k, c, 3))
    return u


def wrong_acceptance_squared(u, A, B, tau, words):
    up = mx.truncated_normal_positive(A / B, np.sqrt(tau / B), words)
    alpha = float(ph.uniform_open0(words[0][3]))
    return up if alpha < (up / u) ** 2 else u


def always_accept(u, A, B, tau, words):
    return mx.truncated_normal_positive(A / B, np.sqrt(tau / B), words)


CASES = [(30.0, 25.0, 0.3), (3.0, 40.0, 0.002), (74.0, 37.0, 0.5)]


@pytest.mark.parametrize("A,B,tau", CASES)
def test_mh_update_leaves_the_u_conditional_invariant(A, B, tau):
    assert A * A / (2 * B * tau) >= 50
    u = run_updates(lambda u, A, B, tau, w: mx.shell_update(u, A, B, tau, w)[0], A, B, tau)
    assert stats.kstest(u, u_conditional_cdf(A, B, tau)).pvalue > 1e-3


@pytest.mark.parametrize("wrong", [wrong_acceptance_squared, always_accept])
def test_planted_acceptance_mistakes_are_detected(wrong):
    A, B, tau = 3.0, 40.0, 0.002
    u = run_updates(wrong, A, B, tau, chains=6000, steps=6)
    assert stats.kstest(u, u_conditional_cdf(A, B, tau)).pvalue < 1e-6


def tiny_problem():
    n = 4
    shape = (n, n, n)
    rng = np.random.default_rng(5)
    Nn = 0.1
    d = rng.normal(size=shape) * np.sqrt(1.0 + Nn)
    prob = sp.make_problem(shape, 4.0, np.full(shape, Nn), np.ones(shape), d, 2, tau_scale=0.5)
    b = prob.bins
    dh = sp.ont(d[None])[0]
    keep = b.bin_of >= 0
    D = np.bincount(b.bin_of[keep], weights=(b.weight * np.abs(dh) ** 2)[keep], minlength=b.n_bins + 1)
    return prob, Nn, D


def shell_posterior_cdf(n_b, D, Nn):
    ls = np.linspace(-30.0, 8.0, 40001)
    S = np.exp(ls)
    lp = -0.5 * n_b * np.log(S + Nn) - D / (2 * (S + Nn))  # S^-1 dS = d log S
    f = np.exp(lp - lp.max())
    c = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(ls))])
    c /= c[-1]
    return lambda v: np.interp(np.log(v), ls, c)


@pytest.mark.parametrize("kind,sweeps", [("mixing", 70), ("plain", 40)])
def test_sweeps_sample_the_closed_form_shell_posterior(kind, sweeps):
    prob, Nn, D = tiny_problem()
    cls = mx.MixingChains if kind == "mixing" else sp.Chains
    ch = cls(prob, seed=11, chain_ids=list(range(1200)))
    ch.sweep(sweeps)
    S = (prob.M / prob.V) * ch.P
    for b in range(prob.bins.n_bins + 1):
        if prob.bins.n_b[b] == 0:
            continue
        p = stats.kstest(S[:, b], shell_posterior_cdf(prob.bins.n_b[b], D[b], Nn)).pvalue
        assert p > 1e-3, (kind, b, p)
