"""Over-dispersed starts (Sec. 3.4: independent chains from over-dispersed
initial conditions): log(P_b / P0_b) / sigma over many chains and shells is
standard normal (KS), chains differ, and sigma = 0 leaves every chain at P0."""
import numpy as np
from scipy import stats

from oracle import sampler as sp


def test_dispersed_starting_powers_are_lognormal():
    shape = (8, 8, 8)
    rng = np.random.default_rng(1)
    prob = sp.make_problem(shape, 8.0, np.full(shape, 0.2), np.ones(shape), rng.normal(size=shape), 6)
    P0 = np.linspace(1.0, 2.0, 7) * prob.V / prob.M
    ch = sp.Chains(prob, seed=5, chain_ids=list(range(500)), P0=P0, start_dispersion=0.7)
    z = np.log(ch.P / P0[None, :]) / 0.7
    assert stats.kstest(z.reshape(-1), "norm").pvalue > 1e-3
    assert np.all(np.std(ch.P, axis=0) > 0)
    plain = sp.Chains(prob, seed=5, chain_ids=[0, 1], P0=P0)
    assert np.array_equal(plain.P, np.tile(P0, (2, 1)))
