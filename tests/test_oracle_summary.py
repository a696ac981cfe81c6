"""Pins of the trace summaries (correlation length and quantiles of P(k)).

* A trace alternating about its mean has C_n = (-1)^n exactly and n_c = 1
  (dividing by R instead of R - n, a plausible slip, breaks this).
* An AR(1) trace with coefficient phi has C_n -> phi^n; for phi = 1/2 the
  correlation length (first C_n < 0.1) is 4.
* A constant trace: C_n = 1 and n_c = -1.
* Quantiles of a shuffled 0 .. R-1 are q (R - 1) exactly, min and max at q = 0
  and 1.
* Gelman-Rubin R-hat: a hand-computed two-chain case; ~1 for chains from one
  distribution, > 1 when their means differ; the constant-chain conventions.
"""
import numpy as np

from oracle import summary


def test_alternating_trace_has_exact_acf():
    R = 1001
    i = np.arange(R)
    tr = np.stack([3.0 + 0.5 * (-1.0) ** i, 7.0 - 2.0 * (-1.0) ** i], axis=1)
    tr[-1] = [3.0, 7.0]  # keep the mean exactly 3 and 7 with an odd length
    C, nc = summary.acf(tr[:-1], 20)
    n = np.arange(21)
    np.testing.assert_allclose(C, np.tile((-1.0) ** n, (2, 1)), atol=1e-12)
    assert list(nc) == [1, 1]


def test_ar1_trace_correlation_length():
    rng = np.random.default_rng(8)
    R, phi = 200000, 0.5
    e = rng.standard_normal(R)
    x = np.empty(R)
    x[0] = e[0]
    for k in range(1, R):
        x[k] = phi * x[k - 1] + np.sqrt(1 - phi * phi) * e[k]
    C, nc = summary.acf(np.stack([x, 10.0 + 2.0 * x], axis=1), 12)
    np.testing.assert_allclose(C, np.tile(phi ** np.arange(13), (2, 1)), atol=0.015)
    assert list(nc) == [4, 4]


def test_constant_trace():
    C, nc = summary.acf(np.full((50, 3), 2.5), 5)
    assert np.all(C == 1.0) and list(nc) == [-1, -1, -1]


def test_quantiles_of_a_permutation():
    R = 1000
    rng = np.random.default_rng(2)
    tr = np.stack([rng.permutation(R), rng.permutation(R)], axis=1).astype(np.float64)
    q = np.array([0.0, 0.025, 0.16, 0.5, 0.84, 0.975, 1.0])
    np.testing.assert_allclose(summary.quantiles(tr, q), np.tile(q * (R - 1), (2, 1)), rtol=0, atol=1e-9)


def test_rhat_hand_computed_case():
    # chains (0, 2) and (2, 4): n = 2, W = 2, B = 4, var+ = 3, R-hat = sqrt(3/2)
    a = np.array([[0.0], [2.0]])
    b = np.array([[2.0], [4.0]])
    np.testing.assert_allclose(summary.rhat([a, b]), [np.sqrt(1.5)], rtol=1e-15)


def test_rhat_limits():
    rng = np.random.default_rng(11)
    same = [rng.standard_normal((20000, 2)) for _ in range(4)]
    r = summary.rhat(same)
    assert np.all(np.abs(r - 1.0) < 0.01)
    shifted = [t + np.array([3.0 * k, 0.0]) for k, t in enumerate(same)]
    r2 = summary.rhat(shifted)
    assert r2[0] > 3.0 and abs(r2[1] - 1.0) < 0.01
    const = [np.full((10, 2), 5.0), np.full((10, 2), 5.0)]
    assert list(summary.rhat(const)) == [1.0, 1.0]
    differ = [np.full((10, 1), 5.0), np.full((10, 1), 6.0)]
    assert np.isinf(summary.rhat(differ)[0])
