"""Pins of the oracle's univariate conditionals and the shell covariance draw.

* tau and N~ on hand-computed cases (Sec. 2).
* The messenger conditional (Sec. 3.1) against the product of the two Gaussian
  factors of the augmented posterior that involve t: N(t; s, T) from the
  (s - t) term and N(d; R t, N~) from the likelihood, combined by precisions —
  a different algebraic route to the same law.
* The mode conditional against the same completing-the-square construction.
* Alg. 2 on shells: X_b ~ chi^2_{n_b} drawn once per shell (KS against the
  chi-square law, moments, independence), the closed-form inverse-gamma
  moments, and the n_b = 1 shell reproducing Alg. 2 literally.
* The modes' Philox words: each stored mode has a call and word pair of its own.
* Noiseless, fully observed data return the binned power of the seeded field.
"""
import itertools

import numpy as np
import pytest
import scipy.stats as st

import mockgen
from oracle import sampler
from oracle.bins import make_bins


def test_tau_and_augmented_noise_hand_cases():
    R = np.array([1.0, 0.5, 0.0, 2.0])
    N = np.array([2.0, 1.0, 5.0, 12.0])
    # N/R^2 on observed voxels: 2, 4, 3 -> tau = 2
    assert sampler.messenger_tau(N, R) == 2.0
    assert sampler.messenger_tau(N, R, 0.5) == 1.0
    np.testing.assert_allclose(sampler.augmented_noise(N, R, 2.0), [0.0, 0.5, 5.0, 4.0])
    with pytest.raises(ValueError):
        sampler.messenger_tau(N, np.zeros(4))


def test_messenger_conditional_by_precisions():
    rng = np.random.default_rng(3)
    n = 1000
    R = rng.uniform(0.1, 2.0, n)
    R[:200] = 0.0
    N = rng.uniform(0.1, 3.0, n)
    s = rng.standard_normal(n)
    d = rng.standard_normal(n)
    tau = 0.7 * sampler.messenger_tau(N, R)
    mu, var = sampler.messenger_moments(s, d, N, R, tau)
    Nt = N - tau * R ** 2
    obs = R > 0
    prec = 1.0 / tau + np.where(obs, R ** 2 / np.where(obs, Nt, 1.0), 0.0)
    mean = (s / tau + np.where(obs, R * d / np.where(obs, Nt, 1.0), 0.0)) / prec
    np.testing.assert_allclose(mu, mean, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(var, 1.0 / prec, rtol=1e-12)
    np.testing.assert_array_equal(mu[~obs], s[~obs])
    np.testing.assert_allclose(var[~obs], tau)


def test_messenger_at_tau_bound_is_deterministic():
    R = np.array([1.0, 0.5])
    N = np.array([0.2, 1.0])
    tau = sampler.messenger_tau(N, R)
    mu, var = sampler.messenger_moments(np.array([3.0, 3.0]), np.array([0.4, 0.1]), N, R, tau)
    assert var[0] == 0.0 and mu[0] == pytest.approx(0.4)


def test_mode_conditional_by_precisions():
    rng = np.random.default_rng(4)
    S = rng.uniform(0.01, 10.0, 500)
    T = 0.3
    th = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    mu, var = sampler.mode_moments(th, S, T)
    prec = 1.0 / S + 1.0 / T
    np.testing.assert_allclose(mu, (th / T) / prec, rtol=1e-13)
    np.testing.assert_allclose(var, 1.0 / prec, rtol=1e-13)


def chi_draws(n_b, sweeps, seed=5, chain=0):
    """X_b for the shells of counts n_b over `sweeps` sweeps, shape (sweeps, B+1)."""
    return np.array([sampler.chi2_shell_draws(n_b, seed, sw, [chain])[0] for sw in range(sweeps)])


NB_LAW = np.array([1, 2, 3, 5, 8, 40, 1000, 200000])


def test_shell_chi_square_law():
    """X_b ~ chi^2_{n_b}: KS per shell against scipy's chi-square law (small
    shape parameters, where a wrong d or c of the gamma method shows, and large
    ones), its mean n_b and variance 2 n_b, and the pooled probability integral
    transform uniform."""
    X = chi_draws(NB_LAW, 1500)
    pooled = []
    for b, nb in enumerate(NB_LAW):
        x = X[:, b]
        assert np.all(np.isfinite(x)) and np.all(x > 0)
        assert st.kstest(x, "chi2", args=(nb,)).pvalue > 1e-4, nb
        assert abs(x.mean() - nb) < 5 * np.sqrt(2 * nb / x.size), nb
        assert abs(x.var() / (2 * nb) - 1) < 0.2, nb
        pooled.append(st.chi2.cdf(x, nb))
    assert st.kstest(np.concatenate(pooled), "uniform").pvalue > 1e-4


def test_shell_chi_square_draws_are_independent():
    """Different shells, chains and sweeps draw from different Philox calls:
    no correlation between shells or between chains."""
    nb = np.full(6, 30)
    X0 = chi_draws(nb, 800, chain=0)
    X1 = chi_draws(nb, 800, chain=1)
    for a, b in ((X0[:, 0], X0[:, 1]), (X0[:, 2], X1[:, 2]), (X0[:-1, 3], X0[1:, 3])):
        assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(a.size)


def test_inverse_gamma_moments():
    """P_b = (V/M) sigma_b / X_b: mean sigma/(n_b - 2), variance
    2 sigma^2 / ((n_b - 2)^2 (n_b - 4)) in S_hat units."""
    nb_all = np.array([20, 64, 300])
    X = chi_draws(nb_all, 3000, seed=9)
    V, M = 1.0, 512
    for b, nb in enumerate(nb_all):
        sig = 3.7 * nb
        P = sampler.covariance_draw(np.full(X.shape, sig), X, nb_all, np.zeros(X.shape), V, M)[:, b]
        S = P * M / V
        mean = sig / (nb - 2)
        var = 2 * sig ** 2 / ((nb - 2) ** 2 * (nb - 4))
        assert abs(S.mean() - mean) < 5 * np.sqrt(var / S.size)
        assert abs(S.var() / var - 1) < 0.25


def test_single_mode_shell_is_alg2():
    """A shell holding one self-conjugate mode (n_b = 1): S = |s_hat|^2 / G^2
    with G the first Box-Muller normal of the shell's Philox call."""
    from oracle import philox as ph
    n, L = 4, 1.0
    kcorner = 2 * np.pi * np.sqrt(12.0)
    edges = np.array([0.0, kcorner - 0.5, kcorner + 0.5])
    tab = make_bins((n, n, n), (L, L, L), 2, edges)
    assert tab.n_b[1] == 1 and tab.bin_of[2, 2, 2] == 1
    rng = np.random.default_rng(1)
    s_hat = (rng.standard_normal((1, n, n, 3)) + 0j)
    sig = sampler.shell_sums(tab, s_hat)
    X = sampler.chi2_shell_draws(tab.n_b, 3, 0, [0])
    P = sampler.covariance_draw(sig, X, tab.n_b, np.zeros((1, 3)), L ** 3, n ** 3)
    w = ph.philox4x32_10(1, 0, 0, ph.STREAM_CHI2, 3)
    u = float(ph.box_muller(w[0], w[1])[0]) ** 2
    assert P[0, 1] * n ** 3 / L ** 3 == pytest.approx(abs(s_hat[0, 2, 2, 2]) ** 2 / u, rel=1e-14)


def test_mode_normals_use_each_philox_word_pair_once():
    """The stored modes kx and n - kx share one Philox call (that of the stored
    index of min(kx, n - kx)), the first taking words (w0, w1), the second
    (w2, w3): every stored mode of a sweep has a call and half of its own, and
    its normals are those of that call."""
    from oracle import philox as ph
    for shape in ((8, 8, 8), (6, 4, 8), (5, 4, 6)):
        nx, ny, nz = shape
        nh = nz // 2 + 1
        _, z0, z1 = sampler.sweep_draws(shape, 11, 2, [3])
        used = set()
        for kx in range(nx):
            kxp = min(kx, nx - kx)
            half = 0 if kx <= nx // 2 else 1
            for ky in range(ny):
                for kz in range(nh):
                    call = (kxp * ny + ky) * nh + kz
                    assert (call, half) not in used
                    used.add((call, half))
                    zz = ph.normals4(call, 2, 3, ph.STREAM_MODES, 11)
                    assert z0[0, kx, ky, kz] == zz[2 * half] and z1[0, kx, ky, kz] == zz[2 * half + 1]


def test_edge_plane_noise_is_conjugate_symmetric_with_lower_rows_canonical():
    """The kz = 0 and nz/2 planes store both k and -k.  There xi(-k) must be the
    conjugate of xi(k) and a self-conjugate mode real (xi = z0), so that s_hat
    stays the transform of a real field; the canonical member of each pair is
    the one with the smaller ky*nx + kx and takes its own (z0 + i z1)/sqrt(2).
    Hence every canonical mode lies in a row ky <= ny - ky: the noise of rows ky
    and ny - ky comes from the calls of the lower of the two alone.  Checked
    mode by mode, on even and odd shapes; a rule keyed on the stored index (kx
    first) fails the row property."""
    for shape in ((8, 8, 8), (6, 4, 8), (5, 4, 6), (4, 5, 4)):
        nx, ny, nz = shape
        nh = nz // 2 + 1
        tab = make_bins(shape, (1.0, 1.0, 1.0), 1, k_edges=np.array([0.0, 1e3]))
        _, z0, z1 = sampler.sweep_draws(shape, 11, 2, [3])
        xi = sampler.mode_noise(tab, z0, z1)[0]
        n_edge = 0
        for kx in range(nx):
            for ky in range(ny):
                for kz in range(nh):
                    own = (z0[0, kx, ky, kz] + 1j * z1[0, kx, ky, kz]) / np.sqrt(2.0)
                    if not tab.edge_plane[kx, ky, kz]:
                        assert xi[kx, ky, kz] == own
                        continue
                    n_edge += 1
                    px, py = (-kx) % nx, (-ky) % ny
                    if (px, py) == (kx, ky):
                        assert xi[kx, ky, kz] == z0[0, kx, ky, kz]
                        continue
                    assert xi[px, py, kz] == np.conj(xi[kx, ky, kz])
                    if ky * nx + kx < py * nx + px:
                        assert xi[kx, ky, kz] == own
                        assert ky <= py
        assert n_edge == 2 * nx * ny


def test_empty_shell_is_held():
    tab = make_bins((8, 8, 8), (1.0, 1.0, 1.0), 8)
    # B = 8 linear shells on an 8^3 grid are k_Nyq/8 = k_f/2 wide: |m| = 1 is
    # the first non-DC shell (b = 2), so shells 0 and 1 are empty
    np.testing.assert_array_equal(tab.n_b[:2], 0)
    assert np.all(tab.n_b[2:] > 0)
    P = sampler.covariance_draw(np.ones((1, 9)), np.ones((1, 9)), tab.n_b,
                                np.full((1, 9), 42.0), 1.0, 512)
    assert np.all(P[0, :2] == 42.0) and np.all(P[0, 2:] == 1.0 / 512)


def test_noiseless_fully_observed_recovers_field_power():
    n = 16
    m = mockgen.make_mock(n, seed=8, n_bins=8)
    eps = 1e-10
    R = np.ones(m.shape)
    N = np.full(m.shape, eps)
    d = m.s_true.copy()
    prob = sampler.make_problem(m.shape, m.L, N, R, d, 8)
    ch = sampler.Chains(prob, seed=2, chain_ids=[0])
    ch.sweep(1)
    # binned power of the seeded field from its full complex FFT, brute force
    F = np.fft.fftn(m.s_true) / np.sqrt(n ** 3)
    f = np.fft.fftfreq(n, 1.0 / n)
    want = np.zeros(9)
    for kx, ky, kz in itertools.product(range(n), repeat=3):
        m2 = f[kx] ** 2 + f[ky] ** 2 + f[kz] ** 2
        if m2 == 0:
            continue
        b = min(int(np.floor(8 * np.sqrt(m2) / (n // 2) + 1e-12)), 8)
        want[b] += abs(F[kx, ky, kz]) ** 2
    np.testing.assert_allclose(ch.last_sig[0], want, rtol=1e-4)
    np.testing.assert_allclose(ch.s[0], m.s_true, atol=1e-4)
