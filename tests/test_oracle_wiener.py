"""The oracle's sweep against the Wiener posterior it must sample (Sec. 2-3.1).

The paper's central claim: with T = tau 1 and N~ = N - R^T T R, alternating the
two univariate draws of Alg. 1 and discarding t samples the Wiener posterior
Pi(s | S, d) (Sec. 2, marginalisation; Sec. 3.1, the iteration).  With P held
fixed one sweep is an affine map with Gaussian noise,
    s' = G s + h + A zeta,   zeta ~ N(0, 1),
so the chain's stationary law is N(m, Sigma) with m = (I - G)^-1 h and
Sigma = G Sigma G^T + A A^T.  Those are compared, deterministically, with the
Wiener mean and covariance found by dense matrix inversion:
    m_WF = S R^T (R S R^T + N)^-1 d,   C_WF = S - S R^T (R S R^T + N)^-1 R S
(written in this form because S is singular: the DC mode has zero power),
restricted to observed voxels.  S is built from the unitary DFT matrix written
out elementwise, not from the oracle's transform.

A statistical version draws many independent chains with the real Philox
normals and checks the whitened samples.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sampler


def dft_matrix(shape):
    """Unitary DFT matrix F[k, i] = exp(-2 pi i k.x / n) / sqrt(M), full grid."""
    nx, ny, nz = shape
    M = nx * ny * nz
    idx = np.array(list(itertools.product(range(nx), range(ny), range(nz))))
    ph = (np.outer(idx[:, 0], idx[:, 0]) / nx + np.outer(idx[:, 1], idx[:, 1]) / ny
          + np.outer(idx[:, 2], idx[:, 2]) / nz)
    return np.exp(-2j * np.pi * ph) / np.sqrt(M)


def full_grid_S_hat(prob, P):
    """S_hat on every full-grid mode, from the stored-mode table via k <-> -k."""
    nx, ny, nz = prob.shape
    Sst = prob.S_hat(P)[0]
    S = np.zeros(prob.shape)
    for kx, ky, kz in itertools.product(range(nx), range(ny), range(nz)):
        if kz <= nz // 2:
            S[kx, ky, kz] = Sst[kx, ky, kz]
        else:
            S[kx, ky, kz] = Sst[(-kx) % nx, (-ky) % ny, nz - kz]
    return S.reshape(-1)


def wiener_solution(prob, P):
    F = dft_matrix(prob.shape)
    S = (F.conj().T @ np.diag(full_grid_S_hat(prob, P)) @ F).real
    obs = prob.R.reshape(-1) > 0
    Ro = np.diag(prob.R.reshape(-1))[obs]
    No = np.diag(prob.N.reshape(-1)[obs])
    K = S @ Ro.T @ np.linalg.inv(Ro @ S @ Ro.T + No)
    m = K @ prob.d.reshape(-1)[obs]
    C = S - K @ Ro @ S
    return m, C


def affine_sweep_map(prob, P):
    """G, h and the noise map A of one fixed-P sweep, by probing the oracle."""
    shape = prob.shape
    M = prob.M
    nh = shape[2] // 2 + 1
    Mh = shape[0] * shape[1] * nh
    zv = np.zeros((1,) + shape)
    zm = np.zeros((1, shape[0], shape[1], nh))

    def run(s, g, z0, z1):
        out = sampler.gibbs_sweep(prob, s, P, g, z0, z1, None, fix_P=True)[0]
        return out.reshape(-1)

    h = run(zv, zv, zm, zm)
    G = np.empty((M, M))
    for i in range(M):
        e = np.zeros(M)
        e[i] = 1
        G[:, i] = run(e.reshape((1,) + shape), zv, zm, zm) - h
    cols = []
    for i in range(M):
        e = np.zeros(M)
        e[i] = 1
        cols.append(run(zv, e.reshape((1,) + shape), zm, zm) - h)
    for q in range(2):
        for j in range(Mh):
            e = np.zeros(Mh)
            e[j] = 1
            e = e.reshape((1, shape[0], shape[1], nh))
            args = (e, zm) if q == 0 else (zm, e)
            cols.append(run(zv, zv, *args) - h)
    A = np.stack(cols, axis=1)
    return G, h, A


def small_problem(shape, seed, tau_scale=1.0, mask_frac=0.3, R_lo=0.3, N_range=(0.05, 0.5),
                  P_scale=3.0):
    rng = np.random.default_rng(seed)
    R = rng.uniform(R_lo, 1.5 if R_lo < 0.5 else 1.3, size=shape)
    R[rng.uniform(size=shape) < mask_frac] = 0.0
    R.flat[0] = 0.8
    N = rng.uniform(N_range[0], N_range[1], size=shape)
    d = np.where(R > 0, rng.standard_normal(shape), 0.0)
    L = (1.0, 1.0, 1.0)
    edges = np.array([0.0, 8.0, 14.0, 30.0])
    prob = sampler.make_problem(shape, L, N, R, d, 3, k_edges=edges, tau_scale=tau_scale)
    P = np.array([[0.9, 0.4, 0.2, 0.1]]) * (prob.V / prob.M) * P_scale
    return prob, P


@pytest.mark.parametrize("shape,tau_scale", [((4, 4, 4), 1.0), ((4, 4, 4), 0.6),
                                             ((4, 2, 6), 1.0), ((2, 4, 4), 0.9)])
def test_stationary_law_is_wiener_posterior(shape, tau_scale):
    prob, P = small_problem(shape, seed=11 + shape[2], tau_scale=tau_scale)
    G, h, A = affine_sweep_map(prob, P)
    rho = max(abs(np.linalg.eigvals(G)))
    assert rho < 1.0
    m = np.linalg.solve(np.eye(prob.M) - G, h)
    Sigma = sla.solve_discrete_lyapunov(G, A @ A.T)
    m_wf, C_wf = wiener_solution(prob, P)
    scale = np.sqrt(np.max(np.diag(C_wf)))
    np.testing.assert_allclose(m, m_wf, atol=1e-10 * max(1.0, np.abs(m_wf).max()))
    np.testing.assert_allclose(Sigma, C_wf, atol=1e-10 * scale ** 2)


def test_planted_mistakes_break_the_pin(monkeypatch):
    """The pin above is sensitive: a wrong mode variance, a dropped noise term
    or a wrong messenger mean each move the stationary law off the Wiener one."""
    prob, P = small_problem((4, 4, 4), seed=3)
    m_wf, C_wf = wiener_solution(prob, P)
    orig_mode, orig_msg = sampler.mode_moments, sampler.messenger_moments

    def bad_mode(t_hat, S_hat, T_hat):
        mu, var = orig_mode(t_hat, S_hat, T_hat)
        return mu, var * 1.1

    def bad_msg(s, d, N, R, tau):
        mu, var = orig_msg(s, d, N, R, tau)
        return mu + 0.01 * (R > 0) * d, var

    for name, fn in (("mode_moments", bad_mode), ("messenger_moments", bad_msg)):
        monkeypatch.setattr(sampler, name, fn)
        G, h, A = affine_sweep_map(prob, P)
        m = np.linalg.solve(np.eye(prob.M) - G, h)
        Sigma = sla.solve_discrete_lyapunov(G, A @ A.T)
        bad = (np.abs(m - m_wf).max() > 1e-6) or (np.abs(Sigma - C_wf).max() > 1e-6)
        assert bad, name
        monkeypatch.setattr(sampler, name, {"mode_moments": orig_mode,
                                            "messenger_moments": orig_msg}[name])


def test_R1_constant_noise_is_one_step_wiener():
    """R = 1 and N = nu constant: tau = nu, N~ = 0, t = d exactly, and one sweep
    is an exact independent draw from the Wiener posterior; its noise-free part
    is S (S + nu)^-1 d."""
    shape = (4, 4, 4)
    rng = np.random.default_rng(5)
    nu = 0.3
    R = np.ones(shape)
    N = np.full(shape, nu)
    d = rng.standard_normal(shape)
    edges = np.array([0.0, 8.0, 14.0, 30.0])
    prob = sampler.make_problem(shape, (1.0, 1.0, 1.0), N, R, d, 3, k_edges=edges)
    assert prob.tau == nu
    mu, var = sampler.messenger_moments(np.zeros(shape), d, N, R, prob.tau)
    np.testing.assert_array_equal(var, 0.0)
    np.testing.assert_allclose(mu, d, rtol=1e-15)
    P = np.array([[0.7, 0.5, 0.1, 0.05]]) * (prob.V / prob.M) * 2
    G, h, A = affine_sweep_map(prob, P)
    np.testing.assert_allclose(G, 0.0, atol=1e-14)
    m_wf, C_wf = wiener_solution(prob, P)
    np.testing.assert_allclose(h, m_wf, atol=1e-12)
    np.testing.assert_allclose(A @ A.T, C_wf, atol=1e-12)


def test_statistical_wiener_with_philox_draws():
    """Independent chains with the real draws: whitened final samples ~ N(0, I)."""
    # a well-mixing case (spectral radius of G about 0.33) keeps the burn-in short
    prob, P = small_problem((4, 4, 4), seed=21, mask_frac=0.2, R_lo=0.7,
                            N_range=(1.0, 1.2), P_scale=0.5)
    G, h, A = affine_sweep_map(prob, P)
    rho = max(abs(np.linalg.eigvals(G)))
    assert rho < 0.5
    sweeps = int(np.ceil(np.log(1e-6) / np.log(rho))) + 2
    C = 3000
    ch = sampler.Chains(prob, seed=77, chain_ids=range(C), P0=P[0], fix_P=True)
    ch.sweep(sweeps)
    x = ch.s.reshape(C, -1)
    m_wf, C_wf = wiener_solution(prob, P)
    # C_wf is singular along the DC direction (the mean of s is pinned at 0)
    w, U = np.linalg.eigh(C_wf)
    keep = w > 1e-12 * w.max()
    Wh = U[:, keep] / np.sqrt(w[keep])
    y = (x - m_wf) @ Wh
    k = y.shape[1]
    assert np.abs(x.mean(axis=1)).max() < 1e-12
    assert np.abs(y.mean(axis=0)).max() < 4.5 / np.sqrt(C)
    cov = (y.T @ y) / C
    off = cov - np.eye(k)
    assert np.abs(off).max() < 5.5 * np.sqrt(2.0 / C)
