"""Seeded synthetic inputs: Gaussian mock surveys for the messenger sampler.

This module generates INPUTS only (the signal field, the response R, the noise
N and the data d).  It holds none of the sampler's arithmetic and is the one
module shared by the CUDA library's users (``bench.py``, the tests) and the
oracle's tests.  Its random numbers come from numpy's own Philox bit generator,
keyed by (seed, purpose), so they are reproducible on any host.

The paper's own mock (Sec. 4: an SDSS-DR7 completeness map and a Schechter
radial selection) needs survey data that is not available here; these Gaussian
mocks stand in for it with the same structure: a smooth radial selection inside
a survey sphere, a masked exterior, optional holes, and a noise level that grows
where the selection falls off.

Recipe (all lengths in the box's units):
  * P(k) = A k / (1 + (k/0.02)^2)^2, A chosen so that the discrete voxel
    variance (1/V) sum_{k != 0} P(|k|) over the grid's modes equals 1.
  * s_true: unit white noise w, s_true = irfftn(sqrt(S_hat) rfftn(w)/sqrt(M))
    * sqrt(M) with S_hat = (M/V) P(|k|), S_hat(0) = 0.
  * R = exp(-(r/300)^2) for r < 450 about the box centre, 0 outside; voxel
    centres at (i + 1/2) L/n.  Optional spherical holes (R = 0 inside) with
    centres uniform in the survey sphere.
  * N = sigma_n / R where R > 0 (and 1 where R = 0; it is ignored there).
  * d = R s_true + sqrt(N) eps where R > 0, 0 elsewhere.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

PURPOSE_FIELD = 1
PURPOSE_NOISE = 2
PURPOSE_HOLES = 3
PURPOSE_WEIGHTS = 4


def rng_for(seed: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(purpose)]))


def power_spectrum_shape(k):
    """P(k)/A = k / (1 + (k/0.02)^2)^2."""
    k = np.asarray(k, dtype=np.float64)
    return k / (1.0 + (k / 0.02) ** 2) ** 2


def full_grid_k(n: int, L: float):
    f = np.fft.fftfreq(n, d=1.0 / n)  # integer wavenumbers
    kf = 2.0 * np.pi / L
    kx = kf * f[:, None, None]
    ky = kf * f[None, :, None]
    kz = kf * f[None, None, :]
    return np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)


def amplitude_for_unit_variance(n: int, L: float) -> float:
    k = full_grid_k(n, L)
    s = power_spectrum_shape(k).sum()  # k = 0 contributes 0
    V = L ** 3
    return V / s


def stored_k(n: int, L: float):
    f = np.fft.fftfreq(n, d=1.0 / n)
    fz = np.arange(n // 2 + 1)
    kf = 2.0 * np.pi / L
    return kf * np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2)


def gaussian_field(n: int, L: float, seed: int) -> np.ndarray:
    M = n ** 3
    V = L ** 3
    A = amplitude_for_unit_variance(n, L)
    S_hat = (M / V) * A * power_spectrum_shape(stored_k(n, L))
    S_hat[0, 0, 0] = 0.0
    w = rng_for(seed, PURPOSE_FIELD).standard_normal((n, n, n))
    wh = np.fft.rfftn(w) / np.sqrt(M)
    return np.fft.irfftn(np.sqrt(S_hat) * wh, s=(n, n, n), axes=(0, 1, 2)) * np.sqrt(M)


def voxel_radius(n: int, L: float) -> np.ndarray:
    c = (np.arange(n) + 0.5) * (L / n) - L / 2.0
    return np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)


def radial_selection(n: int, L: float, r0: float = 300.0, rmax: float = 450.0):
    r = voxel_radius(n, L)
    return np.where(r < rmax, np.exp(-(r / r0) ** 2), 0.0)


def punch_holes(R: np.ndarray, L: float, seed: int, n_holes: int, radius: float,
                rmax: float = 450.0) -> np.ndarray:
    n = R.shape[0]
    rng = rng_for(seed, PURPOSE_HOLES)
    centres = []
    while len(centres) < n_holes:
        p = rng.uniform(-rmax, rmax, size=3)
        if np.dot(p, p) < rmax ** 2:
            centres.append(p)
    c = (np.arange(n) + 0.5) * (L / n) - L / 2.0
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    R = R.copy()
    for p in centres:
        inside = (X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2 < radius ** 2
        R[inside] = 0.0
    return R


@dataclasses.dataclass
class Mock:
    n: int
    L: float
    N: np.ndarray
    R: np.ndarray
    d: np.ndarray
    s_true: np.ndarray
    n_bins: int
    seed: int
    sigma_n: float
    removed_fraction: float = 0.0

    @property
    def shape(self):
        return (self.n, self.n, self.n)


def make_mock(n: int, L: float = 1000.0, sigma_n: float = 0.1, seed: int = 1,
              n_bins: int = 16, n_holes: int = 0, hole_radius: float = 93.0) -> Mock:
    s_true = gaussian_field(n, L, seed)
    R = radial_selection(n, L)
    removed = 0.0
    if n_holes:
        in_survey = R > 0
        R = punch_holes(R, L, seed, n_holes, hole_radius)
        removed = 1.0 - float((R > 0).sum()) / float(in_survey.sum())
    obs = R > 0
    N = np.where(obs, sigma_n / np.where(obs, R, 1.0), 1.0)
    eps = rng_for(seed, PURPOSE_NOISE).standard_normal((n, n, n))
    d = np.where(obs, R * s_true + np.sqrt(N) * eps, 0.0)
    return Mock(n, L, N, R, d, s_true, n_bins, seed, sigma_n, removed)


def mode_weights(n: int, seed: int) -> np.ndarray:
    """Seeded U(0,1) weights w_k over the stored modes (nx, ny, nz/2+1), used by
    the loss sum_k w_k |s_hat_k|^2 of the differentiation workload."""
    return rng_for(seed, PURPOSE_WEIGHTS).uniform(0.0, 1.0, size=(n, n, n // 2 + 1))


# ---------------------------------------------------------------------------
# The five workloads.  Sizes, bins, chain counts and sweeps as stated for the
# benchmark configurations; each returns what the sampler's init needs.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    mocks: List[Mock]
    chains_per_mock: int
    sweeps: int
    precision: int
    seeds: List[int]


def workload(idx: int, n_override: Optional[int] = None) -> Workload:
    """idx 1..5:
      1: 32^3, FP64, 1 chain, 16 linear bins, 200 sweeps, seed 1
      2: 128^3 + 40 holes (r = 93), FP64, 1 chain, 32 bins, 1000 sweeps
      3: 256^3, FP32, 16 chains on the same data, 64 bins, 2000 sweeps
      4: 16 x 64^3 + 16 x 96^3 + 16 x 128^3, each its own data (sigma_n 0.1 for
         the first 8 of each size, 0.5 for the next 8), 16/24/32 bins, FP32
      5: 128^3, FP32, 32 bins, K = 8 sweeps for the adjoint
    ``n_override`` shrinks the grid (tests), keeping everything else.
    """
    if idx == 1:
        n = n_override or 32
        return Workload("gaussian-mock-32^3-fp64-1chain-16bins",
                        [make_mock(n, seed=1, n_bins=16)], 1, 200, 64, [1])
    if idx == 2:
        n = n_override or 128
        return Workload("gaussian-mock-128^3-40holes-fp64-1chain-32bins",
                        [make_mock(n, seed=2, n_bins=32, n_holes=40)], 1, 1000, 64, [2])
    if idx == 3:
        n = n_override or 256
        return Workload("gaussian-mock-256^3-fp32-16chains-64bins",
                        [make_mock(n, seed=3, n_bins=64)], 16, 2000, 32, [3])
    if idx == 4:
        mocks, seeds = [], []
        for size, nb in ((64, 16), (96, 24), (128, 32)):
            sz = min(size, n_override) if n_override else size
            for c in range(16):
                sd = 4000 + size * 100 + c
                mocks.append(make_mock(sz, seed=sd, n_bins=nb,
                                       sigma_n=0.1 if c < 8 else 0.5))
                seeds.append(sd)
        return Workload("gaussian-mock-48chains-16x64^3+16x96^3+16x128^3-fp32",
                        mocks, 1, 500, 32, seeds)
    if idx == 5:
        n = n_override or 128
        return Workload("gaussian-mock-128^3-fp32-adjoint-K8-32bins",
                        [make_mock(n, seed=5, n_bins=32)], 1, 8, 32, [5])
    raise ValueError(idx)
