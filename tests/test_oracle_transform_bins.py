"""Pins of the oracle's orthonormal transform and k-shell table.

* ONT against the DFT written out as a sum (tiny, non-cubic grids), its
  unitarity (Parseval) and the round trip.
* Shell ids against a brute-force pass over the FULL grid computing |m| with
  50-digit decimal arithmetic (ties included), the dof weights against full-grid
  mode counts, the conjugate partners against the definition, and the counting
  invariant sum n_b + 1 = M.
"""
import decimal
import itertools

import numpy as np
import pytest

from oracle import sampler
from oracle.bins import make_bins


def naive_rdft(x):
    nx, ny, nz = x.shape
    out = np.zeros((nx, ny, nz // 2 + 1), dtype=complex)
    for kx, ky, kz in itertools.product(range(nx), range(ny), range(nz // 2 + 1)):
        acc = 0j
        for ix, iy, iz in itertools.product(range(nx), range(ny), range(nz)):
            ph = -2j * np.pi * (kx * ix / nx + ky * iy / ny + kz * iz / nz)
            acc += x[ix, iy, iz] * np.exp(ph)
        out[kx, ky, kz] = acc
    return out / np.sqrt(nx * ny * nz)


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 6), (2, 6, 4)])
def test_ont_equals_naive_dft(shape):
    x = np.random.default_rng(1).standard_normal(shape)
    got = sampler.ont(x[None])[0]
    np.testing.assert_allclose(got, naive_rdft(x), rtol=0, atol=1e-12)


def test_ont_unitary_and_round_trip():
    shape = (8, 6, 10)
    x = np.random.default_rng(2).standard_normal((3,) + shape)
    xh = sampler.ont(x)
    w = np.ones(xh.shape[-1]) * 2.0
    w[0] = 1.0
    w[-1] = 1.0
    energy_k = (w * np.abs(xh) ** 2).sum(axis=(-3, -2, -1))
    np.testing.assert_allclose(energy_k, (x ** 2).sum(axis=(-3, -2, -1)), rtol=1e-13)
    np.testing.assert_allclose(sampler.ont_inv(xh, shape), x, atol=1e-13)


def brute_bins(n, B):
    """Shell of every full-grid mode, |m| evaluated with 50-digit decimals."""
    decimal.getcontext().prec = 50
    h = n // 2
    f = [k if k <= h else k - n for k in range(n)]
    out = {}
    for kx, ky, kz in itertools.product(range(n), range(n), range(n)):
        m2 = f[kx] ** 2 + f[ky] ** 2 + f[kz] ** 2
        if m2 == 0:
            continue
        x = decimal.Decimal(B) * decimal.Decimal(m2).sqrt() / decimal.Decimal(h)
        b = int(x.to_integral_value(rounding=decimal.ROUND_FLOOR))
        # exact ties: x is an integer exactly when B^2 m^2 / h^2 is a square
        if (b + 1) ** 2 * h * h <= B * B * m2:
            b += 1
        out[(kx, ky, kz)] = min(b, B)
    return out


@pytest.mark.parametrize("n,B", [(8, 4), (8, 3), (12, 6), (16, 8), (6, 5)])
def test_linear_bins_against_brute_force(n, B):
    tab = make_bins((n, n, n), (1.0, 1.0, 1.0), B)
    full = brute_bins(n, B)
    nh = n // 2 + 1
    counts = np.zeros(B + 1, dtype=np.int64)
    for (kx, ky, kz), b in full.items():
        counts[b] += 1
        if kz < nh:
            assert tab.bin_of[kx, ky, kz] == b, (kx, ky, kz)
    assert tab.bin_of[0, 0, 0] == -1
    np.testing.assert_array_equal(tab.n_b, counts)
    assert tab.n_b.sum() + 1 == n ** 3


def test_explicit_edges_and_overflow():
    n, L = 8, 100.0
    kf = 2 * np.pi / L
    edges = np.array([0.5, 1.5, 2.5]) * kf
    tab = make_bins((n, n, n), (L, L, L), 2, edges)
    m = np.fft.fftfreq(n, 1.0 / n)
    mz = np.arange(n // 2 + 1)
    kk = kf * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    want = np.where(kk < 1.5 * kf, 0, np.where(kk < 2.5 * kf, 1, 2))
    want[0, 0, 0] = -1
    np.testing.assert_array_equal(tab.bin_of, want)
    assert tab.n_b.sum() + 1 == n ** 3


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 4, 8), (5, 3, 4)])
def test_weights_and_partners(shape):
    nx, ny, nz = shape
    L = (1.0, 1.0, 1.0)
    edges = np.linspace(0, 40, 5)
    tab = make_bins(shape, L, 4, edges)
    nh = nz // 2 + 1
    for kx, ky, kz in itertools.product(range(nx), range(ny), range(nh)):
        edge = kz == 0 or kz == nz // 2
        assert tab.weight[kx, ky, kz] == (1 if edge else 2)
        if edge:
            px, py = (-kx) % nx, (-ky) % ny
            assert tab.partner[kx, ky, kz] == (px * ny + py) * nh + kz
    # every full-grid mode is represented exactly once by (stored mode, weight)
    assert tab.weight.sum() == nx * ny * nz
