"""k-shell bookkeeping for the isotropic covariance (Sec. 3.2, last paragraph).

ORACLE — test infrastructure only (see ``oracle/sampler.py``).

The paper averages the diagonal signal covariance over spherical shells in
Fourier space and defers the details to earlier work.  The reading used here:

* Shell b holds the modes with e_b <= |k| < e_{b+1}.  The default edges are
  linear, e_b = b * k_Nyq / B with k_Nyq = pi n / L (cubic grids only); with
  k = (2 pi / L) m this is the integer test  b^2 (n/2)^2 <= B^2 |m|^2, so ties go
  to the upper shell.  Explicit edges compare |k| in FP64.
* Modes outside [e_0, e_B) (for linear edges: |k| >= k_Nyq, the cube corners)
  go to an extra overflow shell B, sampled like the others.
* The DC mode belongs to no shell (its covariance is fixed at 0).
* A stored mode of the half-complex array stands for w = 2 full-grid modes
  (k and -k) when 0 < kz < nz/2 and for w = 1 on the kz = 0 and kz = nz/2
  planes, where both k and -k are stored.  n_b = sum of w over the shell.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np


@dataclasses.dataclass
class BinTable:
    shape: tuple
    n_bins: int
    bin_of: np.ndarray      # (nx, ny, nz//2+1) int64: shell id, -1 at DC, B = overflow
    weight: np.ndarray      # (nx, ny, nz//2+1) int64: 1 or 2
    partner: np.ndarray     # (nx, ny, nz//2+1) int64: stored index of -k (edge planes)
    edge_plane: np.ndarray  # (nx, ny, nz//2+1) bool: kz in {0, nz/2}
    n_b: np.ndarray         # (B+1,) int64: full-grid modes per shell


def signed_wavenumbers(n: int) -> np.ndarray:
    """m = 0, 1, ..., n/2, -(n/2 - 1), ..., -1 for a DFT axis of length n."""
    k = np.arange(n)
    return np.where(k <= n // 2, k, k - n)


def make_bins(shape: Sequence[int], L: Sequence[float], n_bins: int,
              k_edges: Optional[Sequence[float]] = None) -> BinTable:
    nx, ny, nz = (int(v) for v in shape)
    if nz % 2:
        raise ValueError("nz must be even")
    B = int(n_bins)
    if B < 1:
        raise ValueError("n_bins must be >= 1")
    nh = nz // 2 + 1
    mx = signed_wavenumbers(nx)[:, None, None]
    my = signed_wavenumbers(ny)[None, :, None]
    mz = np.arange(nh)[None, None, :]
    m2 = (mx ** 2 + my ** 2 + mz ** 2).astype(np.int64)
    m2 = np.broadcast_to(m2, (nx, ny, nh))

    if k_edges is None:
        if not (nx == ny == nz and L[0] == L[1] == L[2]):
            raise ValueError("linear default edges need a cubic grid; pass k_edges")
        h = nx // 2
        # largest b with b^2 h^2 <= B^2 m^2, i.e. b = isqrt(B^2 m^2) // h
        uniq, inv = np.unique(m2, return_inverse=True)
        b_u = np.array([math.isqrt(B * B * int(v)) // h for v in uniq], dtype=np.int64)
        b = b_u[inv].reshape(m2.shape)
        b = np.where(b >= B, B, b)
    else:
        e = np.asarray(k_edges, dtype=np.float64)
        if e.size != B + 1 or np.any(np.diff(e) <= 0) or e[0] < 0:
            raise ValueError("k_edges must hold n_bins+1 strictly increasing values >= 0")
        kx = 2 * np.pi * mx / L[0]
        ky = 2 * np.pi * my / L[1]
        kz = 2 * np.pi * mz / L[2]
        kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        kk = np.broadcast_to(kk, (nx, ny, nh))
        b = np.searchsorted(e, kk, side="right") - 1
        b = np.where((b < 0) | (b >= B), B, b).astype(np.int64)

    b = np.array(b, dtype=np.int64)
    b[0, 0, 0] = -1  # DC

    kz_idx = np.broadcast_to(np.arange(nh)[None, None, :], (nx, ny, nh))
    edge = (kz_idx == 0) | (kz_idx == nz // 2)
    weight = np.where(edge, 1, 2).astype(np.int64)
    kxi = np.arange(nx)[:, None, None]
    kyi = np.arange(ny)[None, :, None]
    partner = ((((-kxi) % nx) * ny + ((-kyi) % ny)) * nh + kz_idx).astype(np.int64)
    partner = np.broadcast_to(partner, (nx, ny, nh)).copy()

    keep = b >= 0
    n_b = np.bincount(b[keep], weights=weight[keep], minlength=B + 1).astype(np.int64)
    return BinTable((nx, ny, nz), B, b, weight, partner, edge, n_b)
