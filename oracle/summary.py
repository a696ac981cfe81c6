"""Summaries of a recorded P(k) trace: the statistical-efficiency analysis of
the paper's results section and posterior quantiles, FP64 numpy.

ORACLE — test infrastructure only (see ``oracle/sampler.py``).

trace has shape (R, B+1): R recorded samples of each shell's amplitude.

* Autocorrelation (the paper's correlation coefficient of subsequent
  power-spectrum amplitudes): for lag n,
      C_n = [1/(R-n) sum_{i<R-n} (P_i - <P>)(P_{i+n} - <P>)] / Var(P),
  with <P> and Var(P) = <(P - <P>)^2> over the whole trace (<P> formed as
  P_0 + <P - P_0>, equal in exact arithmetic and exactly P_0 for a constant
  trace; chain means below likewise).  The correlation
  length n_c is the first lag n >= 1 at which C_n drops below 0.1 (the
  paper's criterion); -1 if it does not within the lags asked for.  A constant
  trace has no defined correlation; it is reported as C_n = 1, n_c = -1.
* Gelman-Rubin R-hat across m chains' traces (records burn .. R-1, n of
  them): chain means m_j, unbiased variances v_j, W = mean v_j,
  B = n/(m-1) sum (m_j - mean m)^2, var+ = (n-1)/n W + B/n, R-hat = sqrt(var+/W).
* Quantile q: with the sorted samples x_(0) <= ... <= x_(R-1), h = (R-1) q and
  k = floor(h), x_(k) + (h - k) (x_(k+1) - x_(k)) (linear interpolation).
"""
from __future__ import annotations

import numpy as np


def acf(trace, max_lag: int):
    """Returns (C with shape (B+1, max_lag+1), n_c with shape (B+1,))."""
    x = np.asarray(trace, dtype=np.float64)
    R, B1 = x.shape
    if not 0 <= max_lag < R:
        raise ValueError("need 0 <= max_lag < R")
    C = np.ones((B1, max_lag + 1))
    nc = np.full(B1, -1, dtype=np.int64)
    for b in range(B1):
        col = x[:, b]
        m = col[0] + (col - col[0]).sum() / R  # about the first sample: exact for a constant trace
        dev = col - m
        var = (dev * dev).sum() / R
        if var > 0.0:
            for n in range(max_lag + 1):
                C[b, n] = (dev[:R - n] * dev[n:]).sum() / ((R - n) * var)
        for n in range(1, max_lag + 1):
            if C[b, n] < 0.1:
                nc[b] = n
                break
    return C, nc


def quantiles(trace, q):
    """Returns shape (B+1, len(q))."""
    x = np.sort(np.asarray(trace, dtype=np.float64), axis=0)
    R, B1 = x.shape
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    out = np.empty((B1, q.size))
    for i, qi in enumerate(q):
        h = (R - 1) * qi
        k = int(np.floor(h))
        k1 = min(k + 1, R - 1)
        out[:, i] = x[k] + (h - k) * (x[k1] - x[k])
    return out


def rhat(traces, burn: int = 0):
    """traces: list of m arrays (R, B+1).  Returns shape (B+1,)."""
    x = np.stack([np.asarray(t, dtype=np.float64)[burn:] for t in traces])  # (m, n, B+1)
    m, n, B1 = x.shape
    means = x[:, 0, :] + (x - x[:, :1, :]).sum(axis=1) / n  # about each chain's first sample
    var = ((x - means[:, None, :]) ** 2).sum(axis=1) / (n - 1)
    W = var.mean(axis=0)
    Bv = n / (m - 1) * ((means - means.mean(axis=0)) ** 2).sum(axis=0)
    vplus = (n - 1) / n * W + Bv / n
    out = np.empty(B1)
    for b in range(B1):
        if W[b] > 0:
            out[b] = np.sqrt(vplus[b] / W[b])
        else:
            out[b] = np.inf if Bv[b] > 0 else 1.0
    return out
