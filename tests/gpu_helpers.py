"""Shared helpers of the GPU parity tests: run the CUDA library through its C
ABI and the oracle on the same seeded inputs, and compare."""
import numpy as np
import pytest

import mockgen
from oracle import sampler


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


# Tolerances of the draw-for-draw comparison (relative L2 over a field or P).
TOL = {64: 1e-12, 32: 2e-5}

# Element-wise companions of the L2 bars, so that a few bad voxels or shells
# cannot hide in a large field: (the largest |s_gpu - s_oracle| over the
# oracle field's RMS, the largest per-shell |P_gpu - P_oracle| / P_oracle).
# Set about ten times above the worst seen over every comparison of the GPU
# suite (FP64 3.0e-13 and 1.8e-13; FP32 1.3e-4, at 256^3 after one sweep, and
# 2.8e-5, at 32^3 after 200 sweeps).
EW_TOL = {64: (1e-11, 1e-11), 32: (1e-3, 2e-4)}
EW_SEEN = []  # (precision, worst voxel, worst shell, label) of every comparison made


def elementwise(a, b):
    """(max |a - b| / rms(b)) for a field; use on s."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    rms = float(np.sqrt(np.mean(b * b)))
    return float(np.max(np.abs(a - b)) / (rms if rms > 0 else 1.0))


def per_shell(a, b):
    """max over shells with P > 0 of |a - b| / b; use on P."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    keep = b > 0
    return float(np.max(np.abs(a[keep] - b[keep]) / b[keep])) if keep.any() else 0.0


def check_elementwise(precision, s_gpu, s_orc, p_gpu, p_orc, what=""):
    ev, es = elementwise(s_gpu, s_orc), per_shell(p_gpu, p_orc)
    EW_SEEN.append((precision, ev, es, what))
    assert ev <= EW_TOL[precision][0] and es <= EW_TOL[precision][1], (what, ev, es)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_1763_gb300 import build
    build.build()
    return torch


def oracle_chains(mock, n_bins, seed, chain_ids, P0=None, fix_P=False, k_edges=None, tau_scale=1.0):
    prob = sampler.make_problem(mock.shape, mock.L, mock.N, mock.R, mock.d, n_bins,
                                k_edges=k_edges, tau_scale=tau_scale)
    return sampler.Chains(prob, seed=seed, chain_ids=chain_ids, P0=P0, fix_P=fix_P)


def gpu_sampler(mock, n_bins, seed, precision, n_chains=1, **kw):
    from paper_1402_1763_gb300 import Sampler
    return Sampler.single(mock.n, mock.L, mock.N, mock.R, mock.d, n_bins, seed,
                          precision=precision, n_chains=n_chains, **kw)


def compare_run(mock, n_bins, seed, precision, checkpoints, n_chains=1, chain_ids=None, **kw):
    """Sweep both sides to each checkpoint; return the worst relative L2 of s
    and of P (over all chains) per checkpoint."""
    chain_ids = list(range(n_chains)) if chain_ids is None else chain_ids
    orc = oracle_chains(mock, n_bins, seed, chain_ids, P0=kw.get("P0"), fix_P=kw.get("fix_P", False),
                        k_edges=kw.get("k_edges"), tau_scale=kw.get("tau_scale", 1.0))
    out = []
    with gpu_sampler(mock, n_bins, seed, precision, n_chains=n_chains, **kw) as g:
        done = 0
        for cp in checkpoints:
            orc.sweep(cp - done)
            g.sweep(cp - done)
            done = cp
            es, ep = 0.0, 0.0
            for c in range(n_chains):
                sg, pg = g.read_s(c), g.read_pk(c)
                es = max(es, rel_l2(sg, orc.s[c]))
                ep = max(ep, rel_l2(pg, orc.P[c]))
                check_elementwise(precision, sg, orc.s[c], pg, orc.P[c], f"n={mock.n} sweep {cp} chain {c}")
            out.append((cp, es, ep))
    return out
