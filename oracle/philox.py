"""Philox4x32-10 counter-based generator and the Box-Muller normals drawn from it.

ORACLE — test infrastructure only.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline use it.

The paper (Sec. 3.4) asks for one independent, seeded generator per core so that
parallel univariate draws never collide.  Here that role is played by a
counter-based generator: every draw is a pure function of
(key = seed, counter = (index, sweep, chain, stream)), so any element can be
drawn by any thread in any order.  The generator is Philox4x32 with 10 rounds as
published by Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
1, 2, 3" (SC'11), restated here from that definition:

  * state: four 32-bit counter words (c0, c1, c2, c3), two 32-bit key words;
  * one round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit products,
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
  * between rounds the key is bumped by the Weyl constants (W0, W1);
  * M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85.

Stream ids (counter word 3):
  0 = messenger draw (Alg. 1, first loop), 1 = signal-mode draw (Alg. 1
  second loop), 2 = over-dispersed starts, 4 = the mixing sampler's proposals
  (Alg. 3), 5 = the chi-square draw of each shell (Alg. 2 on shells).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_MESSENGER = 0
STREAM_MODES = 1
STREAM_START = 2   # over-dispersed starting powers (sampler.Chains)
STREAM_MIXING = 4  # the mixing sampler's per-shell proposals (oracle/mixing.py)
STREAM_CHI2 = 5    # the chi-square draw of each shell (sampler.chi2_shell_draws)


def philox4x32_10(c0, c1, c2, c3, seed: int):
    """Return the four 32-bit output words for counters (c0, c1, c2, c3).

    The counter words broadcast against each other (numpy arrays or scalars);
    the key is (seed & 0xffffffff, seed >> 32).  Products are formed in uint64
    so the high and low halves are exact.
    """
    c = [np.asarray(x).astype(np.uint64) & MASK32 for x in (c0, c1, c2, c3)]
    c = list(np.broadcast_arrays(*c))
    c = [x.copy() for x in c]
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    for rnd in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        if rnd != 9:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
    return tuple(x.astype(np.uint32) for x in c)


def uniform_open0(w):
    """Map a 32-bit word to U = (w + 1/2) * 2^-32, exactly in FP64.

    The half-offset keeps U away from 0 so that log(U) in Box-Muller is finite:
    the smallest word maps to 2^-33, the largest to 1 - 2^-33 (which becomes
    exactly 1 once rounded to FP32), so U lies in (0, 1].
    """
    w = np.asarray(w).astype(np.float64)
    return (2.0 * w + 1.0) * 2.0 ** -33


def box_muller(wa, wb):
    """Box & Muller (1958): two independent unit normals from two words.

    r = sqrt(-2 ln U_a), z = r cos(2 pi U_b), z' = r sin(2 pi U_b).
    """
    ua = uniform_open0(wa)
    ub = uniform_open0(wb)
    r = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return r * np.cos(ang), r * np.sin(ang)


def normals4(c0, c1, c2, c3, seed: int):
    """Four unit normals (z0, z1, z2, z3) from one Philox call.

    (z0, z1) come from words (w0, w1) and (z2, z3) from (w2, w3).
    """
    w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, c3, seed)
    z0, z1 = box_muller(w0, w1)
    z2, z3 = box_muller(w2, w3)
    return z0, z1, z2, z3
