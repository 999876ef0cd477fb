"""Counter-based Gaussian test matrix Omega (CPU oracle; test infrastructure).

Philox4x32-10 is written from its published definition (J. Salmon, M. Moraes,
R. Dror, D. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3):
a 4 x 32-bit counter and a 2 x 32-bit key go through 10 rounds; each round
multiplies words 0 and 2 by the two Philox multipliers (64-bit products split
into high and low halves), xors the high halves with the other two counter
words and the key, and permutes; the key is advanced by the two Weyl constants
between rounds.

The randn(n, k+s) of Alg. 1/4/5 (step 1) is realised as follows, identically on
every side that needs it:
  counter = (row i, column j, call_lo, call_hi), key = (seed_lo, seed_hi)
  (x0, x1, x2, x3) = Philox4x32-10(counter, key)
  u1 = (x0 + 1) * 2^-32  in (0, 1],   u2 = x1 * 2^-32  in [0, 1)
  Omega[i, j] = sqrt(-2 ln u1) * cos(2 pi u2)            (Box-Muller)
Column j does not depend on the matrix width, so widening Omega (k growing in
the SVT loop) keeps its leading columns.  This oracle evaluates the transform
in float64.
"""
from __future__ import annotations

import numpy as np

# Philox4x32 constants (Salmon et al., SC'11): round multipliers and the Weyl
# sequence increments used to bump the key between rounds.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32 with 10 rounds.  All inputs are broadcastable
    integer arrays holding 32-bit values; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (x.copy() for x in (c0, c1, c2, c3))
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        p0 = PHILOX_M0 * c0  # < 2^64, exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def philox_words(n: int, k: int, seed: int, call_id: int, col0: int = 0):
    """Raw (x0, x1) words for the n x k block of Omega starting at column col0."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(col0, col0 + k, dtype=np.uint64)[None, :]
    seed = int(seed)
    call_id = int(call_id)
    x0, x1, _, _ = philox4x32_10(i, j, call_id & 0xFFFFFFFF, (call_id >> 32) & 0xFFFFFFFF,
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return x0, x1


def omega(n: int, k: int, seed: int, call_id: int = 0, col0: int = 0) -> np.ndarray:
    """Gaussian test matrix Omega (n x k, float64): Alg. 1/4/5 step 1."""
    x0, x1 = philox_words(n, k, seed, call_id, col0)
    u1 = (x0.astype(np.float64) + 1.0) * 2.0**-32
    u2 = x1.astype(np.float64) * 2.0**-32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
