"""Philox4x32-10 and Box-Muller auxiliary fields (test infrastructure only).

Restated from the published definition of Philox (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit
counter, a 2x32-bit key, ten rounds of two 32x32->64-bit multiplications
with multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl
constants 0x9E3779B9 and 0xBB67AE85 between rounds.  Pinned against the
known-answer vectors published with that paper's Random123 library.

Field layout used by the library (both sides implement it independently):
counter = (q, walker, step, 0), key = (seed low 32 bits, seed high 32 bits),
where q indexes groups of four Cholesky fields n = 4q .. 4q+3.  The four
32-bit outputs (a, b, c, d) become two Box-Muller pairs:
  u1 = (a + 0.5) 2^-32, u2 = (b + 0.5) 2^-32, r = sqrt(-2 ln u1):
  x[4q] = r cos(2 pi u2), x[4q+1] = r sin(2 pi u2), and likewise (c, d) for
  x[4q+2], x[4q+3].
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

__all__ = ["philox4x32_10", "philox_fields"]


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on numpy uint64 arrays holding 32-bit values.

    ctr: tuple of 4 arrays (broadcastable); key: tuple of 2 arrays.  Returns 4 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK for k in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def philox_fields(seed: int, step: int, W: int, Nchol: int) -> np.ndarray:
    """Fields x[w, n] ~ N(0, 1) for one step (float64 [W, Nchol])."""
    nq = (Nchol + 3) // 4
    q = np.arange(nq, dtype=np.uint64)[None, :]
    w = np.arange(W, dtype=np.uint64)[:, None]
    zero = np.zeros((W, nq), dtype=np.uint64)
    a, b, c, d = philox4x32_10((q + zero, w + zero, zero + np.uint64(step), zero),
                               (np.uint64(seed & MASK), np.uint64((seed >> 32) & MASK)))
    inv = 2.0 ** -32
    out = np.empty((W, nq, 4))
    for (u, v), cols in (((a, b), (0, 1)), ((c, d), (2, 3))):
        u1 = (u.astype(np.float64) + 0.5) * inv
        u2 = (v.astype(np.float64) + 0.5) * inv
        r = np.sqrt(-2.0 * np.log(u1))
        out[:, :, cols[0]] = r * np.cos(2.0 * np.pi * u2)
        out[:, :, cols[1]] = r * np.sin(2.0 * np.pi * u2)
    return out.reshape(W, nq * 4)[:, :Nchol].copy()
