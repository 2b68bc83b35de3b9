"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as easy
as 1, 2, 3"), written from the published definition.

One round maps a 4-word counter (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with the 32x32->64 products split into high and low words, M0 = 0xD2511F53,
M1 = 0xCD9E8D57. Between rounds the key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85). Ten rounds, nine bumps.

Stream layout used by the renderer (a reading; the paper names no generator):
key = (seed low word, seed high word), counter = (pid low, pid high, bounce, 0).
A 32-bit output word x becomes the uniform (x >> 8) * 2**-24 in [0, 1), exact in
both float32 and float64.
"""

from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """ctr: (n, 4) uint32 counters; key: (2,) or (n, 2) uint32. Returns (n, 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4).copy()
    k = np.broadcast_to(np.asarray(key, dtype=np.uint64).reshape(-1, 2), (c.shape[0], 2)).copy()
    for r in range(10):
        if r > 0:
            k[:, 0] = (k[:, 0] + np.uint64(W0)) & MASK
            k[:, 1] = (k[:, 1] + np.uint64(W1)) & MASK
        p0 = M0 * c[:, 0]          # < 2**64, exact in uint64
        p1 = M1 * c[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = np.stack([hi1 ^ c[:, 1] ^ k[:, 0], lo1, hi0 ^ c[:, 3] ^ k[:, 1], lo0], axis=1)
    return c.astype(np.uint32)


def uniform24(x: np.ndarray) -> np.ndarray:
    """Top 24 bits of a 32-bit word as a float64 in [0, 1)."""
    return (np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)


def path_uniforms(seed: int, pid: np.ndarray, bounce: int) -> np.ndarray:
    """The four uniforms of path `pid` at `bounce` (counter = (pid lo, pid hi, bounce, 0))."""
    pid = np.asarray(pid, dtype=np.uint64)
    ctr = np.stack([pid & MASK, pid >> np.uint64(32),
                    np.full_like(pid, bounce), np.zeros_like(pid)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    return uniform24(philox4x32_10(ctr, key))
