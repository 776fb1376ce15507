"""Philox4x32-10 counter-based generator and the Gaussian Monte Carlo draws (oracle; FP64).

Generator: Philox4x32 with 10 rounds as published by Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11).  One round maps counter (c0, c1, c2, c3) and key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85).

Draw layout (the definition both implementations follow): the Monte Carlo map number ``draw`` of
stream ``stream`` has, at flat C-order cell index i, the value z_{i mod 4} of Philox block j = i // 4
with key = (seed mod 2^32, seed div 2^32) and counter = (j mod 2^32, j div 2^32, draw, stream).
From the four 32-bit outputs x0..x3, u_q = (x_q + 1/2) 2^-32 and Box-Muller gives
    z0 = r cos(2 pi u1), z1 = r sin(2 pi u1), r = sqrt(-2 ln u0);   z2, z3 likewise from (u2, u3).
These are unit-variance Gaussian white-noise maps: the draws a with A = <a a^T> = I used in the
Girard-Hutchinson Monte Carlo sums of Sec. 3.3.2 (eq. girard-hutchinson) and Sec. 4.3.4.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Arguments are uint32-valued arrays (held as uint64)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def gaussian_draw(ncell: int, seed: int, draw: int, stream: int) -> np.ndarray:
    """The float64 white-noise map number ``draw`` of ``stream`` (flat, length ncell)."""
    nblk = (ncell + 3) // 4
    j = np.arange(nblk, dtype=np.uint64)
    x = philox4x32_10(j & MASK, j >> np.uint64(32), np.uint64(draw), np.uint64(stream),
                      np.uint64(seed) & MASK, np.uint64(seed) >> np.uint64(32))
    u = [(xi.astype(np.float64) + 0.5) * 2.0 ** -32 for xi in x]
    r01 = np.sqrt(-2.0 * np.log(u[0]))
    r23 = np.sqrt(-2.0 * np.log(u[2]))
    z = np.empty((nblk, 4))
    z[:, 0] = r01 * np.cos(2.0 * np.pi * u[1])
    z[:, 1] = r01 * np.sin(2.0 * np.pi * u[1])
    z[:, 2] = r23 * np.cos(2.0 * np.pi * u[3])
    z[:, 3] = r23 * np.sin(2.0 * np.pi * u[3])
    return z.reshape(-1)[:ncell]
