"""k-space grid, shell bins and Legendre weights (oracle; FP64).

Bins are the top-hats Theta_b(k) of Sec. 3.1 (below eq. cf-pk-leg-def) and Sec. 4.1 (eq. Bk-Yam):
Theta_b(k) = 1 for e_b <= |k| < e_{b+1} (half-open), 0 otherwise; the k = 0 mode is never binned.
The box is cubic (one side L, k_F = 2 pi / L), so |k| = k_F sqrt(|n|^2) with integer n; the bin of a
mode is a function of the integer |n|^2, evaluated once in float64 as k_F * sqrt(s).

The line of sight is the last array axis (global line of sight n = z, Sec. 3.3.1): mu = n_z / |n|.
"""
from __future__ import annotations

import math

import numpy as np


def kf_of(box: float) -> float:
    return 2.0 * math.pi / float(box)


def int_freqs(n: int) -> np.ndarray:
    """Integer wave numbers of numpy's FFT ordering: 0, 1, ..., n/2-1, -n/2, ..., -1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def n2_grid(grid) -> np.ndarray:
    """|n|^2 on the full FFT grid (int64)."""
    a, b, c = (int_freqs(g) for g in grid)
    return a[:, None, None] ** 2 + b[None, :, None] ** 2 + c[None, None, :] ** 2


def nz_grid(grid) -> np.ndarray:
    c = int_freqs(grid[2])
    return np.broadcast_to(c[None, None, :], tuple(grid))


def bin_of_s(s: np.ndarray, kf: float, edges: np.ndarray) -> np.ndarray:
    """Bin index for integer |n|^2 = s: b with e_b <= kf*sqrt(s) < e_{b+1}; -1 if none or s == 0."""
    s = np.asarray(s, dtype=np.int64)
    k = kf * np.sqrt(s.astype(np.float64))
    edges = np.asarray(edges, dtype=np.float64)
    b = np.searchsorted(edges, k, side="right") - 1   # largest b with e_b <= k
    valid = (s > 0) & (b >= 0) & (b < len(edges) - 1)
    return np.where(valid, b, -1)


def bin_grid(grid, box: float, edges) -> np.ndarray:
    """Bin index of every mode of the full FFT grid."""
    return bin_of_s(n2_grid(grid), kf_of(box), edges)


def mu2_grid(grid) -> np.ndarray:
    """mu^2 = n_z^2 / |n|^2 (0 at k = 0)."""
    s = n2_grid(grid).astype(np.float64)
    nz = nz_grid(grid).astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(s > 0, nz * nz / np.where(s > 0, s, 1.0), 0.0)


def legendre(ell: int, mu2: np.ndarray) -> np.ndarray:
    """Legendre polynomial L_ell(mu) for even ell, as a function of mu^2."""
    if ell == 0:
        return np.ones_like(mu2)
    if ell == 2:
        return 0.5 * (3.0 * mu2 - 1.0)
    if ell == 4:
        return (35.0 * mu2 * mu2 - 30.0 * mu2 + 3.0) / 8.0
    raise ValueError("only ell = 0, 2, 4 are supported")


def mode_counts(bins: np.ndarray, nb: int) -> np.ndarray:
    """Number of modes of the full k-grid in each bin (both k and -k counted)."""
    return np.bincount(bins[bins >= 0].ravel(), minlength=nb).astype(np.float64)


def triplets(nb: int):
    """All bin triplets a <= b <= c in lexicographic order (Sec. 4.1: b1 <= b2 <= b3)."""
    return [(a, b, c) for a in range(nb) for b in range(a, nb) for c in range(b, nb)]


def degeneracy(a: int, b: int, c: int) -> float:
    """Delta_alpha for ell = 0 (Sec. 4.1, eq. Delta-alpha-def with N_0/N_0 = 1):
    1 if all bins differ, 2 if exactly two coincide (either a = b < c or a < b = c), 6 if a = b = c."""
    if a == b == c:
        return 6.0
    if a == b or b == c:
        return 2.0
    return 1.0
