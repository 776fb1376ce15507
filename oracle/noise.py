"""Poisson shot-noise bias terms of the unwindowed estimators (oracle; FP64).  TEST INFRASTRUCTURE ONLY.

Data model with noise (Sec. 2.3, eqs. data-model, pointing and two-point-noise, pixel window m = 1):
d = n delta + eps with <eps eps^T> = N = diag(n2 / V_cell), the Dirac delta of the continuum becoming 1 / V_cell on
a grid of cells of volume V_cell (n, n2 densities, as for the optimal weighting).  Estimators subtract the bias from
the numerator before the Fisher solve: x_hat = F^-1 (x_num - x_bias) (eqs. pk-estimator-def, bk-estimator-def).

Power spectrum (Sec. 3.3.2, first line of eq. fish-from-Q, A = I, global line of sight):
    p_bias_alpha = 1/2 < (S^-1 N a) . Q^asym_alpha[S^-1 a] >_a = 1/2 Tr(S^-1 N S^-T C_alpha),
one Monte Carlo term being 1/2 (1/N) Re sum_{k in b} L_ell conj(FT[S^-1 N a]) FT[S^-1 a].  For a diagonal weighting
S^-1 = w the trace is closed: C_alpha has the constant diagonal (1/N) sum_{k in b} L_ell(mu_k), so
    p_bias_alpha = 1/2 (sum_x w^2 n2 / V_cell) (1/N) sum_{k in b} L_ell(mu_k).

Bispectrum (Sec. 4.3.3, eq. three-point-noise and the Monte Carlo form after it; A = I, ell = 0, global line of sight):
with the noise split as N_ijk = -2 N3_ijk + (d_i N2_jk + 2 perms), N3[u, v] = n3 u v / V_cell^2 and N2 u = d2 u / V_cell
(n3 the three-point noise density, d2 the doubly-weighted data minus randoms; n3 = n and d2 = d for unit weights),
    b_bias_alpha = -1/3 < beta_alpha[S^-1 N3[a1, a2], S^-1 a1, S^-1 a2] > + 1/2 < beta_alpha[S^-1 N2 a, S^-1 a, S^-1 d] >,
beta_alpha[X, Y, Z] = (1/Delta_alpha) sum_x of g_a g_b g_c over the six assignments of (X, Y, Z) to the bins (a, b, c)
(eq. beta-def).  The second average takes a = a1.  In the units of b_num = (S_abc - lin_abc) / Delta_abc.
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning
from .ideal import shell_maps


def pk_bias_draw(a, n2, vcell: float, sinv, bins, mu2, nb, ells) -> np.ndarray:
    """One Monte Carlo term of p_bias for a weighting given as a callable v -> S^-1 v; shape [len(ells), nb]."""
    a = np.asarray(a, dtype=np.float64)
    X = _fft.fftn(sinv(np.asarray(n2, dtype=np.float64) / vcell * a))
    Y = _fft.fftn(sinv(a))
    cr = (np.conj(X) * Y).real
    sel = bins >= 0
    out = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        L = binning.legendre(ell, mu2)
        out[il] = 0.5 * np.bincount(bins[sel], weights=(L * cr)[sel], minlength=nb) / a.size
    return out


def pk_bias(n2, vcell: float, sinv, bins, mu2, nb, ells, seed: int, n_mc: int, draw, stream: int,
            dtype=np.float64) -> np.ndarray:
    """Average of ``pk_bias_draw`` over draws r = 0..n_mc-1 of ``stream``."""
    out = 0.0
    for r in range(n_mc):
        out = out + pk_bias_draw(draw(np.shape(n2), seed, r, stream, dtype), n2, vcell, sinv, bins, mu2, nb, ells)
    return out / n_mc


def pk_bias_diagonal(w, n2, vcell: float, bins, mu2, nb, ells) -> np.ndarray:
    """Closed form of p_bias for a diagonal weighting S^-1 = w (the exact expectation of the Monte Carlo terms)."""
    w = np.asarray(w, dtype=np.float64)
    tr = float(np.sum(w * w * np.asarray(n2, dtype=np.float64))) / vcell
    sel = bins >= 0
    out = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        L = binning.legendre(ell, mu2)
        out[il] = 0.5 * tr * np.bincount(bins[sel], weights=L[sel], minlength=nb) / bins.size
    return out


def beta_sym(X, Y, Z, bins, nb, trip) -> np.ndarray:
    """Delta_alpha beta_alpha[X, Y, Z] = sum_x over the six assignments of (X, Y, Z) to (a, b, c) of g_a g_b g_c
    (eq. beta-def, ell = 0), for every triplet of ``trip``."""
    gx = shell_maps(_fft.fftn(np.asarray(X, dtype=np.float64)), bins, nb).reshape(nb, -1)
    gy = shell_maps(_fft.fftn(np.asarray(Y, dtype=np.float64)), bins, nb).reshape(nb, -1)
    gz = shell_maps(_fft.fftn(np.asarray(Z, dtype=np.float64)), bins, nb).reshape(nb, -1)
    out = np.empty(len(trip))
    for t, (a, b, c) in enumerate(trip):
        out[t] = (np.dot(gx[a] * gy[b], gz[c]) + np.dot(gx[a] * gz[b], gy[c]) + np.dot(gy[a] * gx[b], gz[c]) +
                  np.dot(gy[a] * gz[b], gx[c]) + np.dot(gz[a] * gx[b], gy[c]) + np.dot(gz[a] * gy[b], gx[c]))
    return out


def bk_bias_draw(a1, a2, d, n3, d2, vcell: float, sinv, bins, nb, trip) -> np.ndarray:
    """One Monte Carlo term of b_bias (weighting a callable v -> S^-1 v)."""
    a1 = np.asarray(a1, dtype=np.float64)
    a2 = np.asarray(a2, dtype=np.float64)
    x3 = sinv(np.asarray(n3, dtype=np.float64) * a1 * a2 / vcell ** 2)
    x2 = sinv(np.asarray(d2, dtype=np.float64) * a1 / vcell)
    s1, s2, sd = sinv(a1), sinv(a2), sinv(np.asarray(d, dtype=np.float64))
    dlt = np.array([binning.degeneracy(*t) for t in trip])
    return (-beta_sym(x3, s1, s2, bins, nb, trip) / 3.0 + beta_sym(x2, s1, sd, bins, nb, trip) / 2.0) / dlt


def bk_bias(d, n3, d2, vcell: float, sinv, bins, nb, trip, seed: int, n_mc: int, draw, streams=(4, 5),
            dtype=np.float64) -> np.ndarray:
    """Average of ``bk_bias_draw`` over the pairs r = 0..n_mc-1 of ``streams``."""
    out = 0.0
    for r in range(n_mc):
        a1 = draw(np.shape(d), seed, r, streams[0], dtype)
        a2 = draw(np.shape(d), seed, r, streams[1], dtype)
        out = out + bk_bias_draw(a1, a2, d, n3, d2, vcell, sinv, bins, nb, trip)
    return out / n_mc
