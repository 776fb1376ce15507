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
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning


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
