"""Masked ("unwindowed") estimators with FKP weighting, global line of sight (oracle; FP64).

Data model (Sec. 2.3, eqs. data-model and pointing, with pixel window m = 1 and no noise):
d(x) = n(x) delta(x), pointing matrix P = n (diagonal).  Weighting (Sec. 2.4, eq. Sinv-fkp, m = 1):
S^-1 = w = 1 / (1 + n P_FKP) (diagonal), so S^-1 P = w n.  Pixel convention throughout; the physical
outputs are P = p V / N and B = b (V / N)^2.

Monte Carlo draws (Sec. 3.3.2 eq. girard-hutchinson; Sec. 4.3.4): unit-variance Gaussian white noise
from ``philox.gaussian_draw`` so that A = I and A^-1 a = a.  Streams: 0 and 1 are the pair (a1, a2) of
the bispectrum Fisher, 2 the power-spectrum Fisher draws.
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning
from .ideal import shell_maps
from .philox import gaussian_draw

STREAM_B1, STREAM_B2, STREAM_P = 0, 1, 2


def fkp_weight(n: np.ndarray, p_fkp: float) -> np.ndarray:
    """w_FKP(x) = 1 / (n(x) P_FKP + 1)  (Sec. 2.4, eq. Sinv-fkp, no pixel window)."""
    return 1.0 / (np.asarray(n, dtype=np.float64) * p_fkp + 1.0)


def draw(grid, seed: int, r: int, stream: int, dtype=np.float64) -> np.ndarray:
    """Monte Carlo map ``r`` of ``stream``; ``dtype=float32`` gives the canonical FP32-rounded map."""
    a = gaussian_draw(int(np.prod(grid)), seed, r, stream).reshape(grid)
    return a.astype(dtype).astype(np.float64)


# ------------------------------------------------------------------------------------------------ P


def alpha_list_p(nb: int, ells):
    """alpha = (ell, b), ell-major: index il * nb + b."""
    return [(ell, b) for ell in ells for b in range(nb)]


def pk_numerator(d, w, bins, mu2, nb, ells) -> np.ndarray:
    """p_num_alpha = (1/2) int_k Theta_b L_ell |FT[S^-1 d]|^2 (Sec. 3.3.1, global line of sight),
    pixel units: (1/2)(1/N) sum_{k in b} L_ell |fftn(w d)|^2.  Shape [len(ells), nb]."""
    N = d.size
    U = _fft.fftn(np.asarray(w, dtype=np.float64) * np.asarray(d, dtype=np.float64))
    pw = np.abs(U) ** 2
    sel = bins >= 0
    out = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        L = binning.legendre(ell, mu2)
        out[il] = 0.5 * np.bincount(bins[sel], weights=(L * pw)[sel], minlength=nb) / N
    return out


def pk_fisher_draw(a, n, w, bins, mu2, nb, ells) -> np.ndarray:
    """One Monte Carlo term of the P Fisher matrix (Sec. 3.3.2, eq. fish-from-Q, global line of sight):

        F_ab = 1/2 (P^T S^-T Q_alpha[S^-1 P a]) . Q^asym_beta[A^-1 a],
        Q_alpha[u] = IFT[Theta_b L_ell FT[u]] (eq. Q-alpha-global),  Q^asym_beta[u](k) = Theta_b' L_ell' u(k),

    evaluated as a Fourier-space dot product: (1/2)(1/N) Re sum_k conj(FT[s Q_alpha[s a]]) Theta_b' L_ell' FT[a],
    with s = w n and A = I."""
    N = a.size
    s = np.asarray(w, dtype=np.float64) * np.asarray(n, dtype=np.float64)
    A = _fft.fftn(a)
    SA = _fft.fftn(s * a)
    alphas = alpha_list_p(nb, ells)
    Lw = {ell: binning.legendre(ell, mu2) for ell in ells}
    sel = bins >= 0          # Y_beta vanishes outside the binned modes: the dot product runs over those only
    Y = np.stack([np.where(bins == b, Lw[ell] * A, 0.0)[sel] for ell, b in alphas])
    X = np.empty_like(Y)
    for i, (ell, b) in enumerate(alphas):
        q = _fft.ifftn(np.where(bins == b, Lw[ell] * SA, 0.0)).real
        X[i] = _fft.fftn(s * q)[sel]
    return 0.5 * (np.conj(X) @ Y.T).real / N


def pk_fisher(n, w, bins, mu2, nb, ells, seed: int, n_mc: int, dtype=np.float64) -> np.ndarray:
    """Average of ``pk_fisher_draw`` over draws r = 0..n_mc-1 of stream 2."""
    F = 0.0
    for r in range(n_mc):
        F = F + pk_fisher_draw(draw(n.shape, seed, r, STREAM_P, dtype), n, w, bins, mu2, nb, ells)
    return F / n_mc


# ------------------------------------------------------------------------------------------------ B


def bk_numerator(d, w, mocks, bins, nb, trip) -> dict:
    """b_num_alpha (Sec. 4.3.2, eq. b-numerator-practical; ell = 0, global line of sight):

        b_num = (1/6) { beta[u,u,u] - ( <beta[u,v,v]>_Delta + 2 perms ) },  u = S^-1 d, v = S^-1 Delta.

    With beta from eq. beta-def (6 permutations, 1/Delta_alpha) this is
        b_num_abc = (1/Delta_abc) ( S_abc[u] - lin_abc ),
        lin_abc   = < sum_x g_a[u] g_b[v] g_c[v] + g_a[v] g_b[u] g_c[v] + g_a[v] g_b[v] g_c[u] >_Delta.
    """
    u = np.asarray(w, dtype=np.float64) * np.asarray(d, dtype=np.float64)
    gu = shell_maps(_fft.fftn(u), bins, nb)
    G = gu.reshape(nb, -1)
    S = np.array([np.dot(G[a] * G[b], G[c]) for a, b, c in trip])
    lin = np.zeros(len(trip))
    for mock in mocks:
        v = np.asarray(w, dtype=np.float64) * np.asarray(mock, dtype=np.float64)
        H = shell_maps(_fft.fftn(v), bins, nb).reshape(nb, -1)
        lin += np.array([np.dot(G[a] * H[b], H[c]) + np.dot(H[a] * G[b], H[c]) + np.dot(H[a] * H[b], G[c])
                         for a, b, c in trip])
    if len(mocks):
        lin /= len(mocks)
    dlt = np.array([binning.degeneracy(*t) for t in trip])
    return {"S": S, "lin": lin, "b_num": (S - lin) / dlt}


def q_maps(u, bins, nb, trip) -> np.ndarray:
    """Q_alpha[u](x) for every triplet (Sec. 4.3.4, eq. Q-bis-global, ell = 0):

        Q_abc[u] = (2/Delta) IFT[ Theta_c FT[g_a g_b] + Theta_a FT[g_b g_c] + Theta_b FT[g_a g_c] ],

    with g = shell_maps(FT[u]); both complex conjugates of eq. Q-bis-global cancel for real u and are
    dropped.  Each pair product is transformed once.  Shape [len(trip), N]."""
    g = shell_maps(_fft.fftn(np.asarray(u, dtype=np.float64)), bins, nb)
    pair_ft = {}

    def P(i, j):
        key = (min(i, j), max(i, j))
        if key not in pair_ft:
            pair_ft[key] = _fft.fftn(g[key[0]] * g[key[1]])
        return pair_ft[key]

    out = np.empty((len(trip), u.size))
    for t, (a, b, c) in enumerate(trip):
        spec = np.where(bins == c, P(a, b), 0.0) + np.where(bins == a, P(b, c), 0.0) \
            + np.where(bins == b, P(a, c), 0.0)
        out[t] = (2.0 / binning.degeneracy(a, b, c)) * _fft.ifftn(spec).real.ravel()
    return out


def bk_fisher_draw(a1, a2, n, w, bins, nb, trip) -> np.ndarray:
    """One Monte Carlo term of the bispectrum Fisher matrix (Sec. 4.3.4, eq. bk-fish-def), A = I:

        F_ab = (1/24) (Q_alpha[S^-1 P a1] - Q_alpha[S^-1 P a2]) . (S^-1 P) . (Q_beta[a1] - Q_beta[a2]),

    the dot being the sum over cells and S^-1 P = w n."""
    s = (np.asarray(w, dtype=np.float64) * np.asarray(n, dtype=np.float64)).ravel()
    X = q_maps(s.reshape(a1.shape) * a1, bins, nb, trip) - q_maps(s.reshape(a2.shape) * a2, bins, nb, trip)
    Y = q_maps(a1, bins, nb, trip) - q_maps(a2, bins, nb, trip)
    return (X * s) @ Y.T / 24.0


def bk_fisher(n, w, bins, nb, trip, seed: int, n_mc: int, dtype=np.float64) -> np.ndarray:
    """Average of ``bk_fisher_draw`` over pairs r = 0..n_mc-1 (streams 0 and 1)."""
    F = 0.0
    for r in range(n_mc):
        a1 = draw(n.shape, seed, r, STREAM_B1, dtype)
        a2 = draw(n.shape, seed, r, STREAM_B2, dtype)
        F = F + bk_fisher_draw(a1, a2, n, w, bins, nb, trip)
    return F / n_mc


def solve(F: np.ndarray, x_num: np.ndarray) -> np.ndarray:
    """x_hat = F^-1 x_num (eq. pk-estimator-def / eq. bk-estimator-def; no bias term in this data model)."""
    return np.linalg.solve(F, x_num)
