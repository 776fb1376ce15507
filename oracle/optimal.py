"""Optimal weighting S^-1 by preconditioned conjugate gradients (Sec. 2.4, eq. cgd-operation-eqn and the transpose
equation beside it; Sec. 3.3.3, eq. Sinv-optimal and its distant-observer form) and the power spectrum estimator built
on it (oracle; FP64).  TEST INFRASTRUCTURE ONLY.

Data model of Sec. 2.3 (eqs. data-model, pointing, two-point-noise) with pixel window m = 1: d = n delta + eps,
C = P xi P^T + N, P = diag(n), N = diag(n2), xi = IFT[P(k) FT[.]] with P(k) = sum_ell P_ell(k) L_ell(mu) about the
global line of sight.  Discretised, int dy int_k e^{ik(x-y)} P(k) u(y) is exactly ifftn(P fftn(u)) (the cell volume
of dy cancels the 1/V_cell of int_k), so n, n2 are densities and P is a power in the matching units: n P is
dimensionless, as in the FKP weight 1 / (1 + n P_FKP).

On the cells with n > 0 (Phi = 1) the distant-observer equation for S^-1,
    n IFT[P FT[Phi S^-1 v]] + (n2 / n) Phi S^-1 v = v,
divided by n, reads A u = v / n with u = Phi S^-1 v and the symmetric positive definite operator (on the subspace)
    A = Phi (K + D) Phi,   K = IFT[P FT[.]],   D = n2 / n^2.
With G = A^-1 on the subspace (0 off it):  S^-1 v = G (v / n)  and, from the transpose equation,
S^-T v = (1/n) G v (Phi).  Hence S^-1 P a = G a and P^T S^-T u = G u when the weighting and the pointing use the
same n.

Preconditioner: the ideal weighting of eq. Sinv-ideal, i.e. the exact inverse for a uniform density, with the
noise level sigma = mean over the cells with n > 0 of n2 / n^2:  M^-1 r = Phi IFT[FT[Phi r] / (P(k) + sigma)].

The fiducial P_ell are given on the integer shells |n|^2 = s = 0 .. len-1 (|k| = k_F sqrt(s)) and are zero beyond,
as in the paper's validation (power outside the range of interest set to zero).
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning


# ------------------------------------------------------------------------------------------------ operator


def fiducial_grid(pfid, grid) -> np.ndarray:
    """P(k) = sum_ell P_ell(|n|^2) L_ell(mu) on the full FFT grid; pfid[il][s] is the multipole ell = 2 il on the
    shell |n|^2 = s, zero for s >= len(pfid[0])."""
    pfid = np.atleast_2d(np.asarray(pfid, dtype=np.float64))
    s = binning.n2_grid(grid)
    mu2 = binning.mu2_grid(grid)
    out = np.zeros(tuple(grid))
    ok = s < pfid.shape[1]
    for il in range(pfid.shape[0]):
        out[ok] += pfid[il][s[ok]] * binning.legendre(2 * il, mu2)[ok]
    return out


def noise_term(n, n2) -> np.ndarray:
    """D = n2 / n^2 where n > 0, else 0."""
    n = np.asarray(n, dtype=np.float64)
    return np.where(n > 0, np.asarray(n2, dtype=np.float64) / np.where(n > 0, n, 1.0) ** 2, 0.0)


def apply_a(u, n, n2, Pk) -> np.ndarray:
    """A u = Phi (IFT[P FT[Phi u]] + D u)."""
    phi = np.asarray(n) > 0
    u = np.where(phi, np.asarray(u, dtype=np.float64), 0.0)
    return np.where(phi, _fft.ifftn(Pk * _fft.fftn(u)).real + noise_term(n, n2) * u, 0.0)


def precond_sigma(n, n2) -> float:
    """sigma = mean of n2 / n^2 over the cells with n > 0."""
    n = np.asarray(n, dtype=np.float64)
    return float(np.mean(noise_term(n, n2)[n > 0]))


def apply_precond(r, n, Pk, sigma: float) -> np.ndarray:
    """M^-1 r = Phi IFT[FT[Phi r] / (P(k) + sigma)] (eq. Sinv-ideal for a uniform density)."""
    phi = np.asarray(n) > 0
    r = np.where(phi, np.asarray(r, dtype=np.float64), 0.0)
    return np.where(phi, _fft.ifftn(_fft.fftn(r) / (Pk + sigma)).real, 0.0)


def pcg(b, apply_A, apply_M, max_iter: int, tol: float):
    """Preconditioned conjugate gradients for A x = b from x = 0 (Hestenes and Stiefel 1952); stops when
    ||r|| <= tol ||b|| or after max_iter iterations.  Returns (x, iterations, ||r|| / ||b||) with r the recursively
    updated residual."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.sqrt(np.sum(b * b))
    if bnorm == 0.0:
        return x, 0, 0.0
    z = apply_M(r)
    p = z.copy()
    rz = np.sum(r * z)
    it = 0
    rel = 1.0
    while it < max_iter:
        q = apply_A(p)
        alpha = rz / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = np.sqrt(np.sum(r * r)) / bnorm
        if rel <= tol:
            break
        z = apply_M(r)
        rz_new = np.sum(r * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel


def g_pcg(rhs, n, n2, Pk, max_iter: int = 500, tol: float = 1e-12, sigma=None):
    """G rhs by PCG with the ideal preconditioner: (x, iterations, relative residual)."""
    sigma = precond_sigma(n, n2) if sigma is None else float(sigma)
    phi = np.asarray(n) > 0
    b = np.where(phi, np.asarray(rhs, dtype=np.float64), 0.0)
    return pcg(b, lambda u: apply_a(u, n, n2, Pk), lambda r: apply_precond(r, n, Pk, sigma), max_iter, tol)


def _over_n(v, n) -> np.ndarray:
    n = np.asarray(n, dtype=np.float64)
    return np.where(n > 0, np.asarray(v, dtype=np.float64) / np.where(n > 0, n, 1.0), 0.0)


def sinv_apply(v, n, n2, Pk, max_iter: int = 500, tol: float = 1e-12) -> np.ndarray:
    """S^-1 v = G (v / n) (eq. cgd-operation-eqn, distant observer), by PCG."""
    return g_pcg(_over_n(v, n), n, n2, Pk, max_iter, tol)[0]


def sinv_t_apply(v, n, n2, Pk, max_iter: int = 500, tol: float = 1e-12) -> np.ndarray:
    """S^-T v = (1/n) G v (the transpose equation, distant observer), by PCG."""
    return _over_n(g_pcg(v, n, n2, Pk, max_iter, tol)[0], n)


# ------------------------------------------------------------------------------------------------ dense forms


def dense_operator(n, n2, Pk):
    """(A, sel): A restricted to the cells with n > 0 (flat indices sel), column j from K e_j = IFT[P FT[e_j]]."""
    grid = np.shape(n)
    nf = np.asarray(n, dtype=np.float64).ravel()
    sel = np.nonzero(nf > 0)[0]
    A = np.empty((len(sel), len(sel)))
    for c, j in enumerate(sel):
        e = np.zeros(nf.size)
        e[j] = 1.0
        A[:, c] = _fft.ifftn(Pk * _fft.fftn(e.reshape(grid))).real.ravel()[sel]
    A[np.arange(len(sel)), np.arange(len(sel))] += noise_term(n, n2).ravel()[sel]
    return A, sel


def g_dense(A, sel, rhs) -> np.ndarray:
    """G rhs by a dense LAPACK solve on the subspace."""
    out = np.zeros(np.size(rhs))
    out[sel] = np.linalg.solve(A, np.asarray(rhs, dtype=np.float64).ravel()[sel])
    return out.reshape(np.shape(rhs))


# ------------------------------------------------------------------------------------------------ P estimator


def pk_numerator_general(d, sinv, bins, mu2, nb, ells) -> np.ndarray:
    """p_num_alpha = 1/2 (1/N) sum_{k in b} L_ell |FT[S^-1 d]|^2 (Sec. 3.3.1, global line of sight) for a weighting
    given as a callable v -> S^-1 v.  Shape [len(ells), nb]."""
    u = sinv(np.asarray(d, dtype=np.float64))
    pw = np.abs(_fft.fftn(u)) ** 2
    sel = bins >= 0
    out = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        L = binning.legendre(ell, mu2)
        out[il] = 0.5 * np.bincount(bins[sel], weights=(L * pw)[sel], minlength=nb) / u.size
    return out


def pk_fisher_draw_general(a, n, sinv, sinv_t, bins, mu2, nb, ells) -> np.ndarray:
    """One Monte Carlo term of the P Fisher matrix (Sec. 3.3.2, eq. fish-from-Q, A = I, global line of sight) for a
    weighting given by callables v -> S^-1 v and v -> S^-T v, pointing P = diag(n):

        F_ab = 1/2 (P^T S^-T Q_alpha[S^-1 P a]) . Q_beta[a],   Q_alpha[u] = IFT[Theta_b L_ell FT[u]],

    as a Fourier-space dot product 1/2 (1/N) Re sum_k conj(FT[P^T S^-T Q_alpha[S^-1 P a]]) Theta_b' L_ell' FT[a]."""
    a = np.asarray(a, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    Afft = _fft.fftn(a)
    SA = _fft.fftn(sinv(n * a))
    alphas = [(ell, b) for ell in ells for b in range(nb)]
    Lw = {ell: binning.legendre(ell, mu2) for ell in ells}
    sel = bins >= 0
    Y = np.stack([np.where(bins == b, Lw[ell] * Afft, 0.0)[sel] for ell, b in alphas])
    X = np.empty_like(Y)
    for i, (ell, b) in enumerate(alphas):
        q = _fft.ifftn(np.where(bins == b, Lw[ell] * SA, 0.0)).real
        X[i] = _fft.fftn(n * sinv_t(q))[sel]
    return 0.5 * (np.conj(X) @ Y.T).real / a.size


def optimal_weighting(nw, n2w, Pk, max_iter: int = 500, tol: float = 1e-12):
    """(sinv, sinv_t) callables of the optimal weighting for the weighting densities (nw, n2w), by PCG."""
    return (lambda v: sinv_apply(v, nw, n2w, Pk, max_iter, tol),
            lambda v: sinv_t_apply(v, nw, n2w, Pk, max_iter, tol))


def pk_numerator_opt(d, nw, n2w, Pk, bins, mu2, nb, ells, max_iter: int = 500, tol: float = 1e-12) -> np.ndarray:
    """Numerator with the optimal weighting (PCG to ``tol``)."""
    return pk_numerator_general(d, optimal_weighting(nw, n2w, Pk, max_iter, tol)[0], bins, mu2, nb, ells)


def pk_fisher_opt(n, nw, n2w, Pk, bins, mu2, nb, ells, seed: int, n_mc: int, draw, stream: int, dtype=np.float64,
                  max_iter: int = 500, tol: float = 1e-12) -> np.ndarray:
    """Average of ``pk_fisher_draw_general`` with the optimal weighting over draws r = 0..n_mc-1 of ``stream``
    (``draw(grid, seed, r, stream, dtype)`` gives the Monte Carlo map)."""
    sinv, sinv_t = optimal_weighting(nw, n2w, Pk, max_iter, tol)
    F = 0.0
    for r in range(n_mc):
        F = F + pk_fisher_draw_general(draw(np.shape(n), seed, r, stream, dtype), n, sinv, sinv_t, bins, mu2, nb, ells)
    return F / n_mc
