"""Power spectrum with a local (Yamamoto) line of sight (oracle; FP64).  TEST INFRASTRUCTURE ONLY.

Sec. 3.1 (eqs. cf-pk-def, xi-p-alpha-deriv) defines the two-point function with the line of sight taken at each end
point x and y of a pair, symmetrised:

    dxi/dp_alpha (x, y) = 1/2 int_k e^{i k.(x - y)} Theta_b(k) [ L_ell(k.x) + (-1)^ell L_ell(k.y) ]   (unit vectors),

and Sec. 3.3 expands L_ell(k.x) = sum_m Ybar_lm(k) Ybar_lm(x) in the normalised real spherical harmonics of the
footnote of Sec. 3.3.1 to reach FFT forms: the numerator eq. pk-num-fft, the derivative maps eq. Q-alpha-local and
their asymmetric Fourier form (above eq. fish-from-Q), and the Monte Carlo Fisher matrix eq. fish-from-Q.  Even
multipoles only (the estimators here: ell = 0, 2, 4).

Pixel convention as in ``unwindowed``: int_k -> (1/N) sum_k, int dx -> sum_x, FT = fftn, IFT = ifftn; u = S^-1 d
with S^-1 = w (diagonal), S^-1 P = w n.  Positions are the cell centres (i + 1/2) L / N_i - L/2 of a box centred on
the origin, measured from an observer at ``observer``; k-directions are n / |n| of the integer wave vectors.
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning

try:  # scipy >= 1.15
    from scipy.special import sph_harm_y as _sph

    def _ylm(ell, m, theta, phi):
        return _sph(ell, m, theta, phi)
except ImportError:  # pragma: no cover - older scipy
    from scipy.special import sph_harm as _sph_old

    def _ylm(ell, m, theta, phi):
        return _sph_old(m, ell, phi, theta)


def ybar(ell: int, m: int, v: np.ndarray) -> np.ndarray:
    """Normalised real spherical harmonic Ybar_lm of the unit vectors v[..., 3], from the complex Y_lm by the footnote
    of Sec. 3.3.1:  sqrt((2l+1)/4pi) Ybar_lm = (i/sqrt2)[Y_lm - (-1)^m Y_l(-m)] (m < 0),
    (1/sqrt2)[Y_l(-m) + (-1)^m Y_lm] (m > 0), Y_l0 (m = 0); so that sum_m Ybar_lm(a) Ybar_lm(b) = L_l(a.b)."""
    v = np.asarray(v, dtype=np.float64)
    theta = np.arccos(np.clip(v[..., 2], -1.0, 1.0))
    phi = np.arctan2(v[..., 1], v[..., 0])
    if m == 0:
        y = _ylm(ell, 0, theta, phi)
    elif m < 0:
        y = (1j / np.sqrt(2.0)) * (_ylm(ell, m, theta, phi) - (-1.0) ** m * _ylm(ell, -m, theta, phi))
    else:
        y = (1.0 / np.sqrt(2.0)) * (_ylm(ell, -m, theta, phi) + (-1.0) ** m * _ylm(ell, m, theta, phi))
    return np.sqrt(4.0 * np.pi / (2 * ell + 1)) * np.real(y)


def position_units(grid, box: float, observer=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Unit vectors from the observer to the cell centres, shape grid + (3,) (the z axis where a centre coincides
    with the observer)."""
    axes = [(np.arange(n) + 0.5) * (box / n) - box / 2.0 - o for n, o in zip(grid, observer)]
    X = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    r = np.linalg.norm(X, axis=-1, keepdims=True)
    out = np.where(r > 0, X / np.where(r > 0, r, 1.0), np.array([0.0, 0.0, 1.0]))
    return out


def mode_units(grid) -> np.ndarray:
    """Unit vectors n / |n| of the FFT wave vectors, shape grid + (3,) (the z axis at n = 0, which is never binned)."""
    f = [binning.int_freqs(g).astype(np.float64) for g in grid]
    K = np.stack(np.meshgrid(*f, indexing="ij"), axis=-1)
    r = np.linalg.norm(K, axis=-1, keepdims=True)
    return np.where(r > 0, K / np.where(r > 0, r, 1.0), np.array([0.0, 0.0, 1.0]))


def _asym_spectra(u, ells, xhat, khat):
    """sum_m Ybar_lm(k) FT[Ybar_lm u](k) for each ell (the Theta-free part of Q^asym, above eq. fish-from-Q)."""
    out = {}
    for ell in ells:
        acc = 0.0
        for m in range(-ell, ell + 1):
            acc = acc + ybar(ell, m, khat) * _fft.fftn(ybar(ell, m, xhat) * u)
        out[ell] = acc
    return out


def pk_numerator_local(d, w, bins, nb, ells, xhat, khat) -> np.ndarray:
    """p_num_alpha = 1/2 sum_m int_k Theta_b Ybar_lm(k) (FT[Ybar_lm S^-1 d])^* FT[S^-1 d]  (Sec. 3.3.1,
    eq. pk-num-fft), pixel units: (1/2)(1/N) sum_k ...; real for even ell.  Shape [len(ells), nb]."""
    u = np.asarray(w, dtype=np.float64) * np.asarray(d, dtype=np.float64)
    N = u.size
    U = _fft.fftn(u)
    A = _asym_spectra(u, ells, xhat, khat)
    sel = bins >= 0
    out = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        val = np.real(np.conj(A[ell]) * U)
        out[il] = 0.5 * np.bincount(bins[sel], weights=val[sel], minlength=nb) / N
    return out


def pk_numerator_local_direct(d, w, bins, nb, ells, xhat, khat) -> np.ndarray:
    """The same numerator straight from its definition, p_num = 1/2 u^T (dxi/dp_alpha) u with eq. xi-p-alpha-deriv
    summed over every pair of cells and every binned mode (no FFTs, no harmonic expansion): O(N^2 N_modes).
    For the pins on small grids."""
    u = (np.asarray(w, dtype=np.float64) * np.asarray(d, dtype=np.float64)).ravel()
    N = u.size
    grid = bins.shape
    xs = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    xh = xhat.reshape(-1, 3)
    f = [binning.int_freqs(g) for g in grid]
    out = np.zeros((len(ells), nb))
    for idx in zip(*np.nonzero(bins >= 0)):
        b = bins[idx]
        n = np.array([f[a][idx[a]] for a in range(3)], dtype=np.float64)
        ph = np.exp(2j * np.pi * (xs @ (n / np.array(grid, dtype=np.float64))))   # e^{i k.x}
        kh = khat[idx]
        mu = xh @ kh
        for il, ell in enumerate(ells):
            L = binning.legendre(ell, mu * mu)
            # sum_{x,y} u_x u_y e^{ik(x-y)} [L(k.x) + L(k.y)] / 2 = Re( (sum_x u_x L_x e^{ikx}) conj(sum_y u_y e^{iky}) )
            s1 = np.sum(u * L * ph)
            s2 = np.sum(u * ph)
            out[il, b] += 0.5 * np.real(s1 * np.conj(s2)) / N
    return out


def q_local(u, bins, b, ell, xhat, khat) -> np.ndarray:
    """Q_alpha[u](x), alpha = (ell, b), for a local line of sight (Sec. 3.3.2, eq. Q-alpha-local, even ell):
    1/2 sum_m { Ybar_lm(x) IFT[Theta_b Ybar_lm FT[u]](x) + IFT[Theta_b Ybar_lm FT[Ybar_lm u]](x) }."""
    sel = bins == b
    U = _fft.fftn(u)
    out = 0.0
    for m in range(-ell, ell + 1):
        yk = ybar(ell, m, khat)
        yx = ybar(ell, m, xhat)
        out = out + yx * _fft.ifftn(np.where(sel, yk * U, 0.0)).real
        out = out + _fft.ifftn(np.where(sel, yk * _fft.fftn(yx * u), 0.0)).real
    return 0.5 * out


def pk_fisher_draw_local(a, n, w, bins, nb, ells, xhat, khat) -> np.ndarray:
    """One Monte Carlo term of the P Fisher matrix with a local line of sight (Sec. 3.3.2, eq. fish-from-Q, A = I):

        F_ab = 1/2 (P^T S^-T Q_alpha[S^-1 P a]) . Q^asym_beta[a]
             = 1/2 (1/N) Re sum_k conj(FT[s Q_alpha[s a]]) Theta_b' sum_m Ybar_l'm(k) FT[Ybar_l'm a](k),  s = w n."""
    N = a.size
    s = np.asarray(w, dtype=np.float64) * np.asarray(n, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    A = _asym_spectra(a, ells, xhat, khat)
    alphas = [(ell, b) for ell in ells for b in range(nb)]
    sel = bins >= 0
    Y = np.stack([np.where(bins == b, A[ell], 0.0)[sel] for ell, b in alphas])
    X = np.empty_like(Y)
    for i, (ell, b) in enumerate(alphas):
        X[i] = _fft.fftn(s * q_local(s * a, bins, b, ell, xhat, khat))[sel]
    return 0.5 * (np.conj(X) @ Y.T).real / N


def pk_fisher_local(n, w, bins, nb, ells, xhat, khat, seed: int, n_mc: int, draw, stream: int,
                    dtype=np.float64) -> np.ndarray:
    """Average of ``pk_fisher_draw_local`` over draws r = 0..n_mc-1 of ``stream`` (``draw`` as unwindowed.draw)."""
    F = 0.0
    for r in range(n_mc):
        F = F + pk_fisher_draw_local(draw(n.shape, seed, r, stream, dtype), n, w, bins, nb, ells, xhat, khat)
    return F / n_mc


def bk_ideal_multipoles_local(delta, box: float, edges, lmax: int, xhat, khat) -> dict:
    """Ideal bispectrum multipoles with a local line of sight (Sec. 4.3.1, eq. g-ell-def and its spherical-harmonic
    expansion; normalised as the global ones, Sec. 4.4.1):

        g_{c,ell}[u] = IFT[Theta_c sum_m Ybar_lm(k) FT[Ybar_lm(x) u]],   S^ell_abc = sum_x g_a g_b g_{c,ell},
        B_ell(a, b, c) = (2 ell + 1) (V^2 / N^3) S^ell_abc / T_abc,

    the line of sight x / |x| from the observer at each cell (xhat), the conjugates of eq. g-ell-def dropped as for
    the global line of sight (for real fields and even ell they reflect every map of a sum at once).  Returns the
    triplets, B[ell index][triplet] and S."""
    from .ideal import closed_triplets, forward, shell_maps, triple_sums, unit_maps
    delta = np.asarray(delta, dtype=np.float64)
    grid = delta.shape
    ncell = int(np.prod(grid))
    vol = float(box) ** 3
    nb = len(edges) - 1
    ells = list(range(0, lmax + 1, 2))
    bins = binning.bin_grid(grid, box, edges)
    G = shell_maps(forward(delta), bins, nb).reshape(nb, -1)
    T = triple_sums(unit_maps(bins, nb))
    trip = closed_triplets(T, ncell)
    Tv = np.array([T[a, b, c] for a, b, c in trip])
    H = _asym_spectra(delta, [e for e in ells if e > 0], xhat, khat)
    S = np.zeros((len(ells), len(trip)))
    for il, ell in enumerate(ells):
        GL = G if ell == 0 else shell_maps(H[ell], bins, nb).reshape(nb, -1)
        for t, (a, b, c) in enumerate(trip):
            S[il, t] = np.dot(G[a] * G[b], GL[c])
    B = np.array([(2 * ell + 1) * (vol * vol / float(ncell) ** 3) * S[il] / Tv for il, ell in enumerate(ells)])
    return {"triplets": trip, "ells": ells, "S": S, "T": Tv, "B": B, "H": H}
