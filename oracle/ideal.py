"""Ideal-limit estimators (oracle; FP64): uniform density, global line of sight, P_fid = nbar = m = 1.

Sec. 3.4.1 (eq. pk-limit, eq. fish-ideal-continuous) for P_ell; Sec. 4.3.1 (eqs. beta-def, g-ell-def,
N-ell-def) and Sec. 4.4.1 (eqs. bk-num-ideal, bk-fish-ideal2) for the bispectrum; Sec. 4.1 (eqs. Bk-Yam, ideal-bk)
for its multipoles ell = 2, 4 about the global line of sight.

Pixel convention: D = fftn(delta); IFT = ifftn (includes 1/N).  With V the box volume and N the number of
cells, the physical outputs are

    P_ell(b) = (2 ell + 1) (V / N^2) sum_{k in b} L_ell(mu) |D(k)|^2 / N_b
    B_abc    = (V^2 / N^3) S_abc / T_abc,  S_abc = sum_x g_a g_b g_c,  T_abc = sum_x t_a t_b t_c,
    g_b = IFT[Theta_b D],  t_b = IFT[Theta_b],  N_abc = N^2 T_abc  (number of closed ordered triangles
    k1 in a, k2 in b, k3 in c with k1 + k2 + k3 = 0 on the periodic grid).
"""
from __future__ import annotations

import numpy as np

from . import _fft, binning


def forward(delta: np.ndarray) -> np.ndarray:
    """D(k) = sum_x e^{-i k.x} delta(x): the discrete form of the paper's FT (Sec. 1, Fourier conventions).
    The input is promoted to float64 exactly."""
    return _fft.fftn(np.asarray(delta, dtype=np.float64))


def shell_maps_ell(D: np.ndarray, bins: np.ndarray, nb: int, ell: int, mu2: np.ndarray) -> np.ndarray:
    """g_{b,ell}(x) = IFT[Theta_b L_ell(k.n) D](x) with the global line of sight n = z (Sec. 4.3.1, eq. g-ell-def,
    distant-observer form; the conjugate is dropped as for ell = 0, see shell_maps)."""
    L = binning.legendre(ell, mu2)
    out = np.empty((nb,) + D.shape, dtype=np.float64)
    for b in range(nb):
        out[b] = _fft.ifftn(np.where(bins == b, L * D, 0.0)).real
    return out


def shell_maps(D: np.ndarray, bins: np.ndarray, nb: int, which=None) -> np.ndarray:
    """g_b(x) = IFT[Theta_b D](x) for ell = 0 and a global line of sight (Sec. 4.3.1, eq. g-ell-def;
    Sec. 4.4.1 g^ideal with P_fid = nbar = 1).  The complex conjugate in eq. g-ell-def only maps
    g(r) -> g(-r) for real input and leaves every triple sum unchanged, so it is dropped."""
    idx = list(range(nb)) if which is None else list(which)
    out = np.empty((len(idx),) + D.shape, dtype=np.float64)
    for j, b in enumerate(idx):
        out[j] = _fft.ifftn(np.where(bins == b, D, 0.0)).real
    return out


def unit_maps(bins: np.ndarray, nb: int, which=None) -> np.ndarray:
    """t_b = IFT[Theta_b]: the shell maps of a unit spectrum (the N_ell FFT form of Sec. 4.3.1,
    ell = 0, P_fid = 1)."""
    return shell_maps(np.ones(bins.shape, dtype=np.complex128), bins, nb, which)


def triple_sums(g: np.ndarray) -> np.ndarray:
    """S[a, b, c] = sum_x g_a(x) g_b(x) g_c(x) for all a, b, c (the real-space sum of eq. beta-def).

    For each a the nb x nb block is the matrix product (g_a * G) G^T over the cells."""
    nb = g.shape[0]
    G = g.reshape(nb, -1)
    S = np.empty((nb, nb, nb))
    for a in range(nb):
        S[a] = (G * G[a]) @ G.T
    return S


def mixed_triple_sums(gu: np.ndarray, gv: np.ndarray) -> np.ndarray:
    """M[i, j, k] = sum_x gu_i(x) gv_j(x) gv_k(x): one field in the first slot, another in the last two."""
    nb = gu.shape[0]
    U = gu.reshape(nb, -1)
    Vm = gv.reshape(gv.shape[0], -1)
    M = np.empty((nb, Vm.shape[0], Vm.shape[0]))
    for i in range(nb):
        M[i] = (Vm * U[i]) @ Vm.T
    return M


def closed_triplets(T: np.ndarray, ncells: int):
    """Triplets a <= b <= c with at least one closed triangle: round(N^2 T_abc) > 0 (lexicographic)."""
    out = []
    nb = T.shape[0]
    for a, b, c in binning.triplets(nb):
        if round(ncells * ncells * T[a, b, c]) > 0:
            out.append((a, b, c))
    return out


def bk_ideal(delta: np.ndarray, box: float, edges) -> dict:
    """Ideal bispectrum, ell = 0 (Sec. 4.4.1).  b_num = S_abc / Delta (eq. bk-num-ideal, pixel units),
    F = N_abc / (N Delta) (eq. bk-fish-ideal2 with the delta_D(0) = N volume factor of a pixel trace),
    so b = F^-1 b_num = N S_abc / N_abc in pixel units and B = (V/N)^2 b in (Mpc/h)^6."""
    grid = delta.shape
    ncell = int(np.prod(grid))
    vol = float(box) ** 3
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    D = forward(delta)
    g = shell_maps(D, bins, nb)
    S = triple_sums(g)
    del g
    t = unit_maps(bins, nb)
    T = triple_sums(t)
    del t
    trip = closed_triplets(T, ncell)
    Sv = np.array([S[a, b, c] for a, b, c in trip])
    Tv = np.array([T[a, b, c] for a, b, c in trip])
    Nabc = np.rint(ncell * ncell * Tv)
    B = (vol * vol / float(ncell) ** 3) * Sv / Tv
    return {"triplets": trip, "S": Sv, "T": Tv, "N_abc": Nabc, "B": B, "S_full": S, "T_full": T}


def bk_ideal_multipoles(delta: np.ndarray, box: float, edges, lmax: int) -> dict:
    """Ideal bispectrum multipoles ell = 0, 2, .., lmax with a global line of sight (Sec. 4.1 eq. ideal-bk, which
    defines b_alpha; Sec. 4.4.1 with the continuous Fisher of eq. bk-fish-ideal2, under which Delta_alpha cancels):

        B_ell(a, b, c) = (2 ell + 1) (V^2 / N^3) S^ell_abc / T_abc,   S^ell_abc = sum_x g_a g_b g_{c,ell},

    the Legendre weight L_ell(k3.n) on the mode of the third (largest) bin, T_abc and the closed triplets as in
    bk_ideal (N_0 = N^2 T_abc).  Returns B[ell index][triplet] and the sums S[ell index][triplet]."""
    grid = delta.shape
    ncell = int(np.prod(grid))
    vol = float(box) ** 3
    nb = len(edges) - 1
    ells = list(range(0, lmax + 1, 2))
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    D = forward(delta)
    g = shell_maps(D, bins, nb)
    T = triple_sums(unit_maps(bins, nb))
    trip = closed_triplets(T, ncell)
    Tv = np.array([T[a, b, c] for a, b, c in trip])
    G = g.reshape(nb, -1)
    S = np.zeros((len(ells), len(trip)))
    for il, ell in enumerate(ells):
        gl = g if ell == 0 else shell_maps_ell(D, bins, nb, ell, mu2)
        GL = gl.reshape(nb, -1)
        # M[a, b, c] = sum_x g_a g_b g_{c,ell}: for each a the matrix product (g_a * G) GL^T
        for t, (a, b, c) in enumerate(trip):
            S[il, t] = np.dot(G[a] * G[b], GL[c])
    B = np.array([(2 * ell + 1) * (vol * vol / float(ncell) ** 3) * S[il] / Tv for il, ell in enumerate(ells)])
    return {"triplets": trip, "ells": ells, "S": S, "T": Tv, "N_abc": np.rint(ncell * ncell * Tv), "B": B}


def pk_ideal(delta: np.ndarray, box: float, edges, lmax: int) -> dict:
    """Ideal P_ell, global line of sight (Sec. 3.4.1).

    Continuous-Fisher normalisation (eq. fish-ideal-continuous):
        P_ell(b) = (2 ell + 1) (V / N^2) sum_{k in b} L_ell |D|^2 / N_b.
    Discrete-Fisher variant (eq. pk-limit): per bin, p_num_ell = (1/2)(1/N) sum_{k in b} L_ell |D|^2 and
    F_{ell ell'} = (1/2) sum_{k in b} L_ell L_ell' (pixel units, including the trace volume factor N);
    p = F^-1 p_num, times V / N for physical units.
    """
    grid = delta.shape
    ncell = int(np.prod(grid))
    vol = float(box) ** 3
    nb = len(edges) - 1
    ells = list(range(0, lmax + 1, 2))
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    D = forward(delta)
    pw = np.abs(D) ** 2
    counts = binning.mode_counts(bins, nb)
    sel = bins >= 0
    num = np.zeros((len(ells), nb))
    for il, ell in enumerate(ells):
        L = binning.legendre(ell, mu2)
        num[il] = np.bincount(bins[sel], weights=(L * pw)[sel], minlength=nb)
    cont = np.zeros_like(num)
    for il, ell in enumerate(ells):
        cont[il] = (2 * ell + 1) * (vol / float(ncell) ** 2) * num[il] / counts
    # discrete Fisher per bin
    disc = np.zeros_like(num)
    fish = np.zeros((nb, len(ells), len(ells)))
    for il, l1 in enumerate(ells):
        for jl, l2 in enumerate(ells):
            w = binning.legendre(l1, mu2) * binning.legendre(l2, mu2)
            fish[:, il, jl] = 0.5 * np.bincount(bins[sel], weights=w[sel], minlength=nb)
    for b in range(nb):
        pnum = 0.5 * num[:, b] / ncell
        disc[:, b] = np.linalg.solve(fish[b], pnum) * (vol / ncell)
    return {"ells": ells, "P": cont, "P_discrete": disc, "num": num, "counts": counts, "fisher": fish}
