"""Exact tiny-grid pins for the Monte Carlo Fisher matrices (CPU only).

On a 4^3 grid every operator of the estimators can be written as an explicit tensor built from DFT
matrices, with no FFT and no shell-filtered maps:

* bispectrum: Z_alpha[i,j,k] = d zeta(x_i, x_j, x_k) / d b_alpha
      = (1/Delta_alpha)(1/N^2) sum_{k1+k2+k3 = 0} e^{i(k1.x_i + k2.x_j + k3.x_k)} [Theta_a Theta_b Theta_c + 5 perms]
  (Sec. 4.1, eq. zeta-deriv in the pixel convention), so Q_alpha[u]_i = Z_alpha[i,j,k] u_j u_k and
  F_alpha,beta = (1/6) sum_ijk s_i s_j s_k Z_alpha Z_beta (eq. bk-estimator-def with S^-1 P = s);
* power spectrum: C_alpha(x, y) = d xi / d p_alpha = (1/N) sum_k e^{ik(x-y)} Theta_b L_ell (eq. xi-p-alpha-deriv,
  global line of sight), F = (1/2) Tr(s C_alpha s C_beta) (eq. pk-estimator-def).

The oracle's FFT-based Q maps and Monte Carlo terms are compared with these exactly (one draw), and the
Monte Carlo averages with the exact traces statistically.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import binning, brute, ideal, unwindowed

N1D = 4
GRID = (N1D,) * 3
BOX = 300.0
KF = binning.kf_of(BOX)
EDGES = KF * np.array([0.5, 1.5, 2.5, 3.5])
NB = 3


def _modes():
    f = binning.int_freqs(N1D)
    n = np.array(list(itertools.product(f, f, f)))        # C order, same as ravel of the grid
    return n


def _dft():
    n = _modes()
    r = np.array(list(itertools.product(range(N1D), range(N1D), range(N1D))))
    return np.exp(2j * math.pi * (r @ n.T) / N1D)          # E[r, k] = e^{i k.r}


def _bins_flat():
    return binning.bin_grid(GRID, BOX, EDGES).ravel()


def _z_tensor(trip):
    """Explicit Z_alpha[i,j,k] from closed triangles (k3 = -k1-k2 on the periodic grid)."""
    n = _modes()
    N = len(n)
    bins = _bins_flat()
    idx = {tuple(v % N1D): q for q, v in enumerate(n)}
    k3 = np.array([[idx[tuple((-(n[p] + n[q])) % N1D)] for q in range(N)] for p in range(N)])
    a, b, c = trip
    A = np.zeros((N, N))
    for p1, p2, p3 in set(itertools.permutations((a, b, c))):
        A += ((bins[:, None] == p1) & (bins[None, :] == p2) & (bins[k3] == p3))
    # multiplicity: permutations of a multiset count each distinct arrangement once in eq. Bk-Yam's
    # "+5 perms" sum; repeated bins repeat the same arrangement.
    mult = 6 // len(set(itertools.permutations((a, b, c))))
    A *= mult
    E = _dft()
    Ahat = (E @ A @ E.T).real                                 # Ahat[r1, r2] = sum A e^{i(k1 r1 + k2 r2)}
    r = np.array(list(itertools.product(range(N1D), range(N1D), range(N1D))))
    ridx = lambda v: ((v[..., 0] % N1D) * N1D + (v[..., 1] % N1D)) * N1D + (v[..., 2] % N1D)
    d1 = ridx(r[:, None, :] - r[None, :, :])                  # (x_i - x_k)
    Z = Ahat[d1[:, None, :], d1[None, :, :]]                  # Z[i,j,k] = Ahat[x_i - x_k, x_j - x_k]
    return Z / (binning.degeneracy(a, b, c) * N * N)


@pytest.fixture(scope="module")
def setup():
    bins = binning.bin_grid(GRID, BOX, EDGES)
    T = ideal.triple_sums(ideal.unit_maps(bins, NB))
    trip = ideal.closed_triplets(T, bins.size)
    Z = np.stack([_z_tensor(t) for t in trip])
    geom_s = 0.3 + np.random.Generator(np.random.PCG64(1)).random(GRID)    # a nonuniform S^-1 P
    return bins, trip, Z, geom_s


def test_q_maps_equal_tensor_contraction(setup):
    """The FFT form of Q_alpha (eq. Q-bis-global, pair products refiltered) equals Z_alpha[i,j,k] u_j u_k."""
    bins, trip, Z, _ = setup
    u = np.random.Generator(np.random.PCG64(2)).standard_normal(GRID)
    q = unwindowed.q_maps(u, bins, NB, trip)
    ref = np.einsum("tijk,j,k->ti", Z, u.ravel(), u.ravel())
    assert np.max(np.abs(q - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ideal_exact_fisher_is_diagonal_count(setup):
    """With S^-1 P = 1 the exact Fisher (1/6) Z.Z is diagonal with F_aa = N_abc / (N Delta_alpha)
    (Sec. 4.4.1, eq. bk-fish-ideal2, including the pixel-trace volume factor N)."""
    bins, trip, Z, _ = setup
    N = bins.size
    F = np.einsum("aijk,bijk->ab", Z, Z) / 6.0
    cnt, _ = brute.brute_bk(None, GRID, KF, EDGES)
    expect = np.diag([cnt[t] / (N * binning.degeneracy(*t)) for t in trip])
    assert np.max(np.abs(F - expect)) < 1e-10 * np.max(expect)


def test_bk_fisher_draw_equals_tensor_formula(setup):
    """One Monte Carlo term of eq. bk-fish-def computed by the oracle equals the explicit tensor formula."""
    bins, trip, Z, s = setup
    a1 = unwindowed.draw(GRID, 5, 0, unwindowed.STREAM_B1)
    a2 = unwindowed.draw(GRID, 5, 0, unwindowed.STREAM_B2)
    F = unwindowed.bk_fisher_draw(a1, a2, s, np.ones(GRID), bins, NB, trip)
    sv = s.ravel()
    Q = lambda u: np.einsum("tijk,j,k->ti", Z, u, u)
    X = Q(sv * a1.ravel()) - Q(sv * a2.ravel())
    Y = Q(a1.ravel()) - Q(a2.ravel())
    ref = (X * sv) @ Y.T / 24.0
    assert np.max(np.abs(F - ref)) < 1e-11 * np.max(np.abs(ref))


def test_bk_fisher_monte_carlo_converges_to_exact_trace(setup):
    """The average of eq. bk-fish-def over Gaussian draw pairs converges to the exact
    (1/6) sum s_i s_j s_k Z_alpha Z_beta (second-order Girard-Hutchinson, Sec. 4.3.4)."""
    bins, trip, Z, s = setup
    sv = s.ravel()
    Fex = np.einsum("aijk,bijk,i,j,k->ab", Z, Z, sv, sv, sv) / 6.0
    R = 1500
    acc = np.zeros_like(Fex)
    acc2 = np.zeros_like(Fex)
    for r in range(R):
        a1 = unwindowed.draw(GRID, 9, r, unwindowed.STREAM_B1)
        a2 = unwindowed.draw(GRID, 9, r, unwindowed.STREAM_B2)
        f = unwindowed.bk_fisher_draw(a1, a2, s, np.ones(GRID), bins, NB, trip)
        acc += f
        acc2 += f * f
    mean = acc / R
    sd = np.sqrt(np.maximum(acc2 / R - mean ** 2, 0.0) / R)
    z = (mean - Fex) / np.maximum(sd, 1e-300)
    assert np.max(np.abs(z)) < 5.0
    # the diagonal is resolved (the check is not vacuous)
    assert np.all(np.abs(np.diag(Fex)) > 4 * np.diag(sd))


def _c_matrix(b, ell):
    n = _modes()
    s2 = (n ** 2).sum(1).astype(float)
    mu2 = np.where(s2 > 0, n[:, 2] ** 2 / np.where(s2 > 0, s2, 1.0), 0.0)
    w = (_bins_flat() == b) * binning.legendre(ell, mu2)
    E = _dft()
    return ((E * w) @ E.conj().T).real / len(n)


def test_pk_fisher_draw_and_trace():
    """P Fisher: one oracle Monte Carlo term equals 1/2 (s C_a s a).(C_b a); the average over draws
    converges to 1/2 Tr(s C_a s C_b); with s = 1 the trace is (1/2) sum_{k in b} L_ell L_ell'."""
    bins = binning.bin_grid(GRID, BOX, EDGES)
    mu2 = binning.mu2_grid(GRID)
    ells = [0, 2]
    alphas = unwindowed.alpha_list_p(NB, ells)
    C = [_c_matrix(b, ell) for ell, b in alphas]
    s = 0.3 + np.random.Generator(np.random.PCG64(4)).random(GRID)
    sv = s.ravel()
    a = unwindowed.draw(GRID, 3, 0, unwindowed.STREAM_P)
    F1 = unwindowed.pk_fisher_draw(a, s, np.ones(GRID), bins, mu2, NB, ells)
    av = a.ravel()
    ref = np.array([[0.5 * (sv * (Ca @ (sv * av))) @ (Cb @ av) for Cb in C] for Ca in C])
    assert np.max(np.abs(F1 - ref)) < 1e-11 * np.max(np.abs(ref))
    Fex = np.array([[0.5 * np.trace(np.diag(sv) @ Ca @ np.diag(sv) @ Cb) for Cb in C] for Ca in C])
    R = 3000
    fs = np.array([unwindowed.pk_fisher_draw(unwindowed.draw(GRID, 3, r, unwindowed.STREAM_P), s, np.ones(GRID),
                                             bins, mu2, NB, ells) for r in range(R)])
    z = (fs.mean(0) - Fex) / np.maximum(fs.std(0) / math.sqrt(R), 1e-300)
    assert np.max(np.abs(z)) < 5.0
    one = np.ones(len(sv))
    Fid = np.array([[0.5 * np.trace(Ca @ Cb) for Cb in C] for Ca in C])
    w = {ell: binning.legendre(ell, mu2).ravel() for ell in ells}
    bf = bins.ravel()
    closed = np.array([[0.5 * np.sum((bf == b1) * (bf == b2) * w[l1] * w[l2]) for l2, b2 in alphas]
                       for l1, b1 in alphas])
    assert np.max(np.abs(Fid - closed)) < 1e-10 * np.max(np.abs(closed))
    del one
