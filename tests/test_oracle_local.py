"""Pins of the local (Yamamoto) line-of-sight power spectrum oracle (oracle/local.py), CPU only.

* The normalised real harmonics of the footnote of Sec. 3.3.1 satisfy the addition theorem
  sum_m Ybar_lm(a) Ybar_lm(b) = L_l(a.b) (closed form).
* The FFT form of the numerator (eq. pk-num-fft) equals its definition 1/2 u^T (dxi/dp_alpha) u summed over every
  pair of cells and binned mode (eq. xi-p-alpha-deriv, no FFTs, no harmonic expansion).
* With the observer far away along z the local estimator tends to the global-line-of-sight one.
* One Monte Carlo term of the Fisher matrix (eq. fish-from-Q with eq. Q-alpha-local) equals the explicit matrix
  product 1/2 a^T (s C_alpha s C^asym_beta) a built from dense N x N derivative matrices.
"""
import numpy as np
import pytest

from oracle import _fft, binning, local, unwindowed
from paper_2404_07249_gb300 import synth


@pytest.mark.parametrize("ell", [0, 2, 4])
def test_addition_theorem(ell):
    rng = np.random.Generator(np.random.PCG64(ell + 1))
    a = rng.standard_normal((200, 3))
    b = rng.standard_normal((200, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    s = sum(local.ybar(ell, m, a) * local.ybar(ell, m, b) for m in range(-ell, ell + 1))
    mu = np.sum(a * b, axis=1)
    assert np.max(np.abs(s - binning.legendre(ell, mu * mu))) < 1e-12


def _setup(grid, box, observer):
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5, 3.5])
    bins = binning.bin_grid(grid, box, edges)
    geom = synth.SurveyGeometry(r_min=0.1 * box, r_max=0.45 * box, n_holes=1, hole_radius=0.05 * box,
                                n0=3.0e-4, r0=0.3 * box, s2=0.02 * box * box)
    n = synth.survey_mask(grid, (box,) * 3, 3, geom)
    w = unwindowed.fkp_weight(n, 1.0e4)
    d = n * synth.lognormal_field(grid, (box,) * 3, 7, kaiser_beta=0.5)
    xhat = local.position_units(grid, box, observer)
    khat = local.mode_units(grid)
    return edges, bins, n, w, d, xhat, khat


def test_numerator_fft_form_equals_definition():
    grid, box = (8, 8, 8), 400.0
    edges, bins, n, w, d, xhat, khat = _setup(grid, box, (13.0, -27.0, 41.0))
    nb = len(edges) - 1
    ells = [0, 2, 4]
    fft = local.pk_numerator_local(d, w, bins, nb, ells, xhat, khat)
    direct = local.pk_numerator_local_direct(d, w, bins, nb, ells, xhat, khat)
    assert np.max(np.abs(fft - direct)) <= 1e-11 * np.max(np.abs(direct))
    # and it differs from the global line of sight (the pin is not trivial)
    glob = unwindowed.pk_numerator(d, w, bins, binning.mu2_grid(grid), nb, ells)
    assert np.max(np.abs(fft[1] - glob[1])) > 1e-3 * np.max(np.abs(glob[1]))


def test_far_observer_tends_to_global_line_of_sight():
    grid, box = (16, 16, 16), 600.0
    edges, bins, n, w, d, _, khat = _setup(grid, box, (0.0, 0.0, 0.0))
    nb = len(edges) - 1
    ells = [0, 2, 4]
    xhat = local.position_units(grid, box, (0.0, 0.0, -1.0e10))   # every cell seen along +z (to 3e-8 rad)
    loc = local.pk_numerator_local(d, w, bins, nb, ells, xhat, khat)
    glob = unwindowed.pk_numerator(d, w, bins, binning.mu2_grid(grid), nb, ells)
    assert np.max(np.abs(loc - glob)) <= 1e-6 * np.max(np.abs(glob))


def _dense_derivatives(bins, b, ell, xhat, khat):
    """C^asym[x, y] = (1/N) sum_k e^{ik(x-y)} Theta_b(k) L_ell(k.y) and C = (C^asym + C^asym^T) / 2 (dense)."""
    grid = bins.shape
    N = bins.size
    xs = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    xh = xhat.reshape(-1, 3)
    f = [binning.int_freqs(g) for g in grid]
    Ca = np.zeros((N, N), dtype=np.complex128)
    for idx in zip(*np.nonzero(bins == b)):
        nvec = np.array([f[a][idx[a]] for a in range(3)], dtype=np.float64)
        ph = np.exp(2j * np.pi * (xs @ (nvec / np.array(grid, dtype=np.float64))))
        mu = xh @ khat[idx]
        L = binning.legendre(ell, mu * mu)
        Ca += np.outer(ph, np.conj(ph) * L)
    Ca = (Ca / N).real
    return 0.5 * (Ca + Ca.T), Ca


def test_fisher_draw_equals_dense_matrix_product():
    grid, box = (4, 4, 4), 300.0
    edges, bins, n, w, _, xhat, khat = _setup(grid, box, (7.0, 11.0, -5.0))
    nb = len(edges) - 1
    ells = [0, 2]
    s = (w * n).ravel()
    a = unwindowed.draw(grid, 99, 0, unwindowed.STREAM_P)
    F = local.pk_fisher_draw_local(a, n, w, bins, nb, ells, xhat, khat)
    alphas = [(ell, b) for ell in ells for b in range(nb)]
    mats = {al: _dense_derivatives(bins, al[1], al[0], xhat, khat) for al in alphas}
    av = a.ravel()
    want = np.zeros_like(F)
    for i, al in enumerate(alphas):
        Ci = mats[al][0]
        left = s * (Ci @ (s * av))              # s C_alpha s a
        for j, be in enumerate(alphas):
            want[i, j] = 0.5 * left @ (mats[be][1] @ av)
    scale = np.sqrt(np.abs(np.outer(np.diag(want), np.diag(want)))) + 1e-300
    assert np.max(np.abs(F - want) / scale) < 1e-10


def test_bk_local_multipole_pins():
    """Local-line-of-sight bispectrum multipoles (oracle local.bk_ideal_multipoles_local):
    * the harmonic spectrum sum_m Ybar_lm(k) FT[Ybar_lm delta](k) equals the definition inside eq. g-ell-def,
      sum_x e^{-ik.x} L_ell(k.x) delta(x) (explicit exponentials, no harmonics);
    * S^ell_abc equals the brute-force sum over closed triangles of D(k1) D(k2) H_ell(k3) (C, no FFT shells);
    * with the observer far away along z every cell sees the global line of sight: the global multipoles."""
    from oracle import brute, ideal
    grid, box = (8, 8, 8), 400.0
    kf = binning.kf_of(box)
    edges = kf * np.array([1.0, 2.0, 3.0, 4.0])
    obs = (31.0, -17.0, 45.0)
    f = synth.lognormal_field(grid, (box,) * 3, 21, kaiser_beta=0.5)
    xhat = local.position_units(grid, box, obs)
    khat = local.mode_units(grid)
    res = local.bk_ideal_multipoles_local(f, box, edges, 4, xhat, khat)
    xs = xhat.reshape(-1, 3)
    fl = f.ravel()
    pos = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    fr = [binning.int_freqs(g) for g in grid]
    for ell in (2, 4):
        H = res["H"][ell]
        for idx in [(1, 0, 0), (0, 2, 1), (3, 7, 2), (6, 1, 4), (2, 2, 2)]:
            nv = np.array([fr[a][idx[a]] for a in range(3)], dtype=np.float64)
            kh = nv / np.linalg.norm(nv)
            mu = xs @ kh
            want = np.sum(np.exp(-2j * np.pi * (pos @ (nv / np.array(grid)))) * binning.legendre(ell, mu * mu) * fl)
            assert abs(H[idx] - want) <= 1e-11 * np.max(np.abs(fl)) * fl.size
        D = ideal.forward(f)
        _, sdd = brute.brute_bk(D, grid, kf, edges, D2=D, D3=H)
        il = res["ells"].index(ell)
        want = np.array([sdd[t] for t in res["triplets"]]) / f.size ** 2
        assert np.max(np.abs(res["S"][il] - want)) <= 1e-10 * np.max(np.abs(want))
    far = local.position_units(grid, box, (0.0, 0.0, -1.0e10))
    loc = local.bk_ideal_multipoles_local(f, box, edges, 4, far, khat)["B"]
    glob = ideal.bk_ideal_multipoles(f, box, edges, 4)["B"]
    assert np.max(np.abs(loc - glob)) <= 1e-6 * np.max(np.abs(glob))
