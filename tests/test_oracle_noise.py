"""Pins of the shot-noise oracle (oracle/noise.py), CPU only.

* One Monte Carlo term of p_bias equals the quadratic form 1/2 a^T N S^T C_alpha S a with a dense derivative matrix
  C_alpha from explicit exponentials, for a diagonal (FKP) and for the optimal (dense) weighting; its expectation
  over unit Gaussian a is then the trace 1/2 Tr(S N S^T C_alpha).
* The closed form for a diagonal weighting equals that trace.
* Uniform density n = n2 = nbar with w = 1: the shot-noise bias of the monopole is 1/nbar in physical units
  (p_bias / F with the ideal Fisher 1/2 nbar^2 Tr(C_alpha C_alpha) = 1/2 nbar^2 N_b, times V_cell).
"""
import numpy as np

from oracle import binning, noise, optimal, unwindowed


def _leg(ell, mu):
    return {0: 1.0, 2: 1.5 * mu * mu - 0.5, 4: (35.0 * mu ** 4 - 30.0 * mu * mu + 3.0) / 8.0}[ell]


def _dense_c(grid, bins, b, ell):
    """C_alpha[x, y] = (1/N) sum_{k in b} e^{ik(x-y)} L_ell(mu_k), explicit exponentials."""
    xs = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    N = xs.shape[0]
    f = [binning.int_freqs(g) for g in grid]
    out = np.zeros((N, N), dtype=np.complex128)
    for idx in zip(*np.nonzero(bins == b)):
        nv = np.array([f[a][idx[a]] for a in range(3)], dtype=np.float64)
        ph = np.exp(2j * np.pi * (xs @ (nv / np.array(grid, dtype=np.float64))))
        out += _leg(ell, nv[2] / np.sqrt(nv @ nv)) * np.outer(ph, np.conj(ph))
    return (out / N).real


def _setup(grid, box):
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5])
    bins = binning.bin_grid(grid, box, edges)
    rng = np.random.Generator(np.random.PCG64(5))
    n = 0.5 + rng.random(grid)
    n[rng.random(grid) < 0.2] = 0.0
    n2 = n * (0.8 + 0.4 * rng.random(grid))
    return edges, bins, binning.mu2_grid(grid), n, n2


def test_draw_is_the_quadratic_form_and_closed_form_is_the_trace():
    grid, box = (4, 4, 4), 8.0
    vcell = box ** 3 / np.prod(grid)
    edges, bins, mu2, n, n2 = _setup(grid, box)
    nb, ells = len(edges) - 1, [0, 2]
    w = unwindowed.fkp_weight(n, 3.0)
    Pk = optimal.fiducial_grid(np.array([[0.0, 4.0, 3.0, 2.5, 2.0, 1.5, 1.2, 1.0, 0.8, 0.7]]), grid)
    N = n.size
    S_opt = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        S_opt[:, j] = optimal.sinv_apply(e.reshape(grid), n, n2, Pk, tol=1e-14).ravel()
    Nm = np.diag(n2.ravel() / vcell)
    a = unwindowed.draw(grid, 3, 0, 3)
    av = a.ravel()
    for S, sinv in ((np.diag(w.ravel()), lambda v: w * v),
                    (S_opt, lambda v: optimal.sinv_apply(v, n, n2, Pk, tol=1e-14))):
        got = noise.pk_bias_draw(a, n2, vcell, sinv, bins, mu2, nb, ells)
        for il, ell in enumerate(ells):
            for b in range(nb):
                C = _dense_c(grid, bins, b, ell)
                want = 0.5 * av @ (Nm @ S.T @ C @ S) @ av
                assert abs(got[il, b] - want) <= 1e-11 * max(abs(want), 1e-300) + 1e-14
    closed = noise.pk_bias_diagonal(w, n2, vcell, bins, mu2, nb, ells)
    S = np.diag(w.ravel())
    for il, ell in enumerate(ells):
        for b in range(nb):
            want = 0.5 * np.trace(S @ Nm @ S.T @ _dense_c(grid, bins, b, ell))
            assert abs(closed[il, b] - want) <= 1e-12 * abs(want) + 1e-15


def test_uniform_density_monopole_is_one_over_nbar():
    grid, box = (16, 16, 16), 400.0
    vcell = box ** 3 / np.prod(grid)
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 2.5, 4.5, 6.5])
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    nbar = 3.0e-4
    n = np.full(grid, nbar)
    pb = noise.pk_bias_diagonal(np.ones(grid), n, vcell, bins, mu2, len(edges) - 1, [0])
    Nb = binning.mode_counts(bins, len(edges) - 1)
    F = 0.5 * nbar ** 2 * Nb                      # ideal Fisher of the monopole, 1/2 nbar^2 Tr(C_a C_a), S^-1 = 1
    assert np.allclose(pb[0] / F * vcell, 1.0 / nbar, rtol=1e-12)
