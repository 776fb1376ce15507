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


def test_beta_of_one_map_is_six_triple_sums():
    grid, box = (12, 12, 12), 12.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5, 3.5])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    trip = binning.triplets(nb)
    u = np.random.Generator(np.random.PCG64(1)).standard_normal(grid)
    S = unwindowed.bk_numerator(u, np.ones(grid), [], bins, nb, trip)["S"]
    assert np.allclose(noise.beta_sym(u, u, u, bins, nb, trip), 6.0 * S, rtol=1e-12, atol=1e-12 * np.max(np.abs(S)))


def test_bk_bias_removes_poisson_shot_noise():
    """Pure Poisson noise on a masked density (delta = 0, unit weights: n3 = n, d2 = d): the numerator's mean is the
    three-point shot noise, and b_num - b_bias has mean zero (within 5 standard errors over 400 realisations),
    while b_num alone is biased at many standard errors."""
    grid, box = (12, 12, 12), 12.0
    vcell = 1.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5, 3.5])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    trip = binning.triplets(nb)
    rng = np.random.Generator(np.random.PCG64(7))
    n = 1.0 + rng.random(grid)
    n[rng.random(grid) < 0.2] = 0.0
    w = unwindowed.fkp_weight(n, 2.0)
    sinv = lambda v: w * v  # noqa: E731
    num, cor = [], []
    for r in range(400):
        d = np.random.Generator(np.random.PCG64(1000 + r)).poisson(n * vcell) / vcell - n
        bn = unwindowed.bk_numerator(d, w, [], bins, nb, trip)["b_num"]
        bb = noise.bk_bias(d, n, d, vcell, sinv, bins, nb, trip, 50 + r, 1, unwindowed.draw)
        num.append(bn)
        cor.append(bn - bb)
    num, cor = np.array(num), np.array(cor)
    se_n = num.std(axis=0, ddof=1) / np.sqrt(len(num))
    se_c = cor.std(axis=0, ddof=1) / np.sqrt(len(cor))
    assert np.all(np.abs(cor.mean(axis=0)) < 5 * se_c)
    assert np.max(np.abs(num.mean(axis=0)) / se_n) > 10


def test_bk_bias_expectation_equals_poisson_shot_noise_exactly():
    """Exact form of the previous test.  For unit Gaussian a1, a2 the Monte Carlo term's expectation is the sum of its
    values at a1 = a2 = e_m over the unit vectors (the second and fourth moments agree), and for pure Poisson noise
    (E[d_i d_j] = n_i / V_cell delta_ij, E[d_i d_j d_k] = n_i / V_cell^2 delta_ijk, n3 = n, d2 = d)
        E[b_bias] = sum_m [ term3(e_m, e_m) + (n_m / V_cell) term2(a = e_m, d2 = e_m, d = e_m) ],
        E[b_num]  = sum_m (n_m / V_cell^2) b_num(e_m),
    which must be equal: -2 + 3 = 1 times the three-point shot noise."""
    grid, box = (6, 6, 6), 9.0
    vcell = box ** 3 / np.prod(grid)
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    trip = binning.triplets(nb)
    rng = np.random.Generator(np.random.PCG64(9))
    n = 0.5 + rng.random(grid)
    n[rng.random(grid) < 0.2] = 0.0
    w = unwindowed.fkp_weight(n, 2.0)
    sinv = lambda v: w * v  # noqa: E731
    zero = np.zeros(grid)
    eb, en = 0.0, 0.0
    for m in range(n.size):
        e = np.zeros(n.size)
        e[m] = 1.0
        e = e.reshape(grid)
        nm = n.ravel()[m]
        eb = eb + noise.bk_bias_draw(e, e, zero, n, zero, vcell, sinv, bins, nb, trip)
        eb = eb + nm / vcell * noise.bk_bias_draw(e, e, e, zero, e, vcell, sinv, bins, nb, trip)
        en = en + nm / vcell ** 2 * unwindowed.bk_numerator(e, w, [], bins, nb, trip)["b_num"]
    assert np.max(np.abs(eb - en)) < 1e-10 * np.max(np.abs(en))
