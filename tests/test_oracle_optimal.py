"""Pins of the optimal-weighting oracle (oracle/optimal.py), CPU only.

* Optimality (Sec. 2.2, eq. general-Sinv-optimality): the S^-1 the PCG route produces satisfies
  S^-1 C S^-T = S^-1 P and (S^-1 C)_IJ = P_IJ on the cells with n > 0, with C = P xi P^T + N built from an explicit
  sum over modes (no FFT; the fiducial P(k, mu) evaluated mode by mode, Legendre polynomials written out).
* Uniform density without holes: G is the Fourier-diagonal inverse 1 / (P(k) + 1/nbar) (eq. Sinv-ideal), and the
  preconditioned iteration (whose preconditioner is then exact) converges in one step.
* PCG reaches the dense LAPACK solution; S^-T is the adjoint of S^-1 (<u, S^-1 v> = <S^-T u, v>).
* With an FKP weighting passed in as the callables, the general numerator and Fisher term reduce to the pinned FKP
  oracle; with the optimal weighting the Fisher term equals 1/2 (P^T S^-T C_alpha S^-1 P a) . (C_beta a) from dense
  derivative matrices.
"""
import numpy as np
import pytest

from oracle import binning, optimal, unwindowed
from paper_2404_07249_gb300 import synth


def _leg(ell, mu):
    if ell == 0:
        return 1.0
    if ell == 2:
        return 1.5 * mu * mu - 0.5
    return (35.0 * mu ** 4 - 30.0 * mu * mu + 3.0) / 8.0


def _modes(grid):
    f = [binning.int_freqs(g) for g in grid]
    return np.array([(a, b, c) for a in f[0] for b in f[1] for c in f[2]], dtype=np.float64)


def _p_of_mode(pfid, nvec):
    s = int(round(nvec @ nvec))
    if s >= len(pfid[0]):
        return 0.0
    mu = nvec[2] / np.sqrt(s) if s > 0 else 0.0
    return sum(pfid[il][s] * _leg(2 * il, mu) for il in range(len(pfid)))


def _dense_xi(grid, weight_of_mode):
    """xi[x, y] = (1/N) sum_k e^{ik(x-y)} W(k), explicit exponentials (cell volume 1)."""
    xs = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    N = xs.shape[0]
    out = np.zeros((N, N), dtype=np.complex128)
    for nvec in _modes(grid):
        wk = weight_of_mode(nvec)
        if wk == 0.0:
            continue
        ph = np.exp(2j * np.pi * (xs @ (nvec / np.array(grid, dtype=np.float64))))
        out += wk * np.outer(ph, np.conj(ph))
    return (out / N).real


def _masked(grid, seed, nbar=1.0, holes=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nbar * (0.5 + rng.random(grid))
    if holes:
        n[rng.random(grid) < 0.25] = 0.0
    n2 = n * (0.7 + 0.6 * rng.random(grid))
    return n, n2


def _pfid(ns, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    p0 = 2.0 + 8.0 * rng.random(ns)
    return np.stack([p0, 0.6 * p0 * rng.random(ns), 0.2 * p0 * rng.random(ns)])


def test_optimality_condition():
    grid = (6, 6, 6)
    n, n2 = _masked(grid, 3)
    pfid = _pfid(20, 4)
    Pk = optimal.fiducial_grid(pfid, grid)
    N = n.size
    S = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        S[:, j] = optimal.sinv_apply(e.reshape(grid), n, n2, Pk, tol=1e-14).ravel()
    xi = _dense_xi(grid, lambda nv: _p_of_mode(pfid, nv))
    Pm = np.diag(n.ravel())
    C = Pm @ xi @ Pm.T + np.diag(n2.ravel())
    lhs = S @ C @ S.T
    rhs = S @ Pm
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(rhs))
    m = n.ravel() > 0
    SC = S @ C
    assert np.max(np.abs(SC[np.ix_(m, m)] - Pm[np.ix_(m, m)])) < 1e-10 * np.max(n)
    assert np.all(S[~m, :] == 0.0) and np.all(S[:, ~m] == 0.0)


def test_uniform_density_is_the_ideal_weighting():
    grid = (8, 8, 8)
    nbar = 0.8
    n = np.full(grid, nbar)
    pfid = _pfid(30, 5)
    Pk = optimal.fiducial_grid(pfid, grid)
    rng = np.random.Generator(np.random.PCG64(6))
    v = rng.standard_normal(grid)
    want = np.fft.ifftn(np.fft.fftn(v) / (Pk + 1.0 / nbar)).real
    A, sel = optimal.dense_operator(n, n, Pk)
    assert np.max(np.abs(optimal.g_dense(A, sel, v) - want)) < 1e-12 * np.max(np.abs(want))
    x, it, rel = optimal.g_pcg(v, n, n, Pk, tol=1e-13)
    assert it == 1 and rel < 1e-13
    assert np.max(np.abs(x - want)) < 1e-12 * np.max(np.abs(want))
    # S^-1 of eq. Sinv-ideal: (1/nbar) IFT[FT[v] / (P + 1/nbar)] = G (v / nbar)
    assert np.max(np.abs(optimal.sinv_apply(v, n, n, Pk) - want / nbar)) < 1e-12 * np.max(np.abs(want / nbar))


def test_pcg_matches_dense_solve_and_adjoint():
    grid = (12, 12, 12)
    n, n2 = _masked(grid, 7, nbar=0.3)
    Pk = optimal.fiducial_grid(_pfid(60, 8), grid)
    rng = np.random.Generator(np.random.PCG64(9))
    v = rng.standard_normal(grid)
    u = rng.standard_normal(grid)
    A, sel = optimal.dense_operator(n, n2, Pk)
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.max(np.abs(A)))
    want = optimal.g_dense(A, sel, v * (n > 0))
    x, it, rel = optimal.g_pcg(v, n, n2, Pk, tol=1e-13)
    assert rel <= 1e-13 and it < 200
    assert np.max(np.abs(x - want)) < 1e-10 * np.max(np.abs(want))
    # unpreconditioned CG reaches the same point
    x0, _, _ = optimal.pcg(np.where(n > 0, v, 0.0), lambda w: optimal.apply_a(w, n, n2, Pk), lambda r: r, 2000, 1e-13)
    assert np.max(np.abs(x0 - want)) < 1e-9 * np.max(np.abs(want))
    lhs = np.sum(u * optimal.sinv_apply(v, n, n2, Pk, tol=1e-14))
    rhs = np.sum(optimal.sinv_t_apply(u, n, n2, Pk, tol=1e-14) * v)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def _survey(grid, box, seed):
    geom = synth.SurveyGeometry(r_min=0.1 * box, r_max=0.45 * box, n_holes=1, hole_radius=0.05 * box,
                                n0=3.0e-4, r0=0.3 * box, s2=0.02 * box * box)
    n = synth.survey_mask(grid, (box,) * 3, seed, geom)
    return n


def test_general_form_reduces_to_fkp():
    grid, box = (16, 16, 16), 500.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5, 3.5, 4.5])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    n = _survey(grid, box, 3)
    w = unwindowed.fkp_weight(n, 1.0e4)
    d = n * synth.lognormal_field(grid, (box,) * 3, 7, kaiser_beta=0.5)
    a = unwindowed.draw(grid, 11, 0, unwindowed.STREAM_P)
    ells = [0, 2]
    fkp = lambda v: w * v  # noqa: E731  (S^-1 = S^-T = w, diagonal)
    got = optimal.pk_numerator_general(d, fkp, bins, mu2, nb, ells)
    want = unwindowed.pk_numerator(d, w, bins, mu2, nb, ells)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    F = optimal.pk_fisher_draw_general(a, n, fkp, fkp, bins, mu2, nb, ells)
    R = unwindowed.pk_fisher_draw(a, n, w, bins, mu2, nb, ells)
    assert np.max(np.abs(F - R)) <= 1e-12 * np.max(np.abs(R))


def test_optimal_fisher_draw_and_numerator_equal_dense_products():
    grid, box = (4, 4, 4), 4.0    # cell volume 1
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    n, n2 = _masked(grid, 12)
    pfid = _pfid(10, 13)
    Pk = optimal.fiducial_grid(pfid, grid)
    ells = [0, 2]
    N = n.size
    S = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        S[:, j] = optimal.sinv_apply(e.reshape(grid), n, n2, Pk, tol=1e-14).ravel()
    Pm = np.diag(n.ravel())
    alphas = [(ell, b) for ell in ells for b in range(nb)]

    def c_alpha(ell, b):
        def wk(nv):
            s = int(round(nv @ nv))
            if s == 0 or bins[tuple(int(x) % g for x, g in zip(nv, grid))] != b:
                return 0.0
            return _leg(ell, nv[2] / np.sqrt(s))
        return _dense_xi(grid, wk)

    Cs = {al: c_alpha(*al) for al in alphas}
    a = unwindowed.draw(grid, 21, 0, unwindowed.STREAM_P).ravel()
    sinv, sinv_t = optimal.optimal_weighting(n, n2, Pk, tol=1e-14)
    F = optimal.pk_fisher_draw_general(a.reshape(grid), n, sinv, sinv_t, bins, mu2, nb, ells)
    want = np.empty_like(F)
    for i, al in enumerate(alphas):
        left = Pm.T @ S.T @ Cs[al] @ S @ Pm @ a
        for j, be in enumerate(alphas):
            want[i, j] = 0.5 * left @ (Cs[be] @ a)
    scale = np.sqrt(np.abs(np.outer(np.diag(want), np.diag(want))))
    assert np.max(np.abs(F - want) / scale) < 1e-10
    d = np.random.Generator(np.random.PCG64(22)).standard_normal(N) * n.ravel()
    u = S @ d
    pnum = optimal.pk_numerator_general(d.reshape(grid), sinv, bins, mu2, nb, ells)
    for i, (ell, b) in enumerate(alphas):
        assert abs(pnum[ells.index(ell), b] - 0.5 * u @ Cs[(ell, b)] @ u) < 1e-10 * abs(0.5 * u @ Cs[(ell, 0)] @ u)
