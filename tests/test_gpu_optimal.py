"""GPU parity of the optimal weighting S^-1 (preconditioned conjugate gradients, eq. cgd-operation-eqn and its transpose
in the distant-observer limit) and of the P estimator built on it, against the FP64 oracle (oracle/optimal.py),
through the C-ABI.

Tolerances.  FP64 contexts: the same iteration as the oracle's in the same precision, so a fixed number of iterations
agrees to rounding (1e-10 relative) and a converged solve (tol 1e-12) agrees with the dense LAPACK solution within
kappa(A) 1e-12 (kappa below 1e2 on these masks: 1e-9).  FP32 contexts: the operator is applied with FP32 transforms
(relative error a few 1e-7 per application), so the residual b - A x the oracle recomputes in FP64 bottoms out near
1e-6 and the solution error is at most kappa(A) times that; the bounds below (2e-5 residual, 2e-4 solution) hold
kappa up to 100 with a factor 2 to spare.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, optimal, unwindowed
from paper_2404_07249_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    pkg.load()
    return pkg


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _random_mask(grid, seed, nbar):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nbar * (0.5 + rng.random(grid))
    n[rng.random(grid) < 0.3] = 0.0
    n2 = n * (0.7 + 0.6 * rng.random(grid))
    return n.astype(np.float32), n2.astype(np.float32)


def _survey(grid, box, seed):
    geom = synth.SurveyGeometry(r_min=0.1 * box, r_max=0.45 * box, n_holes=3, hole_radius=0.05 * box,
                                n0=3.0e-4, r0=0.3 * box, s2=0.02 * box * box)
    n = synth.survey_mask(grid, (box,) * 3, seed, geom).astype(np.float32)
    return n


def _kaiser_table(ns, kf, nell=3, amp=2.0e4):
    """Fiducial multipoles on the shells s = 0 .. ns-1: a smooth monopole and its Kaiser (beta = 0.5) multipoles."""
    k = kf * np.sqrt(np.arange(ns, dtype=np.float64))
    p = amp * (1.0 + k / 0.02) ** -1.5
    beta = 0.5
    pl = [p * (1 + 2 * beta / 3 + beta * beta / 5), p * (4 * beta / 3 + 4 * beta * beta / 7), p * 8 * beta * beta / 35]
    return np.stack(pl[:nell])


# ------------------------------------------------------------------------------------------------ the solver


@pytest.mark.parametrize("grid", [(16, 16, 16), (8, 8, 256)])   # 8 x 8 x 256: the 256-point C2R pass
def test_fixed_iterations_match_the_oracle_fp64(pkg, grid):
    box = 16.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 2.5, 4.5, 6.5])
    n, n2 = _random_mask(grid, 1, 0.4)
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="fp64")
    ns = pb.max_shell() + 1
    pfid = _kaiser_table(ns, kf, amp=5.0)
    Pk = optimal.fiducial_grid(pfid, grid)
    v = np.random.Generator(np.random.PCG64(2)).standard_normal(grid).astype(np.float32)
    for iters in (1, 3, 7):
        pb.set_optimal(_dev(n), pfid, _dev(n2), max_iter=iters, tol=0.0)
        x, it, _ = pb.sinv_optimal(_dev(v))
        assert it == iters
        sig = optimal.precond_sigma(n, n2)
        b = np.where(n > 0, v.astype(np.float64) / np.where(n > 0, n, 1).astype(np.float64), 0.0)
        ref, it_ref, _ = optimal.pcg(b,
                                     lambda u: optimal.apply_a(u, n, n2, Pk),
                                     lambda r: optimal.apply_precond(r, n, Pk, sig), iters, 0.0)
        assert it_ref == iters
        err = np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err < 1e-10, (iters, err)
    pb.close()


@pytest.mark.parametrize("transpose", [False, True])
def test_converged_solve_matches_dense_fp64(pkg, transpose):
    grid, box = (16, 16, 16), 16.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 2.5, 4.5, 6.5])
    n, n2 = _random_mask(grid, 3, 0.4)
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="fp64")
    pfid = _kaiser_table(pb.max_shell() + 1, kf, amp=5.0)
    Pk = optimal.fiducial_grid(pfid, grid)
    pb.set_optimal(_dev(n), pfid, _dev(n2), max_iter=400, tol=1e-12)
    v = np.random.Generator(np.random.PCG64(4)).standard_normal(grid).astype(np.float32)
    x, it, rel = pb.sinv_optimal(_dev(v), transpose=transpose)
    assert rel <= 1e-12 and it < 400
    A, sel = optimal.dense_operator(n, n2, Pk)
    nn = n.astype(np.float64)
    inv_n = np.where(nn > 0, 1.0 / np.where(nn > 0, nn, 1.0), 0.0)
    want = inv_n * optimal.g_dense(A, sel, v) if transpose else optimal.g_dense(A, sel, v * inv_n)
    err = np.max(np.abs(x.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < 1e-9, err
    assert np.all(x.cpu().numpy()[n == 0] == 0.0)
    pb.close()


def test_fp32_solve_on_a_survey_mask(pkg):
    grid, box = (32, 32, 32), 600.0
    kf = binning.kf_of(box)
    edges = kf * np.arange(0.5, 12.0, 1.0)
    n = _survey(grid, box, 5)
    pb = pkg.PolyBin(grid, box, edges, lmax=4, prec="fp32")
    pfid = _kaiser_table(pb.max_shell() + 1, kf)
    Pk = optimal.fiducial_grid(pfid, grid)
    pb.set_optimal(_dev(n), pfid, None, max_iter=300, tol=1e-6)
    d = (n * synth.lognormal_field(grid, (box,) * 3, 6, kaiser_beta=0.5)).astype(np.float32)
    x, it, rel = pb.sinv_optimal(_dev(d))
    b = np.where(n > 0, d.astype(np.float64) / np.where(n > 0, n, 1).astype(np.float64), 0.0)
    xs = x.cpu().numpy().astype(np.float64)
    r_true = b - optimal.apply_a(xs, n, n, Pk)
    res = np.sqrt(np.sum(r_true ** 2) / np.sum(b ** 2))
    ref, it_ref, _ = optimal.g_pcg(b, n, n, Pk, tol=1e-12)
    err = np.max(np.abs(xs - ref)) / np.max(np.abs(ref))
    assert res < 2e-5, res
    assert err < 2e-4, err
    assert abs(it - optimal.g_pcg(b, n, n, Pk, tol=1e-6)[1]) <= 2
    pb.close()


def test_uniform_density_converges_in_one_iteration(pkg):
    """n = n2 = nbar everywhere: the preconditioner is the exact inverse (eq. Sinv-ideal), one step suffices and
    S^-1 v = (1/nbar) IFT[FT[v] / (P + 1/nbar)]."""
    grid, box = (64, 64, 64), 1000.0
    kf = binning.kf_of(box)
    edges = kf * np.arange(0.5, 20.0, 2.0)
    nbar = 3.0e-4
    n = np.full(grid, nbar, dtype=np.float32)
    pb = pkg.PolyBin(grid, box, edges, lmax=4, prec="fp64")
    pfid = _kaiser_table(pb.max_shell() + 1, kf)
    Pk = optimal.fiducial_grid(pfid, grid)
    pb.set_optimal(_dev(n), pfid, None, max_iter=50, tol=1e-10)
    v = np.random.Generator(np.random.PCG64(8)).standard_normal(grid).astype(np.float32)
    x, it, rel = pb.sinv_optimal(_dev(v))
    assert it == 1 and rel < 1e-10
    nb64 = float(np.float32(nbar))
    want = np.fft.ifftn(np.fft.fftn(v.astype(np.float64)) / (Pk + 1.0 / nb64)).real / nb64
    assert np.max(np.abs(x.cpu().numpy() - want)) < 1e-10 * np.max(np.abs(want))
    pb.close()


def test_errors(pkg):
    grid, box = (16, 16, 16), 16.0
    kf = binning.kf_of(box)
    pb = pkg.PolyBin(grid, box, kf * np.array([0.5, 2.5, 4.5]), prec="fp32")
    v = torch.zeros(grid, dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.PolybinError):
        pb.sinv_optimal(v)                      # not configured
    n = torch.ones(grid, dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.PolybinError):
        pb.set_optimal(n, np.ones((1, pb.max_shell() + 2)))   # table beyond the binned shells
    with pytest.raises(pkg.PolybinError):
        pb.set_optimal(torch.zeros_like(n), np.ones((1, 3)))  # empty mask
    pb.set_optimal(n, np.ones((1, 3)), max_iter=5)
    x, it, rel = pb.sinv_optimal(v)                            # zero right-hand side: zero solution, no iteration
    assert it == 0 and rel == 0.0 and float(x.abs().max()) == 0.0
    pb.close()


# ------------------------------------------------------------------------------------------------ the P estimator


@pytest.fixture(scope="module")
def survey16():
    grid, box = (16, 16, 16), 400.0
    kf = binning.kf_of(box)
    edges = kf * np.array([0.5, 1.5, 2.5, 3.5, 4.5])
    n = _survey(grid, box, 9)
    d = (n * synth.lognormal_field(grid, (box,) * 3, 10, kaiser_beta=0.5)).astype(np.float32)
    return grid, box, kf, edges, n, d


def test_fisher_draw_and_numerator_fp64(pkg, survey16):
    grid, box, kf, edges, n, d = survey16
    nb = len(edges) - 1
    ells = [0, 2]
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="fp64")
    pfid = _kaiser_table(pb.max_shell() + 1, kf)
    Pk = optimal.fiducial_grid(pfid, grid)
    pb.set_optimal(_dev(n), pfid, None, max_iter=400, tol=1e-12)
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    sinv, sinv_t = optimal.optimal_weighting(n, n, Pk, tol=1e-13)
    Fd = pb.fisher_draws(_dev(n), None, 77, pkg.FISHER_PK_OPT, 0, 1)[0]
    a = unwindowed.draw(grid, 77, 0, unwindowed.STREAM_P, np.float64)
    R = optimal.pk_fisher_draw_general(a, n, sinv, sinv_t, bins, mu2, nb, ells)
    dg = np.sqrt(np.abs(np.diag(R)))
    assert np.max(np.abs(Fd - R) / np.outer(dg, dg)) < 1e-8
    _, pnum = pb.pk_unwindowed_opt(_dev(d), with_estimate=False)
    ref = optimal.pk_numerator_general(d, sinv, bins, mu2, nb, ells).ravel()
    assert np.max(np.abs(pnum - ref)) < 1e-8 * np.max(np.abs(ref))
    pb.close()


def test_unwindowed_opt_end_to_end_fp32(pkg, survey16):
    grid, box, kf, edges, n, d = survey16
    nb = len(edges) - 1
    ells = [0, 2, 4]
    pb = pkg.PolyBin(grid, box, edges, lmax=4, prec="fp32")
    pfid = _kaiser_table(pb.max_shell() + 1, kf)
    Pk = optimal.fiducial_grid(pfid, grid)
    pb.set_optimal(_dev(n), pfid, None, max_iter=300, tol=1e-6)
    with pytest.raises(pkg.PolybinError):
        pb.pk_unwindowed_opt(_dev(d))           # no Fisher matrix yet
    F, _ = pb.fisher(_dev(n), None, 2, 5, pkg.FISHER_PK_OPT)
    p, pnum = pb.pk_unwindowed_opt(_dev(d))
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    Fref = optimal.pk_fisher_opt(n, n, n, Pk, bins, mu2, nb, ells, 5, 2, unwindowed.draw, unwindowed.STREAM_P,
                                 np.float32)
    dg = np.sqrt(np.abs(np.diag(Fref)))
    assert np.max(np.abs(F - Fref) / np.outer(dg, dg)) < 2e-4
    sinv = optimal.optimal_weighting(n, n, Pk)[0]
    pref = optimal.pk_numerator_general(d, sinv, bins, mu2, nb, ells).ravel()
    assert np.max(np.abs(pnum - pref)) < 2e-4 * np.max(np.abs(pref))
    scale = box ** 3 / d.size
    same = unwindowed.solve(F, pnum) * scale
    assert np.max(np.abs(p - same)) / np.max(np.abs(same)) < 1e-9
    # a new configuration retires the Fisher matrix computed with the old one
    pb.set_optimal(_dev(n), 2.0 * pfid, None, max_iter=300, tol=1e-6)
    with pytest.raises(pkg.PolybinError):
        pb.pk_unwindowed_opt(_dev(d))
    pb.close()
