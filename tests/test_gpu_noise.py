"""GPU parity of the Poisson shot-noise bias of the P numerator (first line of eq. fish-from-Q, global line of sight)
against the FP64 oracle (oracle/noise.py), through the C-ABI.

Same Monte Carlo maps on both sides (stream 3, FP32-rounded for FP32 contexts), so the averages agree element by
element: within 1e-6 of the largest |value| with the FKP weighting (FP32 transforms), within 1e-4 with the optimal
weighting solved to a relative residual of 1e-6 in FP32 (two solves per map; kappa(A) below 1e2 on this mask).
The closed form of a diagonal weighting is the expectation of the Monte Carlo terms: the mean of 64 single-map
estimates lies within 5 of its standard errors (estimated from the same 64 values) of it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, noise, optimal, unwindowed
from paper_2404_07249_gb300 import synth

pytestmark = pytest.mark.gpu

GRID = (32, 32, 32)
BOX = 600.0
EDGES = binning.kf_of(BOX) * np.array([0.0, 2.0, 4.0, 6.0, 8.0, 10.0])


@pytest.fixture(scope="module")
def pkg():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def fields():
    geom = synth.SurveyGeometry(r_min=60.0, r_max=290.0, n_holes=4, hole_radius=30.0, n0=3.0e-4, r0=180.0, s2=2.0e4)
    n = synth.survey_mask(GRID, (BOX,) * 3, 5, geom).astype(np.float32)
    n2 = (n * 1.3).astype(np.float32)
    w = unwindowed.fkp_weight(n, 1.0e4).astype(np.float32)
    return n, n2, w, binning.bin_grid(GRID, BOX, EDGES), binning.mu2_grid(GRID)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_pk_bias_fkp(pkg, fields):
    n, n2, w, bins, mu2 = fields
    nb, ells = len(EDGES) - 1, [0, 2, 4]
    vcell = BOX ** 3 / n.size
    pb = pkg.PolyBin(GRID, BOX, EDGES, lmax=4, prec="fp32")
    got = pb.pk_bias(_dev(n2), _dev(w), pkg.FISHER_PK, n_mc=4, seed=11)
    ref = noise.pk_bias(n2, vcell, lambda v: w.astype(np.float64) * v, bins, mu2, nb, ells, 11, 4, unwindowed.draw, 3,
                        np.float32).ravel()
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    # 64 independent single-map estimates: their mean is within 5 standard errors of the closed form
    per = np.stack([pb.pk_bias(_dev(n2), _dev(w), pkg.FISHER_PK, n_mc=1, seed=100 + i) for i in range(64)])
    closed = noise.pk_bias_diagonal(w, n2, vcell, bins, mu2, nb, ells).ravel()
    se = per.std(axis=0, ddof=1) / np.sqrt(len(per))
    assert np.all(np.abs(per.mean(axis=0) - closed) < 5 * se + 1e-6 * np.max(np.abs(closed)))
    pb.close()


def test_pk_bias_subtracted_by_the_estimate(pkg, fields):
    n, n2, w, bins, mu2 = fields
    pb = pkg.PolyBin(GRID, BOX, EDGES, lmax=4, prec="fp32")
    d = (n * synth.lognormal_field(GRID, (BOX,) * 3, 12, kaiser_beta=0.5)).astype(np.float32)
    F, _ = pb.fisher(_dev(n), _dev(w), 2, 1, pkg.FISHER_PK)
    p0, pnum = pb.pk_unwindowed(_dev(d), _dev(w))
    bias = pb.pk_bias(_dev(n2), _dev(w), pkg.FISHER_PK, n_mc=2, seed=3)
    p1, pnum1 = pb.pk_unwindowed(_dev(d), _dev(w))
    scale = BOX ** 3 / d.size
    assert np.array_equal(pnum, pnum1)
    want = unwindowed.solve(F, pnum - bias) * scale
    assert np.max(np.abs(p1 - want)) < 1e-9 * np.max(np.abs(want))
    pb.pk_bias(None, None, pkg.FISHER_PK, n_mc=0)
    p2, _ = pb.pk_unwindowed(_dev(d), _dev(w))
    assert np.array_equal(p2, p0)
    pb.close()


def test_pk_bias_optimal(pkg, fields):
    n, n2, w, bins, mu2 = fields
    nb, ells = len(EDGES) - 1, [0, 2, 4]
    vcell = BOX ** 3 / n.size
    pb = pkg.PolyBin(GRID, BOX, EDGES, lmax=4, prec="fp32")
    kf = binning.kf_of(BOX)
    pfid = synth.power_law(kf * np.sqrt(np.arange(pb.max_shell() + 1, dtype=np.float64)))[None, :]
    pb.set_optimal(_dev(n), pfid, _dev(n2), max_iter=300, tol=1e-6)
    got = pb.pk_bias(_dev(n2), None, pkg.FISHER_PK_OPT, n_mc=2, seed=21)
    Pk = optimal.fiducial_grid(pfid, GRID)
    sinv = lambda v: optimal.sinv_apply(v, n, n2, Pk)  # noqa: E731
    ref = noise.pk_bias(n2, vcell, sinv, bins, mu2, nb, ells, 21, 2, unwindowed.draw, 3, np.float32).ravel()
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref))
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "split"])
def test_bk_bias_and_estimate(pkg, fields, prec):
    """B shot noise: same Monte Carlo pairs (streams 4, 5) as the oracle, within 2e-5 of the largest |value| (FP32 maps
    and sums of six assignments with cancelling signs), and the estimate F^-1 (b_num - b_bias)."""
    n, n2, w, _, _ = fields
    edges = binning.kf_of(BOX) * np.array([1.0, 3.0, 5.0, 7.0])
    nb = len(edges) - 1
    vcell = BOX ** 3 / n.size
    d = (np.random.Generator(np.random.PCG64(4)).poisson(n.astype(np.float64) * vcell) / vcell - n).astype(np.float32)
    pb = pkg.PolyBin(GRID, BOX, edges, prec=prec)
    trip = [tuple(t) for t in pb.triplets()[0].tolist()]
    got = pb.bk_bias(_dev(n), _dev(d), _dev(d), _dev(w), n_mc=2, seed=17)
    bins = binning.bin_grid(GRID, BOX, edges)
    ref = noise.bk_bias(d, n, d, vcell, lambda v: w.astype(np.float64) * v, bins, nb, trip, 17, 2, unwindowed.draw,
                        (4, 5), np.float32)
    assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref)), np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    F, _ = pb.fisher(_dev(n), _dev(w), 1, 2, pkg.FISHER_BK)
    b, bnum, bias = pb.bk_unwindowed_shot(_dev(d), _dev(w), _dev(n), _dev(d), n_mc=2, seed=17)
    assert np.array_equal(bias, got)
    want = unwindowed.solve(F, bnum - bias) * (BOX ** 3 / n.size) ** 2
    assert np.max(np.abs(b - want)) < 1e-9 * np.max(np.abs(want))
    pb.close()
