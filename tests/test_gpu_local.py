"""GPU parity of the local (Yamamoto) line-of-sight power spectrum against the FP64 oracle (oracle/local.py), through
the C-ABI: numerator (eq. pk-num-fft), one Monte Carlo Fisher term (eq. fish-from-Q with eq. Q-alpha-local), the
end-to-end unwindowed estimate, and the observer bookkeeping; and the ideal bispectrum multipoles with the local
line of sight (eq. g-ell-def with its Ybar_lm expansion).

Setup: the 32^3 masked box of the unwindowed tests (shell with holes, FKP weights), an observer off the box centre,
P bins 0, 2, .., 10 k_F, ell = 0, 2, 4.  Tolerances as for the global line of sight: numerators within 1e-6 of the
largest |value|, Fisher terms within 1e-6 of sqrt(F_aa F_bb), the FP64 solve within 1e-9 of LAPACK on the same F.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, local, unwindowed
from paper_2404_07249_gb300 import synth

from bk_criterion import bk_errors, check, report

pytestmark = pytest.mark.gpu

GRID = (32, 32, 32)
BOX = 600.0
KF = binning.kf_of(BOX)
PK_EDGES = KF * np.array([0.0, 2.0, 4.0, 6.0, 8.0, 10.0])
OBS = (23.0, -41.0, 17.0)
SEED = 31337
ELLS = [0, 2, 4]


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
    w = unwindowed.fkp_weight(n, 1.0e4).astype(np.float32)
    d = (n * synth.lognormal_field(GRID, (BOX,) * 3, 12, kaiser_beta=0.5)).astype(np.float32)
    bins = binning.bin_grid(GRID, BOX, PK_EDGES)
    xhat = local.position_units(GRID, BOX, OBS)
    khat = local.mode_units(GRID)
    return n, w, d, bins, xhat, khat


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _fisher_close(G, R):
    dg = np.sqrt(np.abs(np.diag(R)))
    return np.max(np.abs(G - R) / np.outer(dg, dg))


def test_local_numerator(pkg, fields):
    n, w, d, bins, xhat, khat = fields
    nb = len(PK_EDGES) - 1
    pb = pkg.PolyBin(GRID, BOX, PK_EDGES, lmax=4, prec="fp32")
    pb.set_observer(OBS)
    _, pnum = pb.pk_unwindowed_local(_dev(d), _dev(w), with_estimate=False)
    ref = local.pk_numerator_local(d, w, bins, nb, ELLS, xhat, khat).ravel()
    assert np.max(np.abs(pnum - ref)) < 1e-6 * np.max(np.abs(ref))
    # the local numerator is not the global one (the observer matters)
    _, pglob = pb.pk_unwindowed(_dev(d), _dev(w), with_estimate=False)
    assert np.max(np.abs(pnum[nb:] - pglob[nb:])) > 1e-3 * np.max(np.abs(pglob[nb:]))
    pb.close()


def test_local_fisher_draw(pkg, fields):
    n, w, d, bins, xhat, khat = fields
    nb = len(PK_EDGES) - 1
    pb = pkg.PolyBin(GRID, BOX, PK_EDGES, lmax=4, prec="fp32")
    pb.set_observer(OBS)
    Fd = pb.fisher_draws(_dev(n), _dev(w), SEED, pkg.FISHER_PK_LOCAL, 0, 1)[0]
    a = unwindowed.draw(GRID, SEED, 0, unwindowed.STREAM_P, np.float32)
    R = local.pk_fisher_draw_local(a, n, w, bins, nb, ELLS, xhat, khat)
    assert _fisher_close(Fd, R) < 1e-6
    pb.close()


def test_local_unwindowed_end_to_end_and_observer(pkg, fields):
    n, w, d, bins, xhat, khat = fields
    nb = len(PK_EDGES) - 1
    pb = pkg.PolyBin(GRID, BOX, PK_EDGES, lmax=4, prec="fp32")
    pb.set_observer(OBS)
    F, _ = pb.fisher(_dev(n), _dev(w), 2, SEED, pkg.FISHER_PK_LOCAL)
    p, pnum = pb.pk_unwindowed_local(_dev(d), _dev(w))
    scale = BOX ** 3 / d.size
    same = unwindowed.solve(F, pnum) * scale
    assert np.max(np.abs(p - same)) / np.max(np.abs(same)) < 1e-9
    Fref = local.pk_fisher_local(n, w, bins, nb, ELLS, xhat, khat, SEED, 2, unwindowed.draw, unwindowed.STREAM_P,
                                 np.float32)
    assert _fisher_close(F, Fref) < 1e-6
    ref = unwindowed.solve(Fref, local.pk_numerator_local(d, w, bins, nb, ELLS, xhat, khat).ravel()) * scale
    err = np.max(np.abs(p - ref)) / np.max(np.abs(ref))
    assert err < 3e-6 * np.linalg.cond(Fref), (err, np.linalg.cond(Fref))
    # a new observer discards the local Fisher matrix
    pb.set_observer((0.0, 0.0, 0.0))
    with pytest.raises(pkg.PolybinError):
        pb.pk_unwindowed_local(_dev(d), _dev(w))
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "split", "fp64"])
def test_bk_multipoles_local(pkg, prec):
    """Bispectrum multipoles ell = 0, 2, 4 with the local line of sight (eq. g-ell-def with Ybar_lm) against the oracle,
    triplet by triplet with the criterion of tests/bk_criterion.py (kappa from sum_x |g_a g_b g_{c,ell}|); the
    monopole equals the global one bit for bit."""
    from oracle import ideal
    grid, box = (48, 48, 48), 900.0
    edges = binning.kf_of(box) * (0.5 + 2.0 * np.arange(7))
    obs = (120.0, -310.0, 205.0)
    f = synth.lognormal_field(grid, (box,) * 3, 77, kaiser_beta=0.5).astype(np.float32)
    xhat = local.position_units(grid, box, obs)
    khat = local.mode_units(grid)
    ref = local.bk_ideal_multipoles_local(f, box, edges, 4, xhat, khat)
    pb = pkg.PolyBin(grid, box, edges, prec=prec)
    pb.set_observer(obs)
    Bl = pb.bk_multipoles_local(_dev(f), 4)[0]
    abc, _ = pb.triplets()
    assert [tuple(t) for t in abc.tolist()] == ref["triplets"]
    assert np.array_equal(Bl[0], pb.bk_ideal(_dev(f))[0])
    tol = {"fp32": (1e-6, 1e-6, 10.0), "split": (1e-6, 1e-6, 10.0), "fp64": (1e-12, 1e-11, 1e3)}[prec]
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    G = ideal.shell_maps(ideal.forward(f), bins, nb).reshape(nb, -1)
    for il, ell in enumerate(ref["ells"]):
        GL = G if ell == 0 else ideal.shell_maps(ref["H"][ell], bins, nb).reshape(nb, -1)
        absS = np.array([np.dot(np.abs(G[a] * G[b]), np.abs(GL[c])) for a, b, c in ref["triplets"]])
        e_rel, e_norm, kappa = bk_errors(Bl[il], ref["B"][il], ref["S"][il], absS)
        s = check(ref["triplets"], e_rel, e_norm, kappa, norm_tol=tol[0], rel_tol=tol[1], kappa_max=tol[2],
                  label=f"local {prec} ell {ell}")
        print(report(s, f"local multipole ell={ell} {prec}"))
    # the local quadrupole differs from the global one (the observer matters)
    glob = pb.bk_multipoles(_dev(f), 4)[0]
    assert np.max(np.abs(Bl[1] - glob[1])) > 1e-3 * np.max(np.abs(glob[1]))
    pb.close()
