"""Full-size parity on sampled outputs, in the launch configuration the benchmark times.

* 512^3 lognormal + Kaiser field, 30 bins to 0.3 h/Mpc, split-TF32 path (the benchmark default): every N_abc of a
  sample of triplets equals the oracle's exactly; B_abc of the sample within 1e-6 relative wherever
  kappa <= 10 and 1e-6 of sum|g g g| everywhere; P_0, P_2 of every bin within 1e-6 of P_0.
* 256^3 masked workload (shell with holes, FKP weights, 24 P bins x ell 0,2,4, 16 B bins): the full P Fisher term
  of one draw, and a sampled block of the B Fisher term of one draw pair, within 1e-6 of sqrt(F_aa F_bb).
The oracle computes only the maps these samples need (FP64, all host cores).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import _fft, binning, ideal, unwindowed
from paper_2404_07249_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    pkg.load()
    return pkg


def test_config3_sampled_bispectrum_and_pk(pkg):
    w = synth.WORKLOADS[3]
    grid, box, edges = w.grid, w.box, w.bk_edges
    field = synth.workload_field(3, 0)
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="split")
    B, P = pb.bk_pk(torch.from_numpy(field).cuda())
    abc, nabc = pb.triplets()
    pb.close()
    B, P = B[0], P[0]
    trip = [tuple(t) for t in abc.tolist()]
    N = field.size
    vol = box ** 3
    # sample: first, last, all-equal, two-equal and a few spread out
    pick = sorted({0, len(trip) - 1, trip.index((0, 0, 0)) if (0, 0, 0) in trip else 0,
                   len(trip) // 7, len(trip) // 3, len(trip) // 2, (2 * len(trip)) // 3})
    D = ideal.forward(field)
    bins = binning.bin_grid(grid, box, edges).astype(np.int16)
    need = sorted({b for i in pick for b in trip[i]})
    g, t = {}, {}
    for b in need:
        sel = bins == b
        g[b] = _fft.ifftn(np.where(sel, D, 0.0)).real
        t[b] = _fft.ifftn(sel.astype(np.complex128)).real
    for i in pick:
        a, b, c = trip[i]
        S = np.sum(g[a] * g[b] * g[c])
        T = np.sum(t[a] * t[b] * t[c])
        absS = np.sum(np.abs(g[a] * g[b] * g[c]))
        assert np.rint(N * N * T) == nabc[i], (trip[i], N * N * T, nabc[i])
        Bref = vol * vol / float(N) ** 3 * S / T
        e_norm = abs(B[i] - Bref) / (vol * vol / float(N) ** 3 * absS / T)
        assert e_norm < 1e-6, (trip[i], e_norm)
        if absS / abs(S) <= 10:
            assert abs(B[i] - Bref) / abs(Bref) < 1e-6, (trip[i], B[i], Bref)
    del g, t
    # P_ell over every bin (ell = 0, 2)
    pw = np.abs(D) ** 2
    del D
    mu2 = binning.mu2_grid(grid)
    counts = np.bincount(bins[bins >= 0].ravel(), minlength=len(edges) - 1).astype(float)
    sel = bins >= 0
    P0 = vol / float(N) ** 2 * np.bincount(bins[sel], weights=pw[sel], minlength=len(edges) - 1) / counts
    L2 = binning.legendre(2, mu2)
    P2 = 5 * vol / float(N) ** 2 * np.bincount(bins[sel], weights=(L2 * pw)[sel], minlength=len(edges) - 1) / counts
    ok = counts > 0
    assert np.max(np.abs(P[0][ok] - P0[ok]) / np.abs(P0[ok])) < 1e-6
    assert np.max(np.abs(P[1][ok] - P2[ok]) / np.abs(P0[ok])) < 5e-6


def test_config5_fisher_terms(pkg):
    wl = synth.WORKLOADS[5]
    grid, box = wl.grid, wl.box
    n = synth.survey_mask(grid, (box,) * 3, 5000).astype(np.float32)
    wfk = unwindowed.fkp_weight(n, wl.extra["P0"]).astype(np.float32)
    seed = 77
    nd, wd = torch.from_numpy(n).cuda(), torch.from_numpy(wfk).cuda()
    # --- P Fisher, full matrix of draw 0
    pbp = pkg.PolyBin(grid, box, wl.pk_edges, lmax=4, prec="split")
    Fp = pbp.fisher_draws(nd, wd, seed, 0, 0, 1)[0]
    pbp.close()
    nb = len(wl.pk_edges) - 1
    binsp = binning.bin_grid(grid, box, wl.pk_edges)
    mu2 = binning.mu2_grid(grid)
    a = unwindowed.draw(grid, seed, 0, unwindowed.STREAM_P, np.float32)
    Rp = unwindowed.pk_fisher_draw(a, n, wfk, binsp, mu2, nb, [0, 2, 4])
    dg = np.sqrt(np.abs(np.diag(Rp)))
    assert np.max(np.abs(Fp - Rp) / np.outer(dg, dg)) < 1e-6
    # --- B Fisher, sampled block of draw pair 0
    pbb = pkg.PolyBin(grid, box, wl.bk_edges, prec="split")
    abc, _ = pbb.triplets()
    Fb = pbb.fisher_draws(nd, wd, seed, 1, 0, 1)[0]
    pbb.close()
    trip = [tuple(t) for t in abc.tolist()]
    idx = sorted({0, 1, len(trip) // 3, len(trip) // 2, len(trip) - 1})
    sub = [trip[i] for i in idx]
    nbb = len(wl.bk_edges) - 1
    binsb = binning.bin_grid(grid, box, wl.bk_edges)
    a1 = unwindowed.draw(grid, seed, 0, unwindowed.STREAM_B1, np.float32)
    a2 = unwindowed.draw(grid, seed, 0, unwindowed.STREAM_B2, np.float32)
    Rb = unwindowed.bk_fisher_draw(a1, a2, n, wfk, binsb, nbb, sub)
    G = Fb[np.ix_(idx, idx)]
    dg = np.sqrt(np.abs(np.diag(Rb)))
    assert np.max(np.abs(G - Rb) / np.outer(dg, dg)) < 1e-6
