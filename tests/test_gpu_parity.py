"""GPU parity: every step of the CUDA path against the FP64 oracle, element by element, through the C-ABI.

Tolerances (float32 path): FFT outputs and shell maps within 2e-6 of the L2 norm (relative L2 error; FP32
rounding of ~log2 N radix passes); contraction outputs within 1e-6 of sum_x |g_j g_k h_i| (the
cancellation-aware error); bispectrum: every triplet within e_norm 1e-6, every triplet with kappa =
sum|ggg| / |sum ggg| <= 10 within 1e-6 relative, and the triplets above 1e-6 relative (all with kappa > 10: an
FP32 relative error eps in the maps moves the estimate by up to ~3 kappa eps relative) listed by name
(tests/bk_criterion.py); P_ell within 1e-6 relative; N_abc bit-exact.  FP64 path: 1e-12 in the same metrics.
The bispectrum maps and triplet sums run on the alias-free contraction grid (polybin_contraction_grid), the oracle
on the data grid.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, ideal
from paper_2404_07249_gb300 import synth

from bk_criterion import bk_errors, check, report

pytestmark = pytest.mark.gpu

# kappa_max: e_rel is asserted for triplets with kappa * (FFT noise of the path) below the target, i.e. kappa <= 10
# for the FP32 FFTs (relative noise ~1e-7) and kappa <= 1e3 for FP64; e_norm is asserted for every triplet.
TOL = {"fp32": dict(l2=2e-6, norm=1e-6, rel=1e-6, kappa_max=10.0),
       "split": dict(l2=2e-6, norm=1e-6, rel=1e-6, kappa_max=10.0),
       "fp64": dict(l2=1e-12, norm=1e-12, rel=1e-11, kappa_max=1e3)}


@pytest.fixture(scope="module")
def pkg():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    pkg.load()
    return pkg


def _kf(box):
    return binning.kf_of(box)


CASES = [
    # (grid, box, edges in units of k_F, field)
    ((64, 64, 64), 1000.0, 1.0 + 2.0 * np.arange(9), "grf"),          # config-1 bispectrum bins
    ((48, 48, 48), 900.0, 0.5 + 2.0 * np.arange(7), "lognormal"),      # radix 3
    ((40, 40, 40), 700.0, 1.0 + 1.5 * np.arange(8), "lognormal"),      # radix 5
    ((32, 48, 40), 800.0, 1.0 + 2.0 * np.arange(6), "lognormal"),      # non-cubic grid, cubic box
    ((16, 16, 16), 500.0, np.array([0.5, 3.0, 6.0, 9.5, 14.0]), "lognormal"),  # bins beyond Nyquist (full axes)
    ((16, 8, 512), 2000.0, 1.0 + 6.0 * np.arange(8), "lognormal"),    # 512-point z lines, few z modes
    ((8, 4, 512), 2000.0, 1.0 + 40.0 * np.arange(8), "lognormal"),    # 512-point z lines up to the z Nyquist
    ((8, 6, 288), 2000.0, 1.0 + 20.0 * np.arange(8), "lognormal"),    # 288-point z lines (register-resident pass)
    ((8, 8, 512), 2000.0, 0.5 + 11.9375 * np.arange(9), "lognormal"), # m = 95: contraction grid 8 x 8 x 288
    ((16, 8, 256), 2000.0, 1.0 + 6.0 * np.arange(8), "lognormal"),    # 256-point z lines (register-resident passes)
    ((6, 10, 256), 1500.0, 1.0 + 4.0 * np.arange(7), "lognormal"),    # 256-point lines, radix-3 and radix-5 x, y
    ((8, 8, 256), 2000.0, 0.5 + 11.25 * np.arange(9), "lognormal"),   # m = 90: shells on 256-point z lines
    ((20, 10, 100), 1500.0, 1.0 + 2.0 * np.arange(8), "lognormal"),   # compile-time 100-point passes (z)
    ((100, 100, 20), 1500.0, 1.0 + 2.0 * np.arange(8), "lognormal"),  # compile-time 100-point column passes
    ((6, 288, 8), 2000.0, 1.0 + 20.0 * np.arange(8), "lognormal"),    # 288-point y columns up to |n_y| = 141
    ((4, 288, 64), 2000.0, 1.0 + 4.0 * np.arange(8), "lognormal"),    # 288-point y columns, 29 kz columns (2 CTAs)
    ((288, 6, 8), 2000.0, 1.0 + 20.0 * np.arange(8), "lognormal"),    # 288-point x lines with the shell filter
]


def _field(grid, box, kind, seed):
    if kind == "grf":
        return synth.gaussian_field(grid, (box,) * 3, seed).astype(np.float32)
    return synth.lognormal_field(grid, (box,) * 3, seed).astype(np.float32)


def _oracle_box(D, dims, lo):
    ix = (np.arange(dims[0]) + lo[0]) % D.shape[0]
    iy = (np.arange(dims[1]) + lo[1]) % D.shape[1]
    iz = np.arange(dims[2]) + lo[2]
    return D[np.ix_(ix, iy, iz)]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_and_shell_maps(pkg, case, prec):
    grid, box, ek, kind = CASES[case]
    edges = _kf(box) * ek
    f = _field(grid, box, kind, 10 + case)
    pb = pkg.PolyBin(grid, box, edges, prec=prec)
    d = torch.from_numpy(f).cuda()
    spec = pb.forward(d)
    dims, lo = pb.spectrum_shape()
    D = ideal.forward(f)
    ref = _oracle_box(D, dims, lo)
    got = spec.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < TOL[prec]["l2"], f"forward rel L2 {err}"
    g = pb.shell_maps(spec).cpu().numpy().astype(np.float64)
    bins = binning.bin_grid(grid, box, edges)
    gref = ideal.shell_maps(D, bins, len(edges) - 1)
    for b in range(len(edges) - 1):
        nrm = np.linalg.norm(gref[b])
        if nrm == 0:
            assert np.max(np.abs(g[b])) == 0.0
            continue
        e = np.linalg.norm(g[b] - gref[b]) / nrm
        assert e < TOL[prec]["l2"], f"shell map {b} rel L2 {e}"
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "split", "fp64"])
@pytest.mark.parametrize("nh_same", [True, False])
@pytest.mark.parametrize("shape", [(9, 5, (40, 48, 32)), (30, 30, (24, 20, 18)), (31, 32, (16, 12, 10)),
                                   (2, 1, (6, 4, 2))])
def test_contraction(pkg, prec, nh_same, shape):
    ng, nh, grid = shape
    box = 800.0
    rng = np.random.Generator(np.random.PCG64(7))
    dt = np.float64 if prec == "fp64" else np.float32
    g = rng.standard_normal((ng,) + grid).astype(dt)
    g[min(3, ng - 1)] *= 1e3        # dynamic range between maps
    h = rng.standard_normal((nh,) + grid).astype(dt)
    pb = pkg.PolyBin(grid, box, _kf(box) * np.array([1.0, 2.0]), prec=prec)
    tg = torch.from_numpy(g).cuda()
    if nh_same:
        M = pb.contract(tg)
        hh = g
    else:
        M = pb.contract(tg, torch.from_numpy(h).cuda())
        hh = h
    G = g.astype(np.float64).reshape(ng, -1)
    H = hh.astype(np.float64).reshape(hh.shape[0], -1)
    pairs = pkg.pair_list(ng)
    for p, (j, k) in enumerate(pairs):
        ref = (G[j] * G[k]) @ H.T
        scale = np.abs(G[j] * G[k]) @ np.abs(H).T
        e = np.abs(M[p] - ref) / scale
        assert np.max(e) < TOL[prec]["norm"], (p, np.max(e))
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "split", "fp64"])
@pytest.mark.parametrize("case", [0, 1, 3, 4, 8])
def test_bk_ideal_and_nabc(pkg, case, prec):
    grid, box, ek, kind = CASES[case]
    edges = _kf(box) * ek
    f = _field(grid, box, kind, 20 + case)
    ref = ideal.bk_ideal(f, box, edges)
    pb = pkg.PolyBin(grid, box, edges, prec=prec)
    abc, nabc = pb.triplets()
    assert [tuple(t) for t in abc.tolist()] == ref["triplets"]
    assert np.array_equal(nabc, ref["N_abc"])
    B = pb.bk_ideal(torch.from_numpy(f).cuda())[0]
    if prec == "split":
        assert pb.last_path() == pkg.PATH_TENSOR_SPLIT_TF32X3
    bins = binning.bin_grid(grid, box, edges)
    g = ideal.shell_maps(ideal.forward(f), bins, len(edges) - 1)
    G = g.reshape(g.shape[0], -1)
    absS = np.array([np.sum(np.abs(G[a] * G[b] * G[c])) for a, b, c in ref["triplets"]])
    e_rel, e_norm, kappa = bk_errors(B, ref["B"], ref["S"], absS)
    s = check(ref["triplets"], e_rel, e_norm, kappa, norm_tol=TOL[prec]["norm"], rel_tol=TOL[prec]["rel"],
              kappa_max=TOL[prec]["kappa_max"], label=f"case {case} {prec}")
    print(report(s, f"case {case} {prec} grid {grid} contraction grid {pb.contraction_grid()}"))
    # host input gives the same numbers as device input
    B2 = pb.bk_ideal(f)[0]
    assert np.array_equal(B, B2)
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pk_multipoles(pkg, prec):
    w = synth.WORKLOADS[1]
    grid, box, edges = w.grid, w.box, w.pk_edges
    f = synth.gaussian_field(grid, (box,) * 3, 5, kaiser_beta=0.5).astype(np.float32)
    ref = ideal.pk_ideal(f, box, edges, 4)
    pb = pkg.PolyBin(grid, box, edges, lmax=4, prec=prec)
    assert np.array_equal(pb.mode_counts(), ref["counts"])
    P = pb.pk(torch.from_numpy(f).cuda())[0]
    Pd = pb.pk(torch.from_numpy(f).cuda(), discrete=True)[0]
    # error relative to the l = 0 power of the bin (the natural scale of every multipole's numerator)
    for il in range(3):
        e = np.abs(P[il] - ref["P"][il]) / np.abs(ref["P"][0])
        assert np.max(e) < TOL[prec]["rel"] * (4 * il + 1), (il, np.max(e))
        ed = np.abs(Pd[il] - ref["P_discrete"][il]) / np.abs(ref["P_discrete"][0])
        assert np.max(ed) < 10 * TOL[prec]["rel"] * (4 * il + 1), (il, np.max(ed))
    e0 = np.abs(P[0] - ref["P"][0]) / np.abs(ref["P"][0])
    assert np.max(e0) < TOL[prec]["rel"]
    pb.close()


def test_batch_and_stream(pkg):
    grid, box, ek, kind = CASES[1]
    edges = _kf(box) * ek
    fs = np.stack([_field(grid, box, kind, 40 + i) for i in range(3)])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="fp32", stream=s.cuda_stream)
        B = pb.bk_ideal(torch.from_numpy(fs).cuda())
        P = pb.pk(torch.from_numpy(fs).cuda())
    # a batch gives exactly the per-field results (same kernels, same order), and matches the oracle
    for i in range(3):
        B1 = pb.bk_ideal(torch.from_numpy(fs[i]).cuda())[0]
        assert np.array_equal(B[i], B1)
        ref = ideal.bk_ideal(fs[i], box, edges)
        e_norm_bound = 1e-6 * (box ** 6 / fs[i].size ** 3) / ref["T"]
        bins = binning.bin_grid(grid, box, edges)
        G = ideal.shell_maps(ideal.forward(fs[i]), bins, len(edges) - 1).reshape(len(edges) - 1, -1)
        absS = np.array([np.sum(np.abs(G[a] * G[b] * G[c])) for a, b, c in ref["triplets"]])
        assert np.all(np.abs(B[i] - ref["B"]) <= e_norm_bound * absS)
        pr = ideal.pk_ideal(fs[i], box, edges, 2)["P"]
        assert np.max(np.abs(P[i, 0] - pr[0]) / np.abs(pr[0])) < 1e-6
    pb.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_batched_host_input(pkg, pinned):
    """A batch of host fields is staged through two device buffers on a copy stream (the copy of field f + 1 overlaps
    the transforms of field f): results equal the per-field device calls bit for bit, for pinned and pageable memory."""
    grid, box, ek, kind = CASES[1]
    edges = _kf(box) * ek
    fs = np.stack([_field(grid, box, kind, 60 + i) for i in range(5)])
    host = torch.from_numpy(fs)
    if pinned:
        host = host.pin_memory()
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="split")
    B, P = pb.bk_pk(host)
    for i in range(5):
        B1, P1 = pb.bk_pk(torch.from_numpy(fs[i]).cuda())
        assert np.array_equal(B[i], B1[0]) and np.array_equal(P[i], P1[0])
    pb.close()


@pytest.mark.parametrize("prec", ["fp32", "split", "fp64"])
@pytest.mark.parametrize("case", [1, 8])
def test_bk_multipoles(pkg, case, prec):
    """B_ell, ell = 0, 2, 4, of a redshift-space (Kaiser) field against the oracle (Sec. 4.1, eq. ideal-bk), triplet by
    triplet with the criterion of tests/bk_criterion.py (kappa from sum_x |g_a g_b g_{c,ell}|)."""
    grid, box, ek, _ = CASES[case]
    edges = _kf(box) * ek
    f = synth.lognormal_field(grid, (box,) * 3, 60 + case, kaiser_beta=0.5).astype(np.float32)
    ref = ideal.bk_ideal_multipoles(f, box, edges, 4)
    pb = pkg.PolyBin(grid, box, edges, prec=prec)
    Bl = pb.bk_multipoles(torch.from_numpy(f).cuda(), 4)[0]
    if prec == "split":
        assert pb.last_path() == pkg.PATH_TENSOR_SPLIT_TF32X3
    abc, _ = pb.triplets()
    assert [tuple(t) for t in abc.tolist()] == ref["triplets"]
    # ell = 0 of this call is the monopole of polybin_bk_ideal, bit for bit
    assert np.array_equal(Bl[0], pb.bk_ideal(torch.from_numpy(f).cuda())[0])
    nb = len(edges) - 1
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    D = ideal.forward(f)
    G = ideal.shell_maps(D, bins, nb).reshape(nb, -1)
    for il, ell in enumerate(ref["ells"]):
        GL = G if ell == 0 else ideal.shell_maps_ell(D, bins, nb, ell, mu2).reshape(nb, -1)
        absS = np.array([np.dot(np.abs(G[a] * G[b]), np.abs(GL[c])) for a, b, c in ref["triplets"]])
        e_rel, e_norm, kappa = bk_errors(Bl[il], ref["B"][il], ref["S"][il], absS)
        s = check(ref["triplets"], e_rel, e_norm, kappa, norm_tol=TOL[prec]["norm"], rel_tol=TOL[prec]["rel"],
                  kappa_max=TOL[prec]["kappa_max"], label=f"case {case} {prec} ell {ell}")
        print(report(s, f"multipole ell={ell} case {case} {prec} contraction grid {pb.contraction_grid()}"))
    pb.close()
