"""Batched ideal bispectra over uneven grids in one CUDA-graph launch (polybin_bk_ideal_multi): identical to the
per-field calls (same kernels, same order), stable across cached replays, and every field equal to the oracle
triplet by triplet (tests/bk_criterion.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, ideal
from paper_2404_07249_gb300 import synth

from bk_criterion import bk_errors, check, report

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_multi_matches_single(prec):
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    box = 500.0
    edges = binning.kf_of(box) * (1.0 + 2.0 * np.arange(7))
    grids = [(24, 24, 24), (32, 32, 32), (40, 40, 40)]
    stream = torch.cuda.current_stream().cuda_stream
    pbs = {g: pkg.PolyBin(g, box, edges, prec=prec, stream=stream) for g in grids}
    order = [grids[i % 3] for i in range(7)]
    host = [synth.lognormal_field(g, (box,) * 3, 400 + i).astype(np.float32) for i, g in enumerate(order)]
    fields = [torch.from_numpy(f).cuda() for f in host]
    single = [pbs[g].bk_ideal(f)[0] for g, f in zip(order, fields)]
    for rep in range(2):
        multi = pkg.bk_ideal_multi([pbs[g] for g in order], fields)
        for s, m in zip(single, multi):
            assert np.array_equal(s, m), rep
    nb = len(edges) - 1
    for i, (g, f) in enumerate(zip(order, host)):
        ref = ideal.bk_ideal(f, box, edges)
        bins = binning.bin_grid(g, box, edges)
        absS_full = ideal.triple_sums(np.abs(ideal.shell_maps(ideal.forward(f), bins, nb)))
        absS = np.array([absS_full[a, b, c] for a, b, c in ref["triplets"]])
        e_rel, e_norm, kappa = bk_errors(multi[i], ref["B"], ref["S"], absS)
        s = check(ref["triplets"], e_rel, e_norm, kappa, label=f"field {i} {g}")
        print(report(s, f"field {i} {g} {prec}"))
    for pb in pbs.values():
        pb.close()


def test_multi_batch_of_64_uneven_grids():
    """The 64-field batch of 96^3 / 128^3 / 160^3 lognormal realisations (L = 1000 Mpc/h, 12 bins k_F (1, 3, .., 25)),
    one CUDA graph: every field equals its single-field call bit for bit, and two fields of each grid equal the
    oracle triplet by triplet."""
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    w = synth.WORKLOADS[4]
    grids = [(g, g, g) for g in w.grids]
    stream = torch.cuda.current_stream().cuda_stream
    pbs = {g: pkg.PolyBin(g, w.box, w.bk_edges, prec="split", stream=stream) for g in grids}
    order = [grids[i % len(grids)] for i in range(w.n_fields)]
    host = [synth.workload_field(4, i) for i in range(w.n_fields)]
    fields = [torch.from_numpy(f).cuda() for f in host]
    multi = pkg.bk_ideal_multi([pbs[g] for g in order], fields)
    for g, pb in pbs.items():
        assert pb.contraction_grid() == (80, 80, 80), (g, pb.contraction_grid())
    for i in range(w.n_fields):
        assert np.array_equal(multi[i], pbs[order[i]].bk_ideal(fields[i])[0]), i
    nb = len(w.bk_edges) - 1
    for i in (0, 1, 2, 61, 62, 63):
        g, f = order[i], host[i]
        ref = ideal.bk_ideal(f, w.box, w.bk_edges)
        bins = binning.bin_grid(g, w.box, w.bk_edges)
        absS_full = ideal.triple_sums(np.abs(ideal.shell_maps(ideal.forward(f), bins, nb)))
        absS = np.array([absS_full[a, b, c] for a, b, c in ref["triplets"]])
        e_rel, e_norm, kappa = bk_errors(multi[i], ref["B"], ref["S"], absS)
        s = check(ref["triplets"], e_rel, e_norm, kappa, label=f"field {i} {g}")
        print(report(s, f"batch field {i} {g}"))
    for pb in pbs.values():
        pb.close()
