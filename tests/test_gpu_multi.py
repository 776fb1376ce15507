"""Batched ideal bispectra over uneven grids in one CUDA-graph launch (polybin_bk_ideal_multi): identical to the
per-field calls (same kernels, same order), stable across cached replays, and equal to the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import binning, ideal
from paper_2404_07249_gb300 import synth

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
    ref = ideal.bk_ideal(host[1], box, edges)["B"]
    assert np.median(np.abs(multi[1] - ref) / np.abs(ref)) < 1e-6
    for pb in pbs.values():
        pb.close()
