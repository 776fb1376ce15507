"""Per-stage timing and launch counting: brackets recorded without blocking are all read back, timing does not
change results, and more brackets than the event slots hold are still counted."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_stage_times_count_every_call_and_leave_results_unchanged():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    grid, box = (48, 48, 48), 600.0
    kf = 2 * np.pi / box
    edges = kf * np.array([1.0, 3.0, 5.0, 7.0, 9.0])
    pb = pkg.PolyBin(grid, box, edges, lmax=2, prec="split")
    f = torch.randn(grid, device="cuda")
    B0, P0 = pb.bk_pk(f, True, True)
    pb.set_profiling(True)
    pb.stage_times(reset=True)
    n = 40                                  # 4 stages x 40 calls = 160 brackets > the 64 event slots
    for _ in range(n):
        B1, P1 = pb.bk_pk(f, True, True)
    st = pb.stage_times(reset=True)
    pb.set_profiling(False)
    assert np.array_equal(B0, B1) and np.array_equal(P0, P1)
    for name in pkg.STAGES:
        ms, calls = st[name]
        assert calls == n, (name, calls)
        assert ms > 0.0, name
    assert all(v == (0.0, 0) for v in pb.stage_times(reset=False).values())
    l0 = pb.launch_count()
    pb.bk_pk(f, True, True)
    assert pb.launch_count() > l0
    pb.close()
