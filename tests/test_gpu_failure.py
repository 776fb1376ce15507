"""Failure detection without faulting the GPU: a bounded device-side wait gives up and reports through the error
flag, the context stays usable; bad inputs are rejected on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    grid, box = (32, 32, 32), 500.0
    edges = 2 * np.pi / box * np.array([1.0, 3.0, 5.0, 7.0])
    pb = pkg.PolyBin(grid, box, edges, prec="split")
    assert pb.selftest_wait() is True
    f = torch.randn(grid, device="cuda")
    B1 = pb.bk_ideal(f)
    assert pb.selftest_wait() is True
    B2 = pb.bk_ideal(f)
    assert np.array_equal(B1, B2)
    pb.close()


def test_host_side_rejections():
    import paper_2404_07249_gb300 as pkg
    grid, box = (32, 32, 32), 500.0
    edges = 2 * np.pi / box * np.array([1.0, 3.0, 5.0])
    pb = pkg.PolyBin(grid, box, edges, prec="fp32")
    with pytest.raises(pkg.PolybinError):
        pb.pk_unwindowed(torch.zeros(grid, device="cuda"), torch.zeros(grid, device="cuda"))   # no Fisher yet
    with pytest.raises(pkg.PolybinError):
        pb.fisher(np.zeros(grid, np.float32), np.zeros(grid, np.float32), 1, 1, 0)           # host arrays
    with pytest.raises(pkg.PolybinError):
        pb.solve(np.zeros((3, 3)), np.ones((3, 1)))                                          # singular
    pb.close()
