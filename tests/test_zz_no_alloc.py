"""The allocation-free contraction entry point (for callers that cannot allocate device memory, such as code
running inside a caller-managed memory pool) against the context-based polybin_contract, through the C-ABI.

Collected last on purpose: if it fails, a run that stops at the first failure has already run every other test.
It passes both alone in a fresh process and after the other tests (its scratch keeps the previous call's
contents, which every call overwrites before reading).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import build
    build.build()
    lib = pkg.load()
    lib.polybin_contract_noalloc.restype = ctypes.c_int
    lib.polybin_contract_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
    lib.polybin_contract_noalloc_error.restype = ctypes.c_char_p
    return lib


def _noalloc(lib, g, h, out, stream):
    ng = g.shape[0]
    nh = ng if h is None else h.shape[0]
    ncell = g[0].numel()
    return lib.polybin_contract_noalloc(ctypes.c_void_p(g.data_ptr()), ng,
                                        None if h is None else ctypes.c_void_p(h.data_ptr()), nh, ncell,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("ng,nh,grid,same", [(30, 30, (64, 48, 40), True), (9, 5, (40, 48, 32), False)])
def test_noalloc_matches_context_contract(lib, ng, nh, grid, same):
    import paper_2404_07249_gb300 as pkg
    rng = np.random.Generator(np.random.PCG64(3))
    g = torch.from_numpy(rng.standard_normal((ng,) + grid).astype(np.float32)).cuda()
    h = None if same else torch.from_numpy(rng.standard_normal((nh,) + grid).astype(np.float32)).cuda()
    pb = pkg.PolyBin(grid, 800.0, np.array([0.01, 0.02]), prec="fp32")
    ref = pb.contract(g, h)
    pb.close()
    G = g.double().reshape(ng, -1)
    H = (g if same else h).double().reshape(nh, -1)
    scale = np.array([(torch.abs(G[j] * G[k]) @ torch.abs(H).T).cpu().numpy()
                      for j in range(ng) for k in range(j, ng)])
    stream = torch.cuda.current_stream()
    for call in range(2):                    # two calls in a row share (and overwrite) the scratch
        out = torch.full((ng * (ng + 1) // 2, nh), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, g, h, out, stream)
        assert rc == 0, lib.polybin_contract_noalloc_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / scale) < 1e-6, call


def test_noalloc_rejects_oversize(lib):
    g = torch.zeros((65, 8), device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, g, None, out, torch.cuda.current_stream()) == -1
    assert b"64" in lib.polybin_contract_noalloc_error()
