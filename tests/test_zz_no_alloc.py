"""The allocation-free contraction entry point, through the C-ABI.  It serves callers that cannot allocate device
memory: code running inside a caller-managed memory pool or arena, plugins whose host application owns every
allocation, and threads that must not call cudaMalloc/cudaFree because those calls can synchronise the device.

Its output is checked against an FP64 product of the same maps computed on the host (independent of every CUDA
kernel) and against the context-based polybin_contract, within 1e-6 of sum_x |g_j g_k h_i|, on two calls in a row
and with the number of maps changing between calls (9, 30, 9), which exercises the pair tables it keeps for every
map count.

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


def _noalloc(lib, g, h, out, stream, ng=None):
    ng = g.shape[0] if ng is None else ng
    nh = ng if h is None else h.shape[0]
    ncell = g[0].numel()
    return lib.polybin_contract_noalloc(ctypes.c_void_p(g.data_ptr()), ng,
                                        None if h is None else ctypes.c_void_p(h.data_ptr()), nh, ncell,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def _host_fp64(g, h):
    """M[(j<=k)][i] = sum_x g_j g_k h_i and the scale sum_x |g_j g_k h_i|, in FP64 on the host."""
    G = g.cpu().double().numpy().reshape(g.shape[0], -1)
    H = G if h is None else h.cpu().double().numpy().reshape(h.shape[0], -1)
    ref, scale = [], []
    for j in range(G.shape[0]):
        for k in range(j, G.shape[0]):
            p = G[j] * G[k]
            ref.append(p @ H.T)
            scale.append(np.abs(p) @ np.abs(H).T)
    return np.array(ref), np.array(scale)


CASES = {9: (9, 5, (40, 48, 32), False), 30: (30, 30, (64, 48, 40), True)}


def test_noalloc_matches_fp64_and_context_contract(lib):
    import paper_2404_07249_gb300 as pkg
    rng = np.random.Generator(np.random.PCG64(3))
    data = {}
    for key, (ng, nh, grid, same) in CASES.items():
        g = torch.from_numpy(rng.standard_normal((ng,) + grid).astype(np.float32)).cuda()
        h = None if same else torch.from_numpy(rng.standard_normal((nh,) + grid).astype(np.float32)).cuda()
        ref, scale = _host_fp64(g, h)
        pb = pkg.PolyBin(grid, 800.0, np.array([0.01, 0.02]), prec="fp32")
        ctx_out = pb.contract(g, h)
        pb.close()
        data[key] = (g, h, ref, scale, ctx_out)
    stream = torch.cuda.current_stream()
    # two calls in a row for every size, and the map count changing between calls: 9, 30, 9
    for key in (9, 9, 30, 30, 9):
        g, h, ref, scale, ctx_out = data[key]
        out = torch.full(ref.shape, float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, g, h, out, stream)
        assert rc == 0, lib.polybin_contract_noalloc_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / scale) < 1e-6, key
        assert np.max(np.abs(got - ctx_out) / scale) < 1e-6, key


def test_noalloc_rejects_oversize_and_host_pointers(lib):
    stream = torch.cuda.current_stream()
    g = torch.zeros((65, 8), device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, g, None, out, stream) == -1
    assert b"64" in lib.polybin_contract_noalloc_error()
    # a host array passed by mistake is refused before any kernel runs
    gh = torch.zeros((2, 8))
    out2 = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, gh, None, out2, stream) == -1
    assert b"device memory" in lib.polybin_contract_noalloc_error()
    outh = torch.zeros((3, 2), dtype=torch.float64)
    assert _noalloc(lib, g[:2].contiguous(), None, outh, stream) == -1
