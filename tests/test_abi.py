"""The C-ABI library loads and exports every symbol declared in include/polybin.h; argument validation
works without a GPU (CPU only; no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_07249_gb300 import build
    path = build.build()
    import paper_2404_07249_gb300 as pkg
    return pkg.load(path)


def declared_symbols():
    out = []
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            out += re.findall(r"\b(polybin_\w+)\s*\(", txt)
    return sorted(set(out))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "polybin_init" in names and "polybin_bk_ideal" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def _init(lib, grid=(32, 32, 32), box=(800.0,) * 3, edges=(0.01, 0.02, 0.03), lmax=0, prec=1):
    ctx = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    b = (ctypes.c_double * 3)(*box)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    rc = lib.polybin_init(ctypes.byref(ctx), g, b, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(e) - 1,
                          lmax, prec, None)
    return rc, ctx


@pytest.mark.parametrize("kw", [
    dict(grid=(31, 32, 32)),             # odd
    dict(grid=(32, 32, 14)),             # prime factor 7
    dict(grid=(2048, 32, 32)),           # too long for smem staging
    dict(box=(800.0, 800.0, 700.0)),     # non-cubic box
    dict(box=(0.0, 0.0, 0.0)),
    dict(edges=(0.02, 0.01)),            # descending
    dict(edges=(0.01,)),                 # no bin
    dict(edges=tuple(np.linspace(0, 0.1, 66))),   # 65 bins
    dict(lmax=3),
    dict(lmax=6),
    dict(prec=7),
])
def test_init_rejects_bad_arguments(lib, kw):
    rc, ctx = _init(lib, **kw)
    assert rc == -1
    assert not ctx.value
    assert lib.polybin_last_error(None)


def test_null_arguments(lib):
    assert lib.polybin_init(None, None, None, None, 1, 0, 1, None) == -1
    lib.polybin_destroy(None)
    n = ctypes.c_int()
    assert lib.polybin_num_triplets(None, ctypes.byref(n)) == -1
