"""ctypes wrapper around ``brute.c`` (oracle pin; test infrastructure only).

``build()`` compiles the C file with gcc into ``oracle/_build/libbrute.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libbrute.so")


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "brute.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", _SO, src, "-lm"])
    return _SO


def brute_bk(D, grid, kf: float, edges, D2=None, D3=None) -> tuple[np.ndarray, np.ndarray | None]:
    """(count[a,b,c], sum Re D1(k1) D2(k2) D3(k3) [a,b,c]) over ordered closed triangles
    (k1 in a, k2 in b, k3 in c).  D2 and D3 default to D (single field)."""
    lib = ctypes.CDLL(build())
    nb = len(edges) - 1
    e = np.ascontiguousarray(edges, dtype=np.float64)
    cnt = np.zeros(nb ** 3)
    dp = ctypes.POINTER(ctypes.c_double)
    keep = []
    if D is not None:
        ptrs = []
        for X in (D, D if D2 is None else D2, D if D3 is None else D3):
            re_ = np.ascontiguousarray(X.real, dtype=np.float64)
            im_ = np.ascontiguousarray(X.imag, dtype=np.float64)
            keep += [re_, im_]
            ptrs += [re_.ctypes.data_as(dp), im_.ctypes.data_as(dp)]
        sdd = np.zeros(nb ** 3)
        args = (*ptrs, cnt.ctypes.data_as(dp), sdd.ctypes.data_as(dp))
    else:
        sdd = None
        args = (None, None, None, None, None, None, cnt.ctypes.data_as(dp), None)
    lib.brute_bk3.restype = ctypes.c_int
    rc = lib.brute_bk3(ctypes.c_int(grid[0]), ctypes.c_int(grid[1]), ctypes.c_int(grid[2]), ctypes.c_double(kf),
                       e.ctypes.data_as(dp), ctypes.c_int(nb), *args)
    if rc != 0:
        raise MemoryError("brute_bk failed")
    cnt = cnt.reshape(nb, nb, nb)
    return cnt, (None if sdd is None else sdd.reshape(nb, nb, nb))
