"""Python binding of libpolybin (argument marshalling only; all compute runs in the CUDA library).

The shared library is built in-tree by ``paper_2404_07249_gb300.build.build()`` (nvcc, sm_103a) into
``paper_2404_07249_gb300/_build/libpolybin.so``.  There is no CPU fallback: if the library is missing,
``load()`` raises.

Device arrays are ``torch`` CUDA tensors (torch is used only for device memory and streams); host arrays are
numpy.  Entry points mirror the C-ABI of ``include/polybin.h``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpolybin.so")

FP64, FP32, SPLIT_TF32X3 = 0, 1, 2
_PREC = {"fp64": FP64, "fp32": FP32, "split_tf32x3": SPLIT_TF32X3, "split": SPLIT_TF32X3}

_lib = None

_SIGS = {
    "polybin_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "polybin_destroy": (None, [ctypes.c_void_p]),
    "polybin_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "polybin_num_triplets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "polybin_get_triplets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_bk_ideal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "polybin_pk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "polybin_pk_discrete": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "polybin_mode_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_spectrum_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_shell_maps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_contract": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p]),
    "polybin_bk_pk_ideal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "polybin_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "polybin_get_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "polybin_launch_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "polybin_fkp_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "polybin_mc_draw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "polybin_fisher": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p]),
    "polybin_fisher_draws": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_ulonglong,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "polybin_set_fisher": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "polybin_pk_unwindowed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "polybin_bk_unwindowed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_bk_ideal_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "polybin_selftest_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "polybin_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]),
    "polybin_last_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "polybin_set_observer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_pk_unwindowed_local": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p]),
    "polybin_bk_ideal_multipoles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_void_p]),
    "polybin_contraction_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_bk_ideal_multipoles_local": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                         ctypes.c_void_p]),
    "polybin_contract_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "polybin_max_shell": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "polybin_set_optimal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "polybin_sinv_optimal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "polybin_pk_unwindowed_opt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polybin_bk_bias": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p]),
    "polybin_bk_unwindowed_shot": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p]),
    "polybin_pk_bias": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_ulonglong, ctypes.c_void_p]),
}

FISHER_PK, FISHER_BK, FISHER_PK_LOCAL, FISHER_PK_OPT = 0, 1, 2, 3
PATH_SIMT_FP64, PATH_SIMT_FP32, PATH_TENSOR_SPLIT_TF32X3 = 0, 1, 2

STAGES = ("forward", "shells", "contract", "pk_bin")


class PolybinError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Load libpolybin (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PolybinError(f"libpolybin is not built ({path} missing); run paper_2404_07249_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Raw address of a torch tensor (device or host) or numpy array."""
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _f32(x):
    """float32, C-contiguous view (torch tensor or numpy array)."""
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            x = x.to(torch.float32).contiguous()
        return x
    return np.ascontiguousarray(x, dtype=np.float32)


class PolyBin:
    """One grid + one set of k-bins on one GPU (wraps a polybin_ctx)."""

    def __init__(self, grid, boxsize, k_edges, lmax: int = 0, prec="fp32", stream=None):
        lib = load()
        self.lib = lib
        self.grid = tuple(int(g) for g in grid)
        box = boxsize if np.ndim(boxsize) else (boxsize,) * 3
        self.box = tuple(float(b) for b in box)
        self.edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        self.nb = len(self.edges) - 1
        self.lmax = int(lmax)
        self.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        g = (ctypes.c_int * 3)(*self.grid)
        b = (ctypes.c_double * 3)(*self.box)
        e = self.edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = lib.polybin_init(ctypes.byref(ctx), g, b, e, self.nb, self.lmax, self.prec, ctypes.c_void_p(stream))
        if rc != 0:
            raise PolybinError(f"polybin_init: {rc}: {lib.polybin_last_error(None).decode()}")
        self.ctx = ctx
        self.ncell = int(np.prod(self.grid))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.polybin_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise PolybinError(f"{what}: {rc}: {self.lib.polybin_last_error(self.ctx).decode()}")

    # ---- bispectrum
    def num_triplets(self) -> int:
        n = ctypes.c_int()
        self._check(self.lib.polybin_num_triplets(self.ctx, ctypes.byref(n)), "polybin_num_triplets")
        return n.value

    def triplets(self):
        n = self.num_triplets()
        abc = np.zeros((n, 3), dtype=np.int32)
        cnt = np.zeros(n, dtype=np.float64)
        self._check(self.lib.polybin_get_triplets(self.ctx, _ptr(abc), _ptr(cnt)), "polybin_get_triplets")
        return abc, cnt

    def bk_ideal(self, delta) -> np.ndarray:
        delta = _f32(delta)
        batch = delta.shape[0] if delta.ndim == 4 else 1
        out = np.zeros((batch, self.num_triplets()), dtype=np.float64)
        self._check(self.lib.polybin_bk_ideal(self.ctx, _ptr(delta), batch, _ptr(out)), "polybin_bk_ideal")
        return out

    def bk_multipoles(self, delta, lmax_b: int = 2) -> np.ndarray:
        """B_ell for ell = 0, 2, .., lmax_b: array [batch][lmax_b / 2 + 1][n_triplets]."""
        delta = _f32(delta)
        batch = delta.shape[0] if delta.ndim == 4 else 1
        out = np.zeros((batch, lmax_b // 2 + 1, self.num_triplets()), dtype=np.float64)
        self._check(self.lib.polybin_bk_ideal_multipoles(self.ctx, _ptr(delta), batch, int(lmax_b), _ptr(out)),
                    "polybin_bk_ideal_multipoles")
        return out

    def bk_multipoles_local(self, delta, lmax_b: int = 2) -> np.ndarray:
        """B_ell with the local line of sight of set_observer: array [batch][lmax_b / 2 + 1][n_triplets]."""
        delta = _f32(delta)
        batch = delta.shape[0] if delta.ndim == 4 else 1
        out = np.zeros((batch, lmax_b // 2 + 1, self.num_triplets()), dtype=np.float64)
        self._check(self.lib.polybin_bk_ideal_multipoles_local(self.ctx, _ptr(delta), batch, int(lmax_b), _ptr(out)),
                    "polybin_bk_ideal_multipoles_local")
        return out

    # ---- power spectrum
    def pk(self, delta, discrete: bool = False) -> np.ndarray:
        delta = _f32(delta)
        batch = delta.shape[0] if delta.ndim == 4 else 1
        out = np.zeros((batch, self.lmax // 2 + 1, self.nb), dtype=np.float64)
        fn = self.lib.polybin_pk_discrete if discrete else self.lib.polybin_pk
        self._check(fn(self.ctx, _ptr(delta), batch, _ptr(out)), "polybin_pk")
        return out

    def bk_pk(self, delta, want_bk: bool = True, want_pk: bool = True):
        """(B [batch][n_triplets] or None, P [batch][n_ell][nb] or None) from one forward transform per field."""
        delta = _f32(delta)
        batch = delta.shape[0] if delta.ndim == 4 else 1
        B = np.zeros((batch, self.num_triplets()), dtype=np.float64) if want_bk else None
        P = np.zeros((batch, self.lmax // 2 + 1, self.nb), dtype=np.float64) if want_pk else None
        self._check(self.lib.polybin_bk_pk_ideal(self.ctx, _ptr(delta), batch, None if B is None else _ptr(B),
                                                 None if P is None else _ptr(P)), "polybin_bk_pk_ideal")
        return B, P

    def set_profiling(self, on: bool):
        self._check(self.lib.polybin_set_profiling(self.ctx, int(bool(on))), "polybin_set_profiling")

    def stage_times(self, reset: bool = True) -> dict:
        ms = np.zeros(4, dtype=np.float64)
        calls = np.zeros(4, dtype=np.int64)
        self._check(self.lib.polybin_get_stage_times(self.ctx, _ptr(ms), _ptr(calls), int(reset)),
                    "polybin_get_stage_times")
        return {n: (float(ms[i]), int(calls[i])) for i, n in enumerate(STAGES)}

    def selftest_wait(self) -> bool:
        """True when the bounded device-side wait gave up as designed (see polybin_selftest_wait)."""
        t = ctypes.c_int(0)
        self._check(self.lib.polybin_selftest_wait(self.ctx, ctypes.byref(t)), "polybin_selftest_wait")
        return t.value == 1

    def last_path(self) -> int:
        """Which contraction kernel produced the last result (PATH_* constants; -1 before the first)."""
        p = ctypes.c_int()
        self._check(self.lib.polybin_last_path(self.ctx, ctypes.byref(p)), "polybin_last_path")
        return p.value

    def contraction_grid(self):
        """Lengths of the alias-free grid the triplet sums are evaluated on."""
        d = np.zeros(3, dtype=np.int32)
        self._check(self.lib.polybin_contraction_grid(self.ctx, _ptr(d)), "polybin_contraction_grid")
        return tuple(int(v) for v in d)

    def contract_plan_info(self) -> dict:
        """The closed-triplet tensor-core plan and the autotuner's choice (-1 entries before the first estimate)."""
        info = np.zeros(6, dtype=np.int32)
        ms = ctypes.c_float(0.0)
        self._check(self.lib.polybin_contract_plan_info(self.ctx, _ptr(info), ctypes.byref(ms)),
                    "polybin_contract_plan_info")
        keys = ("tile_cost", "group_cap", "cta_mode", "row_groups", "ctas_per_group", "candidates_timed")
        out = {k: int(v) for k, v in zip(keys, info)}
        out["ms"] = float(ms.value)
        return out

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        self._check(self.lib.polybin_launch_count(self.ctx, ctypes.byref(n)), "polybin_launch_count")
        return n.value

    # ---- masked estimators
    def n_alpha(self, which: int) -> int:
        return self.num_triplets() if which == FISHER_BK else (self.lmax // 2 + 1) * self.nb

    def set_observer(self, pos):
        """Observer of the local line of sight, box coordinates centred on the origin (Mpc/h)."""
        p = np.ascontiguousarray(pos, dtype=np.float64)
        self._check(self.lib.polybin_set_observer(self.ctx, _ptr(p)), "polybin_set_observer")

    def pk_unwindowed_local(self, d_dev, w_dev, with_estimate: bool = True):
        na = self.n_alpha(FISHER_PK_LOCAL)
        p = np.zeros(na)
        pnum = np.zeros(na)
        self._check(self.lib.polybin_pk_unwindowed_local(self.ctx, _ptr(_f32(d_dev)), _ptr(_f32(w_dev)),
                                                         _ptr(p) if with_estimate else None, _ptr(pnum)),
                    "polybin_pk_unwindowed_local")
        return (p if with_estimate else None), pnum

    def fkp_weights(self, n_dev, p_fkp: float):
        import torch
        w = torch.empty_like(n_dev, dtype=torch.float32)
        self._check(self.lib.polybin_fkp_weights(self.ctx, _ptr(_f32(n_dev)), float(p_fkp), _ptr(w)),
                    "polybin_fkp_weights")
        return w

    def mc_draw(self, seed: int, draw: int, stream: int, device="cuda"):
        import torch
        out = torch.empty(self.grid, dtype=torch.float32, device=device)
        self._check(self.lib.polybin_mc_draw(self.ctx, int(seed), int(draw), int(stream), _ptr(out)), "polybin_mc_draw")
        return out

    def fisher(self, n_dev, w_dev, n_mc: int, seed: int, which: int, checkpoint: str | None = None):
        """Monte Carlo Fisher matrix and its inverse; w_dev may be None for FISHER_PK_OPT."""
        na = self.n_alpha(which)
        F = np.zeros((na, na))
        Finv = np.zeros((na, na))
        ck = checkpoint.encode() if checkpoint else None
        n32 = _f32(n_dev)
        w32 = None if w_dev is None else _f32(w_dev)
        self._check(self.lib.polybin_fisher(self.ctx, _ptr(n32), None if w32 is None else _ptr(w32), int(n_mc),
                                            int(seed), int(which), _ptr(F), _ptr(Finv), ck), "polybin_fisher")
        return F, Finv

    def fisher_draws(self, n_dev, w_dev, seed: int, which: int, r0: int, r1: int):
        na = self.n_alpha(which)
        out = np.zeros((r1 - r0, na, na))
        n32 = _f32(n_dev)
        w32 = None if w_dev is None else _f32(w_dev)
        self._check(self.lib.polybin_fisher_draws(self.ctx, _ptr(n32), None if w32 is None else _ptr(w32), int(seed),
                                                  int(which), int(r0), int(r1), _ptr(out)), "polybin_fisher_draws")
        return out

    def pk_bias(self, n2_dev, w_dev=None, which: int = FISHER_PK, n_mc: int = 1, seed: int = 0):
        """Shot-noise bias of the P numerator (pixel units, cached and subtracted by the estimates; n_mc = 0 clears)."""
        out = np.zeros(self.n_alpha(which))
        n2 = None if n2_dev is None else _f32(n2_dev)
        w = None if w_dev is None else _f32(w_dev)
        self._check(self.lib.polybin_pk_bias(self.ctx, None if n2 is None else _ptr(n2), None if w is None else _ptr(w),
                                             int(which), int(n_mc), int(seed), _ptr(out)), "polybin_pk_bias")
        return out

    def bk_bias(self, n3_dev, d2_dev, d_dev, w_dev, n_mc: int = 1, seed: int = 0):
        """Shot-noise bias of the B numerator (units of b_num), FKP weighting."""
        out = np.zeros(self.num_triplets())
        args = [_f32(x) for x in (n3_dev, d2_dev, d_dev, w_dev)]
        self._check(self.lib.polybin_bk_bias(self.ctx, *[_ptr(x) for x in args], int(n_mc), int(seed), _ptr(out)),
                    "polybin_bk_bias")
        return out

    def bk_unwindowed_shot(self, d_dev, w_dev, n3_dev, d2_dev, mocks_dev=None, n_mc: int = 1, seed: int = 0):
        """(b = F^-1 (b_num - b_bias) in physical units, b_num, b_bias)."""
        nt = self.num_triplets()
        b, bnum, bias = np.zeros(nt), np.zeros(nt), np.zeros(nt)
        args = [_f32(x) for x in (d_dev, w_dev, n3_dev, d2_dev)]
        nm = 0 if mocks_dev is None else int(mocks_dev.shape[0])
        mk = None if mocks_dev is None else _f32(mocks_dev)
        self._check(self.lib.polybin_bk_unwindowed_shot(self.ctx, _ptr(args[0]), _ptr(args[1]),
                                                        None if mk is None else _ptr(mk), nm, _ptr(args[2]),
                                                        _ptr(args[3]), int(n_mc), int(seed), _ptr(b), _ptr(bnum),
                                                        _ptr(bias)), "polybin_bk_unwindowed_shot")
        return b, bnum, bias

    # ---- optimal weighting (conjugate gradients)
    def max_shell(self) -> int:
        """Largest binned |n|^2: fiducial tables hold up to max_shell() + 1 shells."""
        v = ctypes.c_int(0)
        self._check(self.lib.polybin_max_shell(self.ctx, ctypes.byref(v)), "polybin_max_shell")
        return v.value

    def set_optimal(self, n_w_dev, pfid, n2_w_dev=None, max_iter: int = 10, tol: float = 0.0):
        """Configure S^-1 = optimal weighting: pfid[l][s] the fiducial multipole 2 l on the shell |n|^2 = s."""
        pf = np.ascontiguousarray(np.atleast_2d(pfid), dtype=np.float64)
        nw = _f32(n_w_dev)
        n2 = None if n2_w_dev is None else _f32(n2_w_dev)
        self._check(self.lib.polybin_set_optimal(self.ctx, _ptr(nw), None if n2 is None else _ptr(n2), _ptr(pf),
                                                 int(pf.shape[0]), int(pf.shape[1]), int(max_iter), float(tol)),
                    "polybin_set_optimal")

    def sinv_optimal(self, v_dev, transpose: bool = False):
        """(S^-1 v or S^-T v as a device tensor of the working type, iterations, final relative residual)."""
        import torch
        v = _f32(v_dev)
        out = torch.empty(tuple(self.grid), dtype=self._real_dtype(), device=v.device)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        self._check(self.lib.polybin_sinv_optimal(self.ctx, _ptr(v), int(bool(transpose)), _ptr(out), ctypes.byref(it),
                                                  ctypes.byref(rel)), "polybin_sinv_optimal")
        return out, it.value, rel.value

    def pk_unwindowed_opt(self, d_dev, with_estimate: bool = True):
        na = self.n_alpha(FISHER_PK_OPT)
        p = np.zeros(na)
        pnum = np.zeros(na)
        d = _f32(d_dev)
        self._check(self.lib.polybin_pk_unwindowed_opt(self.ctx, _ptr(d), _ptr(p) if with_estimate else None,
                                                       _ptr(pnum)), "polybin_pk_unwindowed_opt")
        return (p if with_estimate else None), pnum

    def set_fisher(self, which: int, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        self._check(self.lib.polybin_set_fisher(self.ctx, int(which), _ptr(F)), "polybin_set_fisher")

    def pk_unwindowed(self, d_dev, w_dev, with_estimate: bool = True):
        na = self.n_alpha(FISHER_PK)
        p = np.zeros(na)
        pnum = np.zeros(na)
        self._check(self.lib.polybin_pk_unwindowed(self.ctx, _ptr(_f32(d_dev)), _ptr(_f32(w_dev)),
                                                   _ptr(p) if with_estimate else None, _ptr(pnum)),
                    "polybin_pk_unwindowed")
        return (p if with_estimate else None), pnum

    def bk_unwindowed(self, d_dev, w_dev, mocks_dev=None, with_estimate: bool = True):
        nt = self.num_triplets()
        b = np.zeros(nt)
        bnum = np.zeros(nt)
        lin = np.zeros(nt)
        nm = 0 if mocks_dev is None else int(mocks_dev.shape[0])
        self._check(self.lib.polybin_bk_unwindowed(self.ctx, _ptr(_f32(d_dev)), _ptr(_f32(w_dev)),
                                                   None if mocks_dev is None else _ptr(_f32(mocks_dev)), nm,
                                                   _ptr(b) if with_estimate else None, _ptr(bnum), _ptr(lin)),
                    "polybin_bk_unwindowed")
        return (b if with_estimate else None), bnum, lin

    def solve(self, A, B):
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        B2 = B.reshape(B.shape[0], -1)
        X = np.zeros_like(B2)
        self._check(self.lib.polybin_solve(self.ctx, _ptr(A), A.shape[0], _ptr(B2), B2.shape[1], _ptr(X)),
                    "polybin_solve")
        return X.reshape(B.shape)

    def mode_counts(self) -> np.ndarray:
        out = np.zeros(self.nb, dtype=np.float64)
        self._check(self.lib.polybin_mode_counts(self.ctx, _ptr(out)), "polybin_mode_counts")
        return out

    # ---- steps
    def spectrum_shape(self):
        dims = np.zeros(3, dtype=np.int32)
        lo = np.zeros(3, dtype=np.int32)
        self._check(self.lib.polybin_spectrum_shape(self.ctx, _ptr(dims), _ptr(lo)), "polybin_spectrum_shape")
        return tuple(int(d) for d in dims), tuple(int(v) for v in lo)

    def _real_dtype(self):
        import torch
        return torch.float64 if self.prec == FP64 else torch.float32

    def forward(self, delta_dev):
        import torch
        dims, _ = self.spectrum_shape()
        cdt = torch.complex128 if self.prec == FP64 else torch.complex64
        out = torch.empty(dims, dtype=cdt, device=delta_dev.device)
        d = _f32(delta_dev)
        self._check(self.lib.polybin_forward(self.ctx, _ptr(d), _ptr(out)), "polybin_forward")
        return out

    def shell_maps(self, spec_dev):
        import torch
        out = torch.empty((self.nb,) + self.grid, dtype=self._real_dtype(), device=spec_dev.device)
        self._check(self.lib.polybin_shell_maps(self.ctx, _ptr(spec_dev), _ptr(out)), "polybin_shell_maps")
        return out

    def contract(self, g_dev, h_dev=None) -> np.ndarray:
        ng = g_dev.shape[0]
        nh = ng if h_dev is None else h_dev.shape[0]
        out = np.zeros((ng * (ng + 1) // 2, nh), dtype=np.float64)
        self._check(self.lib.polybin_contract(self.ctx, _ptr(g_dev), ng, None if h_dev is None else _ptr(h_dev), nh,
                                              _ptr(out)), "polybin_contract")
        return out


def bk_ideal_multi(pbs, fields):
    """Ideal bispectra of fields on several grids in one CUDA-graph launch (polybin_bk_ideal_multi).
    pbs[i]: the PolyBin of field i (one stream for all); fields[i]: device float32 tensor."""
    lib = load()
    n = len(pbs)
    ctxs = (ctypes.c_void_p * n)(*[pb.ctx.value for pb in pbs])
    fs = [_f32(f) for f in fields]
    fptr = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fs])
    outs = [np.zeros(pb.num_triplets()) for pb in pbs]
    optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    rc = lib.polybin_bk_ideal_multi(ctxs, fptr, n, optr)
    if rc != 0:
        raise PolybinError(f"polybin_bk_ideal_multi: {rc}: {lib.polybin_last_error(pbs[0].ctx).decode()}")
    return outs


def pair_list(n: int):
    """Pairs (j <= k) in the lexicographic order used by ``PolyBin.contract``."""
    return [(j, k) for j in range(n) for k in range(j, n)]
