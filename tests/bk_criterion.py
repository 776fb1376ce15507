"""Acceptance criterion of a bispectrum against the FP64 oracle, triplet by triplet (shared by the GPU tests, the
smoke run and the benchmark).

For every closed triplet (a, b, c) with oracle sums S = sum_x g_a g_b g_c and A = sum_x |g_a g_b g_c|:

* e_rel  = |B - B_ref| / |B_ref|                       (the target: <= 1e-6)
* e_norm = |B - B_ref| / (|B_ref| kappa) = |dS| / A     (error on the scale of the summands)
* kappa  = A / |S|                                      (conditioning of the sum: cancellation between cells)

A map error of relative size eps moves S by up to ~3 eps A, i.e. B by up to ~3 eps kappa relative.  The FP32
FFTs of the maps carry eps ~ 1e-7, so e_rel <= 1e-6 is reachable where kappa <= 10; where the sum cancels more
(kappa > 10) the FP64 reference itself depends on the last bits of the maps, and such triplets are held to
e_norm <= 1e-6 and listed, never passed silently.
"""
from __future__ import annotations

import numpy as np


def bk_errors(B, B_ref, S_ref, absS):
    B = np.asarray(B, dtype=np.float64)
    B_ref = np.asarray(B_ref, dtype=np.float64)
    kappa = np.asarray(absS, dtype=np.float64) / np.abs(np.asarray(S_ref, dtype=np.float64))
    e_rel = np.abs(B - B_ref) / np.abs(B_ref)
    e_norm = e_rel / kappa
    return e_rel, e_norm, kappa


def summarise(triplets, e_rel, e_norm, kappa, rel_tol=1e-6, kappa_max=10.0) -> dict:
    """Statistics and the explicit list of triplets above rel_tol (with their kappa and e_norm)."""
    above = np.nonzero(e_rel > rel_tol)[0]
    order = above[np.argsort(-e_rel[above])]
    return {
        "rel_tol": rel_tol,
        "kappa_max": kappa_max,
        "n_triplets": int(len(e_rel)),
        "max": float(np.max(e_rel)) if len(e_rel) else 0.0,
        "median": float(np.median(e_rel)) if len(e_rel) else 0.0,
        "max_e_norm": float(np.max(e_norm)) if len(e_norm) else 0.0,
        "n_above_tol": int(len(above)),
        "frac_le_tol": float(np.mean(e_rel <= rel_tol)) if len(e_rel) else 1.0,
        "max_e_rel_well_conditioned": (float(np.max(e_rel[kappa <= kappa_max])) if np.any(kappa <= kappa_max)
                                       else 0.0),
        "above_tol": [{"abc": [int(v) for v in triplets[i]], "e_rel": float(e_rel[i]), "kappa": float(kappa[i]),
                       "e_norm": float(e_norm[i])} for i in order],
    }


def check(triplets, e_rel, e_norm, kappa, norm_tol=1e-6, rel_tol=1e-6, kappa_max=10.0, label="") -> dict:
    """Assert the criterion; return the summary (whose `above_tol` list the caller prints)."""
    s = summarise(triplets, e_rel, e_norm, kappa, rel_tol, kappa_max)
    assert np.all(e_norm <= norm_tol), f"{label}: e_norm {np.max(e_norm):.3e} > {norm_tol}"
    bad = [x for x in s["above_tol"] if x["kappa"] <= kappa_max]
    assert not bad, f"{label}: triplets above {rel_tol} with kappa <= {kappa_max}: {bad[:5]}"
    return s


def report(s: dict, label: str) -> str:
    lines = [f"{label}: {s['n_triplets']} triplets, e_rel max {s['max']:.3e} median {s['median']:.3e}, "
             f"max e_norm {s['max_e_norm']:.3e}, {s['n_above_tol']} above {s['rel_tol']:g} "
             f"(max e_rel where kappa <= {s['kappa_max']:g}: {s['max_e_rel_well_conditioned']:.3e})"]
    for x in s["above_tol"]:
        lines.append(f"  {tuple(x['abc'])}: e_rel {x['e_rel']:.3e}, kappa {x['kappa']:.1f}, e_norm {x['e_norm']:.3e}")
    return "\n".join(lines)
