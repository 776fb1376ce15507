"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module generates *inputs only*: density fields with a prescribed power
spectrum, the survey-mask geometry and the bin edges of the standard
workloads.  It contains none of the estimator arithmetic (no shell filters,
no triplet sums, no Legendre binning, no weights): both the CUDA path and the
FP64 oracle receive the arrays produced here and do their own work.

Recipes (all host-side numpy / scipy.fft in float64, stored as float32):

* Gaussian random field (GRF): white noise w_x ~ N(0,1) from numpy's PCG64
  seeded with ``seed``; W = rfftn(w); D = W * sqrt(P(|k|) N / V) with the
  k = 0 mode set to zero; delta = irfftn(D).  With this normalisation
  <|D(k)|^2> = N^2 P(k) / V, i.e. the pixel-convention power spectrum is P.
* Lognormal field: delta = exp(delta_G) / mean(exp(delta_G)) - 1
  (unit mean density, mean exactly zero up to rounding).
* Linear Kaiser factor: D(k) <- D(k) (1 + beta mu^2) with mu = k_z/|k| along
  the last array axis, applied after the lognormal transform, D(0) = 0.
* Survey mask: spherical shell r_min < r < r_max around the box centre with
  seeded spherical holes; inside, n(x) = n0 exp(-(r - r0)^2 / s2).

The standard workloads (grid, box, field type and bins) are listed in
``WORKLOADS``; the random seed of realisation ``i`` of workload ``c`` is
``1000 * c + i``.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

try:  # scipy.fft is multithreaded; numpy.fft is the fallback
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=os.cpu_count())

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=os.cpu_count())
except ImportError:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)


def power_law(k: np.ndarray, amp: float = 2.0e4, k0: float = 0.1, slope: float = -1.5) -> np.ndarray:
    """P(k) = amp (k/k0)^slope for k > 0, zero at k = 0 (units (Mpc/h)^3, k in h/Mpc)."""
    out = np.zeros_like(k, dtype=np.float64)
    pos = k > 0
    out[pos] = amp * (k[pos] / k0) ** slope
    return out


def _kgrid_half(grid, box):
    """|k| and k_z on the rfftn half-spectrum grid, as broadcastable arrays."""
    n0, n1, n2 = grid
    kf = [2.0 * math.pi / b for b in box]
    kx = np.fft.fftfreq(n0, d=1.0 / n0) * kf[0]
    ky = np.fft.fftfreq(n1, d=1.0 / n1) * kf[1]
    kz = np.fft.rfftfreq(n2, d=1.0 / n2) * kf[2]
    return kx[:, None, None], ky[None, :, None], kz[None, None, :]


def _apply_half(spec, grid, box, fn):
    """spec[ix] *= fn(kmag, kz) slab by slab (keeps memory bounded at 512^3)."""
    kx, ky, kz = _kgrid_half(grid, box)
    for i in range(grid[0]):
        k2 = kx[i, 0, 0] ** 2 + ky[0] ** 2 + kz[0] ** 2  # (n1, n2h)
        spec[i] *= fn(np.sqrt(k2), np.broadcast_to(kz[0], k2.shape))
    return spec


def gaussian_field(grid, box, seed: int, pk=power_law, kmin: float | None = None,
                   kmax: float | None = None, kaiser_beta: float = 0.0) -> np.ndarray:
    """Seeded GRF in float64 with power spectrum ``pk`` (optionally zeroed outside [kmin, kmax)),
    optionally multiplied by the linear Kaiser factor (1 + beta mu^2) in k-space."""
    grid = tuple(int(g) for g in grid)
    box = tuple(float(b) for b in box)
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal(grid)
    spec = _rfftn(white)
    del white
    ntot = float(np.prod(grid))
    vol = float(np.prod(box))

    def amp(kmag, kz):
        p = pk(kmag)
        if kmin is not None:
            p = np.where(kmag >= kmin, p, 0.0)
        if kmax is not None:
            p = np.where(kmag < kmax, p, 0.0)
        a = np.sqrt(p * ntot / vol)
        if kaiser_beta:
            with np.errstate(invalid="ignore", divide="ignore"):
                mu2 = np.where(kmag > 0, (kz / np.where(kmag > 0, kmag, 1.0)) ** 2, 0.0)
            a = a * (1.0 + kaiser_beta * mu2)
        return a

    _apply_half(spec, grid, box, amp)
    spec[0, 0, 0] = 0.0
    return _irfftn(spec, grid)


def lognormal_field(grid, box, seed: int, pk=power_law, kaiser_beta: float = 0.0) -> np.ndarray:
    """exp(GRF) normalised to unit mean, minus one; optional Kaiser factor (1 + beta mu^2)."""
    g = gaussian_field(grid, box, seed, pk)
    np.exp(g, out=g)
    g /= g.mean()
    g -= 1.0
    if kaiser_beta:
        spec = _rfftn(g)

        def fac(kmag, kz):
            with np.errstate(invalid="ignore", divide="ignore"):
                mu2 = np.where(kmag > 0, (kz / np.where(kmag > 0, kmag, 1.0)) ** 2, 0.0)
            return 1.0 + kaiser_beta * mu2

        _apply_half(spec, grid, box, fac)
        spec[0, 0, 0] = 0.0
        g = _irfftn(spec, grid)
    return g


def plane_wave_field(grid, waves) -> np.ndarray:
    """Sum of cosines: waves = [(amplitude, (nx, ny, nz), phase), ...] with integer wave numbers."""
    n0, n1, n2 = grid
    x = np.arange(n0)[:, None, None] / n0
    y = np.arange(n1)[None, :, None] / n1
    z = np.arange(n2)[None, None, :] / n2
    out = np.zeros(grid, dtype=np.float64)
    for amp, (a, b, c), ph in waves:
        out += amp * np.cos(2.0 * math.pi * (a * x + b * y + c * z) + ph)
    return out


@dataclass
class SurveyGeometry:
    r_min: float = 600.0
    r_max: float = 1400.0
    n_holes: int = 20
    hole_radius: float = 50.0
    n0: float = 3.0e-4
    r0: float = 1000.0
    s2: float = 4.0e5


def survey_mask(grid, box, seed: int, geom: SurveyGeometry = SurveyGeometry()) -> np.ndarray:
    """Background density n(x) (h/Mpc)^3: shell around the box centre with seeded spherical holes.

    Cell centres are x_i = (i + 1/2) L / N - L / 2 (observer at the origin = box centre).  Hole
    centres are drawn uniformly in the shell volume (radius from the r^2 law, isotropic direction).
    Regions of the shell clipped by the box faces are simply absent (periodic wrap accepted).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(geom.n_holes)
    rh = (geom.r_min ** 3 + u * (geom.r_max ** 3 - geom.r_min ** 3)) ** (1.0 / 3.0)
    v = rng.standard_normal((geom.n_holes, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    centres = v * rh[:, None]
    axes = [(np.arange(n) + 0.5) * (L / n) - L / 2.0 for n, L in zip(grid, box)]
    x = axes[0][:, None, None]
    y = axes[1][None, :, None]
    z = axes[2][None, None, :]
    r = np.sqrt(x * x + y * y + z * z)
    inside = (r > geom.r_min) & (r < geom.r_max)
    for c in centres:
        d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        inside &= d2 >= geom.hole_radius ** 2
    return np.where(inside, geom.n0 * np.exp(-((r - geom.r0) ** 2) / geom.s2), 0.0)


# ---------------------------------------------------------------------------------------------
# Standard workloads (grid, box, field recipe, bins).  Edges are in h/Mpc, half-open [e_b, e_b+1).


def _kf(box):
    return 2.0 * math.pi / box


@dataclass
class Workload:
    name: str
    grid: tuple
    box: float
    field: str                      # "grf" | "lognormal" | "lognormal_kaiser" | "masked_grf"
    bk_edges: np.ndarray | None = None
    pk_edges: np.ndarray | None = None
    lmax: int = 0
    grids: tuple = ()               # batched workload: grid of realisation i = grids[i % len]
    n_fields: int = 1
    extra: dict = field(default_factory=dict)


def _edges_odd(kf, n_bins):
    """k_F (1, 3, 5, ...): bins of width 2 k_F starting at k_F."""
    return kf * (1.0 + 2.0 * np.arange(n_bins + 1))


def _edges_even(kf, n_bins):
    """k_F (0, 2, 4, ...): bins of width 2 k_F starting at 0 (k = 0 itself is never binned)."""
    return kf * (2.0 * np.arange(n_bins + 1))


WORKLOADS = {
    1: Workload("grf64", (64, 64, 64), 1000.0, "grf",
                bk_edges=_edges_odd(_kf(1000.0), 8), pk_edges=_edges_even(_kf(1000.0), 16), lmax=4),
    2: Workload("lognormal256", (256, 256, 256), 2000.0, "lognormal",
                bk_edges=np.linspace(0.0, 0.2, 21)),
    3: Workload("lognormal_kaiser512", (512, 512, 512), 2000.0, "lognormal_kaiser",
                bk_edges=np.linspace(0.0, 0.3, 31), pk_edges=np.linspace(0.0, 0.3, 31), lmax=2),
    4: Workload("lognormal_batch", (128, 128, 128), 1000.0, "lognormal",
                bk_edges=_edges_odd(_kf(1000.0), 12), grids=(96, 128, 160), n_fields=64),
    5: Workload("masked256", (256, 256, 256), 2500.0, "masked_grf",
                bk_edges=_edges_odd(_kf(2500.0), 16), pk_edges=_edges_even(_kf(2500.0), 24), lmax=4,
                extra={"P0": 1.0e4, "n_mc": 10, "n_mocks": 10}),
}


def workload_field(cfg: int, i: int = 0, grid=None) -> np.ndarray:
    """Realisation ``i`` of workload ``cfg`` as float32 (seed 1000*cfg + i)."""
    w = WORKLOADS[cfg]
    seed = 1000 * cfg + i
    if grid is None:
        grid = (w.grids[i % len(w.grids)],) * 3 if w.grids else w.grid
    box = (w.box,) * 3
    if w.field == "grf":
        f = gaussian_field(grid, box, seed)
    elif w.field == "lognormal":
        f = lognormal_field(grid, box, seed)
    elif w.field == "lognormal_kaiser":
        f = lognormal_field(grid, box, seed, kaiser_beta=0.5)
    elif w.field == "masked_grf":
        lo = float(min(w.bk_edges[0], w.pk_edges[0]))
        hi = float(max(w.bk_edges[-1], w.pk_edges[-1]))
        f = gaussian_field(grid, box, seed, kmin=lo if lo > 0 else None, kmax=hi)
    else:  # pragma: no cover
        raise ValueError(w.field)
    return np.ascontiguousarray(f, dtype=np.float32)


def uniform_edges(kf: float, start: float, width: float, n_bins: int) -> np.ndarray:
    """Edges kf * (start + width * b), b = 0..n_bins."""
    return kf * (start + width * np.arange(n_bins + 1))
