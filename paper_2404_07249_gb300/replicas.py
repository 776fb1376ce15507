"""Host-side combination of Monte Carlo Fisher terms computed by independent replicas (one process per GPU).

The hot path shards over independent Monte Carlo draws; the only exchange is the FP64 sum of the per-draw
Fisher terms (Sec. 3.3.2 and Sec. 4.3.4: the Fisher matrix is the mean over draws).  Each rank computes a
contiguous range of draws with ``PolyBin.fisher_draws``; ``combine_fisher_draws`` gathers the per-draw matrices on
every rank (gloo or any torch.distributed backend, on CPU tensors) and sums them in draw order, so the result is
bit-identical to a single process computing all draws in sequence.
"""
from __future__ import annotations

import numpy as np


def draw_range(n_mc: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of draws [r0, r1) for ``rank`` out of ``world`` (sizes differ by at most one)."""
    base, extra = divmod(n_mc, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def combine_fisher_draws(per_draw: np.ndarray, r0: int, n_mc: int, group=None) -> np.ndarray:
    """Mean over all ranks' draws of the per-draw Fisher terms, summed in draw order (deterministic).

    per_draw: this rank's [r1 - r0][n][n] float64 terms for draws r0 .. r1-1.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = per_draw.shape[-1]
    mine = torch.from_numpy(np.ascontiguousarray(per_draw, dtype=np.float64).reshape(-1, n, n))
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([mine.shape[0]], dtype=torch.int64), group=group)
    starts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(starts, torch.tensor([r0], dtype=torch.int64), group=group)
    maxc = int(max(c.item() for c in counts))
    padded = torch.zeros((maxc, n, n), dtype=torch.float64)
    padded[: mine.shape[0]] = mine
    gathered = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(gathered, padded, group=group)
    terms = {}
    for g, c, s in zip(gathered, counts, starts):
        for i in range(int(c.item())):
            terms[int(s.item()) + i] = g[i].numpy()
    if sorted(terms) != list(range(n_mc)):
        raise ValueError(f"draws gathered {sorted(terms)} do not cover 0..{n_mc - 1}")
    acc = np.zeros((n, n))
    for r in range(n_mc):
        acc = acc + terms[r]
    return acc / n_mc
