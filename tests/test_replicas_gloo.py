"""Replicas-only multi-GPU path on CPU: two gloo ranks each hold a block of per-draw Fisher terms (computed here by
the oracle on a tiny grid); the host-side combination equals the single-process mean bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2404_07249_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _per_draw_terms(n_mc):
    from oracle import binning, unwindowed
    grid, box = (8, 8, 8), 300.0
    edges = binning.kf_of(box) * np.array([0.5, 1.5, 2.5, 3.5])
    bins = binning.bin_grid(grid, box, edges)
    mu2 = binning.mu2_grid(grid)
    n = 1.0 + 0.5 * np.random.Generator(np.random.PCG64(0)).random(grid)
    w = unwindowed.fkp_weight(n, 1.0)
    return np.stack([unwindowed.pk_fisher_draw(unwindowed.draw(grid, 7, r, unwindowed.STREAM_P), n, w, bins, mu2, 3,
                                               [0, 2]) for r in range(n_mc)])


def _worker(rank, world, port, n_mc, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r0, r1 = replicas.draw_range(n_mc, rank, world)
        terms = _per_draw_terms(n_mc)[r0:r1]
        F = replicas.combine_fisher_draws(terms, r0, n_mc)
        q.put((rank, F))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_mc", [5, 2])
def test_two_rank_combination_is_bit_identical(n_mc):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_mc, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    terms = _per_draw_terms(n_mc)
    ref = np.zeros(terms.shape[1:])
    for r in range(n_mc):
        ref = ref + terms[r]
    ref = ref / n_mc
    for F in results.values():
        assert np.array_equal(F, ref)


def test_draw_ranges_partition():
    for n_mc in range(0, 13):
        for world in range(1, 5):
            rs = [replicas.draw_range(n_mc, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n_mc
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
