"""Throughput benchmark of the ideal bispectrum + P_ell hot path on one GB300 per rank.

Default workload: 512^3 lognormal field with a Kaiser factor, box 2000 Mpc/h, 30 linear k-bins to 0.3 h/Mpc,
bispectrum of every closed triplet plus P_ell (ell = 0, 2).  A step = one field through the whole ideal path
(forward FFT, shell filter + inverse FFTs, triplet contraction, P_ell binning) via polybin_bk_pk_ideal.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec split|fp32|fp64] [--impl ours|reference]

Under torchrun each rank runs its own realisation on its own GPU (weak scaling, no data-path collective);
timing is bracketed by a barrier + synchronize and the maximum over ranks is reported.  Inputs (537 MB per
field) are larger than L2, so no flush is needed between steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "512^3 bispectrum estimates/s, split-TC vs FP64 GPU path at 1e-6 rel. error"
UNIT = "estimates/s"


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the contraction kernel, from one ncu
# capture of the named workload and precision, keyed by the SHA-256 of the kernel source the capture ran.  The
# figure is reported only while that source is unchanged; otherwise traffic is null.  The capture ran the 512^3
# workload's bins, field model and box on a 320^3 data grid, whose contraction grid (288^3) is the 512^3 workload's:
# the contraction launch is the same (the same 30 maps of 288^3 cells).
E2E_BATCH = 8   # fields a call in the end-to-end measurement (pinned host memory: 8 x 537 MB at 512^3)

CAPTURED_TRAFFIC = {
    ("d0adcdac6517b4a7bcd1f13ff32d196a0d7b114e6af7dc113e7bf9bd4606e7a5", "lognormal_kaiser512", "split"):
        2866680832 + 3096832,
}


def _captured_traffic(workload: str, prec: str):
    import hashlib
    src = os.path.join(ROOT, "paper_2404_07249_gb300", "csrc", "contract_tc.cu")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return CAPTURED_TRAFFIC.get((digest, workload, prec))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(cfg: int):
    from paper_2404_07249_gb300 import synth
    w = synth.WORKLOADS[cfg]
    edges = w.bk_edges
    return w, edges


ORACLE_BINS = (0, 1, 4, 9, 14, 19, 24, 27, 29)   # bins of the sampled oracle comparison (all triplets among them)


def cpu_baseline(cfg: int, field: np.ndarray, edges, box: float, gpu=None) -> dict:
    """The FP64 oracle as it stands, timed on the host cores on a bounded sample of the same workload:
    one forward FFT of the field, one shell map (filter + inverse FFT) and the oracle's triple-sum routine on
    all n_b shell maps restricted to a contiguous slab of cells; the per-estimate time is
    t_forward + n_b t_shell + t_triple (N / N_slab) (every step of the oracle pipeline scales linearly in these).

    gpu = (B, triplets) of the GPU path on the same field: the oracle then also evaluates B_abc of every closed
    triplet among the bins ORACLE_BINS (shell and unit maps of those bins on the data grid, one pair product per
    pair) and the comparison is returned under "B_rel_err_vs_oracle" (tests/bk_criterion.py statistics, with the
    triplets above 1e-6 listed)."""
    from oracle import _fft, binning, ideal
    nb = len(edges) - 1
    N = field.size
    t0 = time.perf_counter()
    D = ideal.forward(field)
    t_fwd = time.perf_counter() - t0
    bins = binning.bin_grid(field.shape, box, edges)
    t0 = time.perf_counter()
    g0 = ideal.shell_maps(D, bins, nb, which=[nb // 2])
    t_shell = time.perf_counter() - t0
    slab = max(1, min(field.shape[0], int(field.shape[0] * min(1.0, 2.0e6 / N * 4))))
    rng = np.random.Generator(np.random.PCG64(1))
    gs = rng.standard_normal((nb, slab) + field.shape[1:])
    t0 = time.perf_counter()
    ideal.triple_sums(gs)
    t_tri = (time.perf_counter() - t0) * (field.shape[0] / slab)
    del g0, gs
    per = t_fwd + nb * t_shell + t_tri
    out = {"value": 1.0 / per, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"FP64 oracle, 1 forward FFT + 1 of {nb} shell maps + triple sums of {nb} maps over "
                     f"{slab}/{field.shape[0]} slabs, scaled to one {field.shape[0]}^3 estimate "
                     f"(t_fwd {t_fwd:.2f}s, t_shell {t_shell:.2f}s, t_triple {t_tri:.2f}s)",
           "extrapolated": True}
    if gpu is not None:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from bk_criterion import bk_errors, summarise
        B, trip = gpu
        keep = set(b for b in ORACLE_BINS if b < nb)
        pick = [i for i, t in enumerate(trip) if set(t) <= keep]
        t0 = time.perf_counter()
        g, tm = {}, {}
        for b in sorted(keep):
            sel = bins == b
            g[b] = _fft.ifftn(np.where(sel, D, 0.0)).real
            tm[b] = _fft.ifftn(sel.astype(np.complex128)).real
        S, T, A = np.zeros(len(pick)), np.zeros(len(pick)), np.zeros(len(pick))
        by_pair = {}
        for q, i in enumerate(pick):
            by_pair.setdefault(trip[i][1:], []).append((q, trip[i][0]))
        for (b, c), items in by_pair.items():
            pg, pt = (g[b] * g[c]).ravel(), (tm[b] * tm[c]).ravel()
            pa = np.abs(pg)
            for q, a in items:
                S[q] = np.dot(g[a].ravel(), pg)
                T[q] = np.dot(tm[a].ravel(), pt)
                A[q] = np.dot(np.abs(g[a]).ravel(), pa)
        del g, tm
        vol = float(box) ** 3
        Bref = vol * vol / float(N) ** 3 * S / T
        e_rel, e_norm, kappa = bk_errors(np.asarray(B)[pick], Bref, S, A)
        cmp_ = summarise([trip[i] for i in pick], e_rel, e_norm, kappa)
        cmp_["sample"] = (f"every closed triplet among bins {sorted(keep)} ({len(pick)} of {len(trip)}), FP64 oracle on "
                          f"the {'x'.join(str(n) for n in field.shape)} data grid ({time.perf_counter() - t0:.1f} s)")
        out["B_rel_err_vs_oracle"] = cmp_
    del D
    return out


def run_reference(args) -> None:
    """--impl reference: the FP64 CPU oracle on the same workload, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2404_07249_gb300 import synth
    w, edges = _workload(args.config)
    field = synth.workload_field(args.config, 0)
    vals = []
    last = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(args.config, field, edges, w.box)
        if i >= args.warmup:
            vals.append(r["value"])
        last = r
    v = float(np.mean(vals))
    cb = dict(last)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.grid), "box": w.box, "n_kbins": len(edges) - 1,
                       "statistics": "B_abc(all closed) + P_ell(0,2)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def cufft_comparison(field_dev, cgrid, nb, stream) -> dict:
    """cuFFT (through torch.fft) on the transforms the hot path replaces, timed with CUDA events on `stream`: the
    full R2C of the data grid (the path's forward stage computes only the reachable box) and n_b full C2R onto the
    contraction grid (the path's shell stage: n_b pruned inverse transforms).  A timed comparison only."""
    import torch
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        out["r2c_data_grid_ms"] = timed(lambda: torch.fft.rfftn(field_dev))
        half = torch.zeros((nb,) + tuple(cgrid[:2]) + (cgrid[2] // 2 + 1,), dtype=torch.complex64, device=field_dev.device)
        out[f"c2r_{nb}x_contraction_grid_ms"] = timed(lambda: torch.fft.irfftn(half, s=tuple(cgrid), dim=(1, 2, 3)))
        del half
    out["library"] = "cuFFT via torch.fft (full, unpruned transforms)"
    return out


def other_workloads(pkg, synth, stream, dev) -> dict:
    """Throughput of the remaining standard workloads (host-timed around synchronising C-ABI calls)."""
    import torch
    out = {}
    # 64^3 GRF: plain FP64 path, B (8 bins) and P_ell (16 bins, ell 0,2,4)
    w = synth.WORKLOADS[1]
    f = torch.from_numpy(synth.workload_field(1, 0)).to(dev)
    pbb = pkg.PolyBin(w.grid, w.box, w.bk_edges, prec="fp64", stream=stream.cuda_stream)
    pbp = pkg.PolyBin(w.grid, w.box, w.pk_edges, lmax=4, prec="fp64", stream=stream.cuda_stream)
    pbb.num_triplets()
    tb = _time(lambda: pbb.bk_ideal(f), 5)
    tp = _time(lambda: pbp.pk(f), 5)
    out["grf64_fp64"] = {"bk_per_s": 1 / tb, "pk_per_s": 1 / tp, "n_triplets": pbb.num_triplets()}
    pbb.close(); pbp.close()
    # 256^3 lognormal, 20 bins, split-TF32
    w = synth.WORKLOADS[2]
    f = torch.from_numpy(synth.workload_field(2, 0)).to(dev)
    pb = pkg.PolyBin(w.grid, w.box, w.bk_edges, prec="split", stream=stream.cuda_stream)
    pb.num_triplets()
    t = _time(lambda: pb.bk_ideal(f), 5)
    out["lognormal256_split"] = {"bk_per_s": 1 / t, "n_triplets": pb.num_triplets(),
                                 "contraction_grid": list(pb.contraction_grid())}
    pb.close()
    del f
    # 64 fields of 96^3 / 128^3 / 160^3, 12 bins, one CUDA graph
    w = synth.WORKLOADS[4]
    grids = [(g, g, g) for g in w.grids]
    pbs = {g: pkg.PolyBin(g, w.box, w.bk_edges, prec="split", stream=stream.cuda_stream) for g in grids}
    order = [grids[i % len(grids)] for i in range(w.n_fields)]
    fields = [torch.from_numpy(synth.workload_field(4, i)).to(dev) for i in range(w.n_fields)]
    t = _time(lambda: pkg.bk_ideal_multi([pbs[g] for g in order], fields), 3)
    out["lognormal_batch64_split_graph"] = {"fields_per_s": w.n_fields / t, "graph_launches_per_batch": 1}
    for pb in pbs.values():
        pb.close()
    del fields
    # masked 256^3: P and B Monte Carlo Fisher (per draw / draw pair) and the unwindowed estimates
    w = synth.WORKLOADS[5]
    n = synth.survey_mask(w.grid, (w.box,) * 3, 5000).astype(np.float32)
    nd = torch.from_numpy(n).to(dev)
    pbp = pkg.PolyBin(w.grid, w.box, w.pk_edges, lmax=4, prec="split", stream=stream.cuda_stream)
    wd = pbp.fkp_weights(nd, w.extra["P0"])
    dG = torch.from_numpy((n * synth.workload_field(5, 0)).astype(np.float32)).to(dev)
    tfp = _time(lambda: pbp.fisher_draws(nd, wd, 1, 0, 0, 1), 1)
    pbp.fisher(nd, wd, 2, 1, 0)
    tpu = _time(lambda: pbp.pk_unwindowed(dG, wd), 3)
    tpb = _time(lambda: pbp.pk_bias(nd, wd, pkg.FISHER_PK, n_mc=1, seed=3), 3)   # n2 = n (unit weights)
    pbp.pk_bias(None, None, pkg.FISHER_PK, n_mc=0)
    pbp.close()
    pbb = pkg.PolyBin(w.grid, w.box, w.bk_edges, prec="split", stream=stream.cuda_stream)
    nt = pbb.num_triplets()
    tfb = _time(lambda: pbb.fisher_draws(nd, wd, 1, 1, 0, 1), 1)
    mocks = torch.stack([torch.from_numpy((n * synth.workload_field(5, 1 + i)).astype(np.float32)) for i in range(2)]).to(dev)
    pbb.fisher(nd, wd, 1, 1, 1)
    tbu = _time(lambda: pbb.bk_unwindowed(dG, wd, mocks), 1)
    tbb = _time(lambda: pbb.bk_bias(nd, dG, dG, wd, n_mc=1, seed=3), 1)         # n3 = n, d2 = d (unit weights)
    pbb.close()
    out["masked256_split"] = {"pk_fisher_s_per_draw": tfp, "bk_fisher_s_per_draw_pair": tfb, "n_triplets": nt,
                              "pk_unwindowed_s": tpu, "bk_unwindowed_s_with_2_mocks": tbu,
                              "pk_shot_noise_s_per_draw": tpb, "bk_shot_noise_s_per_pair": tbb}
    out["masked256_optimal_fp32"] = optimal_workload(pkg, synth, stream, dev)
    out["masked256_local_split"] = local_workload(pkg, synth, stream, dev)
    return out


def noise_workload(pkg, synth, stream, dev) -> dict:
    """Shot-noise bias terms on the masked 256^3 workload (unit weights: n2 = n3 = n, d2 = d): one Monte Carlo map for
    P, one pair for B."""
    import torch
    w = synth.WORKLOADS[5]
    n = synth.survey_mask(w.grid, (w.box,) * 3, 5000).astype(np.float32)
    nd = torch.from_numpy(n).to(dev)
    d = torch.from_numpy((n * synth.workload_field(5, 0)).astype(np.float32)).to(dev)
    out = {}
    pb = pkg.PolyBin(w.grid, w.box, w.pk_edges, lmax=4, prec="split", stream=stream.cuda_stream)
    wd = pb.fkp_weights(nd, w.extra["P0"])
    out["pk_bias_s_per_draw"] = _time(lambda: pb.pk_bias(nd, wd, pkg.FISHER_PK, n_mc=1, seed=3), 3)
    pb.close()
    pbb = pkg.PolyBin(w.grid, w.box, w.bk_edges, prec="split", stream=stream.cuda_stream)
    pbb.num_triplets()
    out["bk_bias_s_per_pair"] = _time(lambda: pbb.bk_bias(nd, d, d, wd, n_mc=1, seed=3), 1)
    pbb.close()
    return out


def local_workload(pkg, synth, stream, dev) -> dict:
    """Local (Yamamoto) line of sight on the masked 256^3 workload, observer at the box centre (the survey geometry's
    own): the P numerator, one P Fisher draw, and the ideal bispectrum multipoles ell = 0, 2 of one field."""
    import torch
    w = synth.WORKLOADS[5]
    n = synth.survey_mask(w.grid, (w.box,) * 3, 5000).astype(np.float32)
    nd = torch.from_numpy(n).to(dev)
    d = torch.from_numpy((n * synth.workload_field(5, 0)).astype(np.float32)).to(dev)
    out = {}
    pb = pkg.PolyBin(w.grid, w.box, w.pk_edges, lmax=4, prec="split", stream=stream.cuda_stream)
    pb.set_observer((0.0, 0.0, 0.0))
    wd = pb.fkp_weights(nd, w.extra["P0"])
    out["pk_numerator_s"] = _time(lambda: pb.pk_unwindowed_local(d, wd, with_estimate=False), 3)
    out["pk_fisher_s_per_draw"] = _time(lambda: pb.fisher_draws(nd, wd, 1, pkg.FISHER_PK_LOCAL, 0, 1), 1)
    pb.close()
    pbb = pkg.PolyBin(w.grid, w.box, w.bk_edges, prec="split", stream=stream.cuda_stream)
    pbb.set_observer((0.0, 0.0, 0.0))
    pbb.num_triplets()
    out["bk_multipoles_l2_s"] = _time(lambda: pbb.bk_multipoles_local(d, 2), 3)
    out["bk_multipoles_l2_global_s"] = _time(lambda: pbb.bk_multipoles(d, 2), 3)
    pbb.close()
    return out


def optimal_workload(pkg, synth, stream, dev, fisher: bool = True) -> dict:
    """Optimal weighting S^-1 on the masked 256^3 workload (global line of sight, fiducial = the field's own power
    law, n2 = n): conjugate gradients with 10 iterations as in the paper's optimal-weight test (Sec. 6.1.2), and to a
    relative residual of 1e-5; one P Fisher draw (1 + n_alpha solves) and the unwindowed estimate."""
    import torch
    w = synth.WORKLOADS[5]
    n = synth.survey_mask(w.grid, (w.box,) * 3, 5000).astype(np.float32)
    nd = torch.from_numpy(n).to(dev)
    d = torch.from_numpy((n * synth.workload_field(5, 0)).astype(np.float32)).to(dev)
    pb = pkg.PolyBin(w.grid, w.box, w.pk_edges, lmax=4, prec="fp32", stream=stream.cuda_stream)
    kf = 2.0 * np.pi / w.box
    pfid = synth.power_law(kf * np.sqrt(np.arange(pb.max_shell() + 1, dtype=np.float64)))[None, :]
    out = {"grid": list(w.grid), "n_alpha": pb.n_alpha(pkg.FISHER_PK_OPT)}
    pb.set_optimal(nd, pfid, None, max_iter=10, tol=0.0)
    res = pb.sinv_optimal(d)
    t10 = _time(lambda: pb.sinv_optimal(d), 5)
    out.update({"solve_ms_10_iterations": 1e3 * t10, "ms_per_iteration": 1e3 * t10 / 10,
                "relres_after_10": res[2]})
    pb.set_optimal(nd, pfid, None, max_iter=200, tol=1e-5)
    res = pb.sinv_optimal(d)
    t5 = _time(lambda: pb.sinv_optimal(d), 3)
    out.update({"iterations_to_1e-5": res[1], "solve_ms_to_1e-5": 1e3 * t5})
    if fisher:
        pb.set_optimal(nd, pfid, None, max_iter=10, tol=0.0)
        out["pk_fisher_s_per_draw"] = _time(lambda: pb.fisher_draws(nd, None, 1, pkg.FISHER_PK_OPT, 0, 1), 1)
        pb.fisher(nd, None, 1, 1, pkg.FISHER_PK_OPT)
        out["pk_unwindowed_s"] = _time(lambda: pb.pk_unwindowed_opt(d), 3)
    pb.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split", choices=["split", "fp32", "fp64"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=1, help="steps of the FP64 GPU comparator (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, nargs=3, default=None,
                    help="profiling only: run the workload's field model, box and bins on another grid")
    ap.add_argument("--optimal-only", action="store_true",
                    help="profiling only: time the optimal-weighting solves on the masked 256^3 workload and exit")
    ap.add_argument("--only", choices=["local", "noise"], default=None,
                    help="profiling only: time the local line-of-sight or the shot-noise workload (masked 256^3) and exit")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the other workloads (64^3 FP64, 256^3, batched uneven grids, masked 256^3)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_2404_07249_gb300 as pkg
    from paper_2404_07249_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.optimal_only:
        out = optimal_workload(pkg, synth, torch.cuda.current_stream(dev), dev, fisher=False)
        if rank == 0:
            print(json.dumps({"workload": "masked256_optimal_fp32", **out}), flush=True)
        return
    if args.only:
        fn = local_workload if args.only == "local" else noise_workload
        out = fn(pkg, synth, torch.cuda.current_stream(dev), dev)
        if rank == 0:
            print(json.dumps({"workload": f"masked256_{args.only}", **out}), flush=True)
        return

    w, edges = _workload(args.config)
    grid, box = (tuple(args.grid) if args.grid else w.grid), w.box
    field = synth.workload_field(args.config, rank, grid=grid if args.grid else None)
    d = torch.from_numpy(field).to(dev)
    stream = torch.cuda.current_stream(dev)
    pb = pkg.PolyBin(grid, box, edges, lmax=max(w.lmax, 0), prec=args.prec, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    ntrip = pb.num_triplets()            # N_abc (FP64, cached): timed separately
    t_nabc = time.perf_counter() - t0
    want_pk = w.pk_edges is not None

    def step(x):
        return pb.bk_pk(x, True, want_pk)

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize(dev)

    # ---- device-resident throughput; per-stage CUDA events are recorded inside the same timed region (the
    # library reads them back only after the loop, so recording does not stall the host)
    pb.set_profiling(True)
    pb.stage_times(reset=True)
    launches0 = pb.launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(d)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = pb.launch_count() - launches0
    st = pb.stage_times(reset=True)
    pb.set_profiling(False)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in st.items()}
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1000.0 / ms

    # ---- end to end through the C-ABI with host buffers (pinned), H2D copy of every field inside the timed region:
    # batched calls of up to E2E_BATCH fields, which the library stages through two device buffers so that the copy
    # of field f + 1 overlaps the transforms of field f
    nbat = max(1, min(args.steps, E2E_BATCH))
    hbatch = torch.empty((nbat,) + field.shape, dtype=torch.float32, pin_memory=True)
    for i in range(nbat):
        hbatch[i].copy_(torch.from_numpy(field))
    step(hbatch[:nbat] if nbat > 1 else hbatch[0])   # warm-up with the same batch: the staging buffers exist before timing
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    left = args.steps
    while left > 0:
        k = min(left, nbat)
        step(hbatch[:k] if k > 1 else hbatch[0])
        left -= k
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps
    del hbatch
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = field.nbytes
    d2h = ntrip * 8 + (3 * (len(edges) - 1) * 8 if want_pk else 0)

    peaks, peak_src = _peaks()
    N = float(np.prod(grid))
    cgrid = pb.contraction_grid()
    Nc = float(np.prod(cgrid))
    nb = len(edges) - 1
    # dominant kernel: the triplet contraction over the cells of the alias-free contraction grid.  Algorithmic
    # work per launch: 2 flops per closed triplet per cell; algorithmic bytes: the n_b float32 maps read once.  The
    # intensity (2 ntrip / (4 n_b) flop per byte, ~47 at 30 bins) is below the TF32 ridge (peak TF/s over peak
    # TB/s, ~129), so the binding roof is HBM; the tensor-side rate is reported next to it.
    algo_flops = 2.0 * ntrip * Nc
    algo_bytes = 4.0 * nb * Nc
    t_con = stage_ms["contract"] / 1000.0
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks["hbm_gbs"])
    roof = {"bound": "hbm", "unit": "GB/s", "peak": hbm, "peak_source": f"{peak_src} hbm_gbs (copy bandwidth)"}
    roof["achieved"] = algo_bytes / t_con / 1e9 if t_con > 0 else None
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] else None
    if args.prec == "split":
        peak_tf = float(peaks["bf16_tflops_sustained"]) / 2.0        # TF32 dense = bf16 / 2 (nominal ratio)
        roof["tensor_side"] = {"achieved_tflops": algo_flops / t_con / 1e12 if t_con > 0 else None,
                               "peak_tflops": peak_tf,
                               "peak_source": f"{peak_src} bf16 sustained x 1/2 (TF32/bf16 nominal ratio)"}
    else:
        alu = 152 * 128 * 2 * sm_max * 1e6 / 1e12 if args.prec == "fp32" else 152 * 2 * 2 * sm_max * 1e6 / 1e12
        roof["alu_side"] = {"achieved_tflops": algo_flops / t_con / 1e12 if t_con > 0 else None, "peak_tflops": alu}
    roof["ridge_flop_per_byte"] = (roof.get("tensor_side", roof.get("alu_side"))["peak_tflops"] * 1e12) / (hbm * 1e9)
    roof["intensity_flop_per_byte"] = algo_flops / algo_bytes
    roof["traffic"] = _captured_traffic(w.name, args.prec)
    roof["kernel"] = ("k_contract_tc (triplet contraction, a3)" if args.prec == "split"
                      else "k_contract (triplet contraction, a3)")
    roof["algorithmic"] = (f"{nb} maps x {int(Nc)} cells x 4 B = {algo_bytes:.3e} B and 2 x {ntrip} closed triplets x "
                           f"{int(Nc)} cells = {algo_flops:.3e} flop per launch on the {cgrid} contraction grid (the "
                           f"same sums over the {int(N)} data-grid cells would be {2.0 * ntrip * N:.3e} flop)")
    roof["stage_ms"] = stage_ms
    roof["hbm_gbs_of_stages"] = {
        "forward": (N * 4 + 0) / (stage_ms["forward"] / 1e3) / 1e9 if stage_ms["forward"] else None,
        "shells_write_g": (nb * Nc * 4) / (stage_ms["shells"] / 1e3) / 1e9 if stage_ms["shells"] else None,
        "contract_read_g": (nb * Nc * 4) / (t_con) / 1e9 if t_con else None,
        "hbm_peak_gbs": hbm}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"split": "tf32x3", "fp32": "f32", "fp64": "f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": w.name + ("_grid_override" if args.grid else ""), "grid": list(grid), "box": box,
                       "n_kbins": nb, "n_triplets": ntrip, "contraction_grid": list(cgrid),
                       "statistics": "B_abc(all closed) + P_ell(0,2)", "precision_mode": args.prec,
                       "l2": f"inputs {field.nbytes / 1e6:.0f} MB" + (" > L2 (no flush needed)" if field.nbytes > 129e6
                                                                       else " (not larger than L2)"),
                       "nabc_init_s": t_nabc, "contraction_plan": pb.contract_plan_info()},
            "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks, "roofline": roof}

    # ---- FP64 GPU comparator (the plain double-precision path)
    if args.fp64_steps > 0 and args.prec != "fp64":
        pb64 = pkg.PolyBin(grid, box, edges, lmax=max(w.lmax, 0), prec="fp64", stream=stream.cuda_stream)
        pb64.num_triplets()
        pb64.bk_pk(d, True, want_pk)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            B64, _ = pb64.bk_pk(d, True, want_pk)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        B32, _ = step(d)
        rel = np.abs(B32[0] - B64[0]) / np.abs(B64[0])
        line["fp64_gpu_path"] = {"value": world * 1000.0 / ms64, "unit": UNIT, "ms_per_step": ms64,
                                 "speedup_of_value": (world * 1000.0 / ms) / (world * 1000.0 / ms64),
                                 "work": "same closed-triplet pairs and windows on the same contraction grid, FP64 "
                                         "FFTs and FP64 SIMT contraction",
                                 "B_rel_err_vs_fp64_gpu": {"max": float(rel.max()), "median": float(np.median(rel)),
                                                           "frac_le_1e-6": float(np.mean(rel <= 1e-6))}}
        pb64.close()

    # bispectrum quadrupole (ell = 2) of the same field: B_0 and B_2 from one forward transform
    t_mp = _time(lambda: pb.bk_multipoles(d, 2), max(1, args.steps // 2))
    line["bk_multipoles_ell_0_2"] = {"value": world / t_mp, "unit": "estimates/s (B_0 and B_2 of one field)",
                                     "ms_per_estimate": 1000.0 * t_mp}
    line["cufft_comparison"] = cufft_comparison(d, cgrid, nb, stream)
    line["cufft_comparison"]["ours_forward_ms"] = stage_ms["forward"]
    line["cufft_comparison"]["ours_shells_ms"] = stage_ms["shells"]
    B_last, _ = step(d)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        abc, _ = pb.triplets()
        cb = cpu_baseline(args.config, field, edges, box, gpu=(B_last[0], [tuple(t) for t in abc.tolist()]))
        cmp_ = cb.pop("B_rel_err_vs_oracle", None)
        line["cpu_baseline"] = cb
        if cmp_ is not None:
            line["B_rel_err_vs_oracle"] = cmp_
    if not args.no_other_workloads and world == 1 and not args.grid:
        del d
        torch.cuda.empty_cache()
        line["other_workloads"] = other_workloads(pkg, synth, stream, dev)
    pb.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
