#!/usr/bin/env python
"""Neighbourhood-graph benchmark (exact kNN + fuzzy connectivities).

One step = rsc_knn (prep, candidate search, exact FP32 re-rank) followed by
rsc_connectivities (rho/sigma/weights, fuzzy union, CSR) over the whole
1,000,000-cell x 50-PC workload, inputs resident in HBM.  Prints one JSON
line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own
seeded input (the graph step has no exchange): weak scaling, value = all
cells / max-over-ranks time.  ``--impl reference`` times the FP64 CPU oracle
on bounded query samples of the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neighbors graph cells/s (50 PCs, k=15): BF16+rerank vs FP32 at recall@15≥0.999"
WORKLOAD = ("1,000,000 cells x 50 PCs fp32, 100-cluster Gaussian mixture (means ~N(0,4I), "
            "PC variance 1/t), euclidean, k=15")

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one search
# phase, from an ncu capture summarised under profiles/; valid only while the
# sources it was measured on are unchanged (their hash is checked).
SEARCH_SOURCES = ("knn_tc.cuh", "knn_tc_prune.cu", "prune.cu", "topk.cuh", "tc_ptx.cuh")
CONN_SOURCES = ("connectivities.cu",)
TRAFFIC = {
    # window pass + list pass of the 1,000,000-cell graph (profiles/knn_tc_pruned_passes_bf16_1m.md):
    # 256.1 + 206.3 MB and 1403.3 + 116.5 MB, cold-cache under ncu; the bound kernels are not included
    ("knn_tc.cuh", "pruned"): {"bytes_per_launch": 1_982_258_744, "kernel_sha": "dcf8edee4e3e25bc"},
    # the eight launches of one rsc_connectivities call on the 1,000,000-cell k = 15 lists
    # (profiles/connectivities_graph_1m_k15.md), cold-cache under ncu
    ("connectivities.cu", "graph"): {"bytes_per_launch": 1_800_462_336, "kernel_sha": "d6300e549cd22f3b"},
    # one UMAP epoch of the 1,000,000-cell k = 15 graph (profiles/umap_epoch_1m.md): 220.9 + 8.1 MB
    ("umap.cu", "epoch"): {"bytes_per_launch": 228_918_272, "kernel_sha": "3b64a6d38e4b0abd"},
    # one edist_tc_kernel launch of the 300,000-cell, 2,000-group screen
    # (profiles/edist_tc_groups_60k_300k.md): 17.45 GB + 24.63 MB as ncu rounds them
    # (hash taken after the entry point gained its trace range; the kernel is unchanged)
    ("edist.cu", "screen"): {"bytes_per_launch": 17_474_630_000, "kernel_sha": "9948e3aed94fcac2"},
    # the eight join launches of one 1,000,000-cell rsc_knn_descent call
    # (profiles/nndescent_join_1m_300k.md)
    ("nndescent.cu", "call"): {"bytes_per_launch": 106_520_583_424, "kernel_sha": "186c10799f37c1d6"},
}
ED_SOURCES = ("edist.cu", "knn_tc.cuh", "tc_ptx.cuh")
NND_SOURCES = ("nndescent.cu",)

ORDER_MIN_ROWS = 16384   # automatic locality ordering from this many rows (BF16 path)


def launches_per_step(metric, precision, n):
    """Kernels this library launches per graph step.

    rsc_knn: FP32 prep (column sums + column means + prep for Euclidean, prep
    alone for cosine), the BF16 operand prep (tensor-core path), the locality
    ordering (two k-means levels of 1 init + 2 Lloyd rounds x 6 + 5 for the
    full assignment and sort, a sort being 4 launches, 2 chain passes, + 1
    gather of the re-rank rows), the candidate
    search (one launch, or 12 when pruned: window pass, 2 sphere passes, group
    spheres, tau, count, scan (2), fill, offsets, item order, list pass) and
    the re-rank;
    rsc_connectivities: 8 (smooth, push, match, two scan launches, emit and the
    two queued-row sorts).
    """
    knn = (3 if metric == "euclidean" else 1) + 2
    if precision == "bf16":
        knn += 1 + (39 + 12 if n >= ORDER_MIN_ROWS else 0)
    return knn + 8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["auto", "fp32", "bf16", "fp8"], default="auto")
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--k", type=int, default=15)
    p.add_argument("--fp32-steps", type=int, default=1, help="timed steps of the plain FP32 path for comparison")
    p.add_argument("--locality", choices=["auto", "on", "off"], default="auto",
                   help="locality ordering of the BF16 search (graph workload)")
    p.add_argument("--prune", choices=["auto", "on", "off"], default="auto",
                   help="exact tile pruning of the BF16 search (graph workload)")
    p.add_argument("--full-scan-steps", type=int, default=2,
                   help="timed steps of the BF16 path with pruning off, for comparison")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--candidates", type=int, default=0, help="candidates per row before the exact re-rank (0 = default)")
    p.add_argument("--workload", choices=["graph", "batched", "partitioner", "cosine", "umap", "edistance",
                                          "nndescent", "leiden"],
                   default="graph",
                   help="graph: the 1M-cell neighbourhood graph (headline); batched: 64 samples, ~3M cells; "
                        "partitioner: learned-partition kNN graph of 5M cells; cosine: 11M-cell cosine graph, k=30; "
                        "umap: 200-epoch UMAP layout of the 1M-cell graph; edistance: all-pairs E-distance of a "
                        "300k-cell, 2,000-group screen")
    p.add_argument("--epochs", type=int, default=200, help="UMAP layout epochs (umap workload)")
    return p.parse_args()


def _kernel_sha(names):
    h = hashlib.sha256()
    for name in names:
        src = os.path.join(ROOT, "paper_2603_02402_gb300", "csrc", name)
        if not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    return h.hexdigest()[:16]


def exact_distances(X, q, gi, metric="euclidean"):
    """FP64 distances between query rows q and their returned ids gi [len(q), k]:
    Euclidean, or cosine 1 - cos with zero rows at 0 from each other and 1 from
    every other row (the oracle's conventions)."""
    import numpy as np
    xq = X[q].astype(np.float64)
    yg = X[gi].astype(np.float64)
    if metric == "euclidean":
        return np.sqrt(((xq[:, None, :] - yg) ** 2).sum(-1))
    nq = np.linalg.norm(xq, axis=1)[:, None]
    ng = np.linalg.norm(yg, axis=2)
    cos = np.einsum("qd,qjd->qj", xq, yg) / np.maximum(nq * ng, 1e-300)
    return np.where((nq == 0) & (ng == 0), 0.0, np.where((nq == 0) | (ng == 0), 1.0, 1.0 - cos))


def recall_by_distance(dex, kth):
    """recall@k, tie-tolerant: a returned id counts when its FP64 distance dex
    is within the oracle's k-th distance kth (per query)."""
    import numpy as np
    return float((dex <= np.asarray(kth)[:, None] * (1 + 1e-6) + 1e-12).mean())


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def setup_dist(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_barrier(world):
    """Barrier over the ranks of the job (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (one rank: x itself)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank processes its own units)."""
    return world * units_per_rank / (ms / 1e3)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on bounded query samples."""
    world, rank, _ = setup_dist(args)
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2603_02402_gb300 import synth
    oracle.build()
    X = synth.mixture(args.n, 50, n_comp=100, seed=0)
    per_step = max(16, int(os.environ.get("RSC_REF_QUERIES", "0")) or 0)
    # size each step so W + K steps fit in about two minutes
    t0 = time.perf_counter()
    oracle.knn(X, args.k, queries=synth.query_sample(args.n, 16, seed=99))
    t16 = time.perf_counter() - t0
    budget = 120.0 / max(1, args.warmup + args.steps)
    per_step = max(per_step, int(16 * budget / max(t16, 1e-3)))
    per_step = min(per_step, args.n)
    times = []
    for s in range(args.warmup + args.steps):
        q = synth.query_sample(args.n, per_step, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.knn(X, args.k, queries=q)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    cores = oracle.num_threads()
    sample = f"{per_step} seeded query rows per step against all {args.n} rows (kNN stage; FP64, {cores} threads)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "d": 50, "k": args.k, "sample_queries": per_step},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    rsc.lib()
    n, d, k = args.n, 50, args.k
    metric = "euclidean"

    X = synth.mixture(n, d, n_comp=100, seed=rank)
    X_pin = torch.from_numpy(X).pin_memory()
    Xd = X_pin.to(dev)
    stream = torch.cuda.current_stream(dev)

    precision = args.precision
    if precision == "auto":
        try:
            rsc.rsc_knn_workspace_size(n, d, k, metric, "bf16")
            precision = "bf16"
        except rsc.RscError:
            precision = "fp32"

    def buffers(prec, prune=args.prune):
        ws_knn = torch.empty(rsc.rsc_knn_workspace_size(n, d, k, metric, prec, locality=args.locality, prune=prune),
                             dtype=torch.uint8, device=dev)
        return ws_knn

    cap = rsc.rsc_connectivities_max_nnz(n, k)
    ws_conn = torch.empty(rsc.rsc_connectivities_workspace_size(n, k), dtype=torch.uint8, device=dev)
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    dst = torch.empty((n, k), dtype=torch.float32, device=dev)
    indptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    indices = torch.empty(cap, dtype=torch.int32, device=dev)
    data = torch.empty(cap, dtype=torch.float32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    sigma = torch.empty(n, dtype=torch.float32, device=dev)

    def make_events(count):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(count)]
        for e in evs:
            e.record(stream)     # materialise the underlying cudaEvent_t
        torch.cuda.synchronize(dev)
        return evs

    def step(prec, ws_knn, ev=None, prune=args.prune):
        arr = None
        if ev is not None:
            arr = (ctypes.c_void_p * 4)(*[e.cuda_event for e in ev[:4]])
        rsc.rsc_knn(Xd, k, metric, prec, workspace=ws_knn, out=(idx, dst), phase_events=arr, locality=args.locality,
                    prune=prune)
        rsc.rsc_connectivities(idx, dst, nnz_capacity=cap, workspace=ws_conn,
                               out=(indptr, indices, data, rho, sigma))
        if ev is not None:
            ev[4].record(stream)

    def barrier():
        rank_barrier(world)

    def max_ms(x):
        return max_over_ranks(x, world, dev)

    def timed(prec, steps, warmup, clocks=False, prune=args.prune):
        ws_knn = buffers(prec, prune)
        for _ in range(warmup):
            step(prec, ws_knn, prune=prune)
        torch.cuda.synchronize(dev)
        phase = [make_events(5) for _ in range(steps)]
        start, end = make_events(2)
        sampler = ClockSampler(_smi_id(dev)) if clocks else None
        if sampler:
            sampler.__enter__()
        barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for s in range(steps):
            step(prec, ws_knn, phase[s], prune=prune)
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        if sampler:
            sampler.__exit__()
        if rsc.rsc_workspace_status(ws_knn) != rsc.RSC_OK or rsc.rsc_workspace_status(ws_conn) != rsc.RSC_OK:
            raise RuntimeError("a kernel recorded a failure status")
        ms = max_ms(start.elapsed_time(end) / steps)
        search = [p[1].elapsed_time(p[2]) for p in phase]
        rerank = [p[2].elapsed_time(p[3]) for p in phase]
        prep = [p[0].elapsed_time(p[1]) for p in phase]
        conn = [p[3].elapsed_time(p[4]) for p in phase]
        return ms, {"search_ms": statistics.mean(search), "rerank_ms": statistics.mean(rerank),
                    "prep_ms": statistics.mean(prep), "connectivities_ms": statistics.mean(conn)}, \
            (sampler.summary() if sampler else None), ws_knn

    ms, phases, clocks, ws_knn = timed(precision, args.steps, args.warmup, clocks=True)
    scanned, pairs_total = rsc.rsc_knn_scan_stats(n, d, k, ws_knn, metric, precision, locality=args.locality,
                                                  prune=args.prune)
    nnz = int(indptr[-1].item())
    idx_main = idx.clone()
    dist_main = dst.clone()

    # end to end through the public API: pinned host X in, graph out to pinned host memory
    out_host = {
        "idx": torch.empty((n, k), dtype=torch.int32).pin_memory(),
        "dist": torch.empty((n, k), dtype=torch.float32).pin_memory(),
        "indptr": torch.empty(n + 1, dtype=torch.int64).pin_memory(),
        "indices": torch.empty(nnz, dtype=torch.int32).pin_memory(),
        "data": torch.empty(nnz, dtype=torch.float32).pin_memory(),
    }

    # the kNN lists go back to the host on a second stream while the
    # connectivities run
    copy_stream = torch.cuda.Stream(device=dev)
    knn_done = torch.cuda.Event()

    def e2e_step():
        Xd.copy_(X_pin, non_blocking=True)
        rsc.rsc_knn(Xd, k, metric, precision, workspace=ws_knn, out=(idx, dst), locality=args.locality,
                    prune=args.prune)
        knn_done.record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(knn_done)
            out_host["idx"].copy_(idx, non_blocking=True)
            out_host["dist"].copy_(dst, non_blocking=True)
        rsc.rsc_connectivities(idx, dst, nnz_capacity=cap, workspace=ws_conn,
                               out=(indptr, indices, data, rho, sigma))
        out_host["indptr"].copy_(indptr, non_blocking=True)
        out_host["indices"].copy_(indices[:nnz], non_blocking=True)
        out_host["data"].copy_(data[:nnz], non_blocking=True)
        stream.wait_stream(copy_stream)

    e2e_step()
    torch.cuda.synchronize(dev)
    e_start, e_end = make_events(2)
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    e_start.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = max_ms(e_start.elapsed_time(e_end) / e2e_steps)
    h2d = X_pin.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in out_host.values())

    fp32 = None
    if precision != "fp32" and args.fp32_steps > 0:
        f_ms, f_ph, _, _ = timed("fp32", args.fp32_steps, 1)
        fp32 = {"value": job_rate(n, world, f_ms), "ms_per_step": f_ms, "search_ms": f_ph["search_ms"]}

    # roofline of the dominant kernel (candidate search): algorithmic flops =
    # 2 * d per (query, database row) pair computed.  The full scan computes
    # all n^2 pairs; the pruned scan computes the 128 x 256 pairs of each
    # (query tile, database tile) it keeps (rsc_knn_scan_stats), and its time
    # is the whole search phase (window pass, bounds, list pass).
    full_pairs = float(n) * float(n)
    pairs = full_pairs if scanned == pairs_total else float(scanned) * 128.0 * 256.0
    flops = 2.0 * d * pairs
    peaks = _peaks()
    search_s = phases["search_ms"] / 1e3
    achieved = flops / search_s / 1e12
    full_scan = None
    if precision == "bf16" and scanned < pairs_total and args.full_scan_steps > 0:
        fs_ms, fs_ph, _, _ = timed("bf16", args.full_scan_steps, 1, prune="off")
        fs_ach = 2.0 * d * full_pairs / (fs_ph["search_ms"] / 1e3) / 1e12
        full_scan = {"ms_per_step": fs_ms, "search_ms": fs_ph["search_ms"], "value": job_rate(n, world, fs_ms),
                     "achieved_tflops": fs_ach,
                     "frac": fs_ach / (peaks.get("bf16_tflops_sustained") or 1700.0),
                     "note": "same workload with pruning off (every tile pair scanned)"}
    if precision == "bf16":
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        bound, src = "tensor", "bf16_tflops_sustained of measured" if peaks else "fallback 1.7 PFLOP/s"
        kname = "knn_tc.cuh"
    elif precision == "fp8":
        # no FP8 peak is measured: twice the measured BF16 figure (the nominal
        # dense ratio), stated as assumed
        peak = 2.0 * (peaks.get("bf16_tflops_sustained") or 1700.0)
        bound, src = "tensor", "2 x bf16_tflops_sustained of measured (FP8 peak assumed)"
        kname = "knn_tc_fp8.cu"
    else:
        smc = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        peak = 152 * 128 * 2 * smc * 1e6 / 1e12       # FP32 FFMA lanes x 2 flops x max SM clock
        bound, src = "alu", f"FP32 FFMA: 152 SMs x 128 lanes x 2 flop x {smc:.0f} MHz"
        kname = "knn_simt.cuh"
    tr = TRAFFIC.get((kname, "pruned" if scanned < pairs_total else "full"))
    traffic = tr["bytes_per_launch"] if tr and tr.get("kernel_sha") == _kernel_sha(SEARCH_SOURCES) else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "peak_source": src,
                "algorithmic": "2*d flops per (query, row) pair computed: n^2 for the full scan, "
                               "128*256 per kept tile pair when pruned; time = the whole search phase"}

    # the connectivities step is bound by HBM: algorithmic bytes = read idx and
    # dist (8 n k), write indptr (8 (n + 1)), indices and data (8 nnz), rho and
    # sigma (8 n), over its CUDA-event time inside the timed steps
    conn_bytes = 8.0 * n * k + 8.0 * (n + 1) + 8.0 * nnz + 8.0 * n
    conn_gbs = conn_bytes / (phases["connectivities_ms"] / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs") or 6800.0
    ctr = TRAFFIC.get(("connectivities.cu", "graph"))
    roofline_conn = {"bound": "hbm", "achieved": conn_gbs, "peak": hbm, "unit": "GB/s", "frac": conn_gbs / hbm,
                     "traffic": ctr["bytes_per_launch"] if ctr and ctr.get("kernel_sha") == _kernel_sha(CONN_SOURCES)
                     else None,
                     "kernel": "connectivities.cu (smooth, push, match, scan, emit, row sorts)",
                     "peak_source": "hbm_gbs of measured" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
                     "algorithmic": "8nk + 8(n+1) + 8 nnz + 8n bytes per graph over the step's CUDA-event time"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X, idx_main.cpu().numpy(), dist_main.cpu().numpy(), k, args.cpu_seconds)

    if rank == 0:
        value = job_rate(n, world, ms)
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16", "fp8": "e4m3"}.get(precision, "f32"), "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "d": d, "k": k,
                       "precision": f"{precision} candidates + fp32 exact re-rank",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (X 200 MB, operands re-streamed from HBM/L2 each step)",
                       "nnz": nnz,
                       "pruning": {"scanned_tile_pairs": scanned, "total_tile_pairs": pairs_total,
                                   "frac": scanned / pairs_total}},
            "phases_ms": phases,
            "roofline": roofline,
            "roofline_connectivities": roofline_conn,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(n, world, e2e_ms), "unit": "cells/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": launches_per_step(metric, precision, n) * args.steps,
            "clocks": clocks,
        }
        if fp32:
            line["fp32_path"] = fp32
        if full_scan:
            line["full_scan"] = full_scan
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _smi_id(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return dev.index


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


def cpu_baseline(X, gpu_idx, gpu_dist, k, seconds):
    """The FP64 oracle on a bounded query sample, plus recall of the GPU rows."""
    import numpy as np
    import oracle
    from paper_2603_02402_gb300 import synth
    oracle.build()
    n = len(X)
    t0 = time.perf_counter()
    oracle.knn(X, k, queries=synth.query_sample(n, 16, seed=77))
    t16 = time.perf_counter() - t0
    m = int(min(n, max(64, 16 * seconds / max(t16, 1e-3))))
    q = synth.query_sample(n, m, seed=5)
    t0 = time.perf_counter()
    oi, od, _ = oracle.knn(X, k, queries=q)
    dt = time.perf_counter() - t0
    gi = gpu_idx[q]
    dex = exact_distances(X, q, gi)
    rel = np.abs(gpu_dist[q] - dex) / np.maximum(dex, 1e-30)
    return {"value": m / dt, "unit": "cells/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{m} seeded query rows against all {n} rows (kNN stage, FP64 brute force)",
            "recall_at_k": recall_by_distance(dex, od[:, -1]), "id_exact": float((gi == oi).mean()),
            "max_rel_dist_err": float(np.where(dex > 0, rel, 0).max())}


BATCHED_WORKLOAD = ("Batched: 64 samples, log-uniform sizes 2,000-200,000 (~3M cells) x 50 PCs fp32, "
                    "30-cluster mixtures with per-sample offsets ~N(0,0.5I); per-sample k=15 plus k=3 from every "
                    "sample, BF16 candidates + FP32 re-rank, one persistent launch replayed from a CUDA graph")


def run_batched(args):
    """Batched workload: cells/s of one rsc_knn_batched call (CUDA-graph replay)."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    sizes = synth.batched_sizes(64, seed=rank)
    X, off = synth.batched(sizes, d=50, n_comp=30, seed=rank)
    n = len(X)
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.Stream(dev)
    kw, kx = 15, 3
    ws = torch.empty(rsc.rsc_knn_batched_workspace_size(n, 50, off, kw, kx), dtype=torch.uint8, device=dev)
    out = (torch.empty((n, kw), dtype=torch.int32, device=dev), torch.empty((n, kw), device=dev),
           torch.empty((n, 64 * kx), dtype=torch.int32, device=dev), torch.empty((n, 64 * kx), device=dev))
    with torch.cuda.stream(stream):
        # autotuner (column parts x pipeline stages, timed on this data); the
        # timed calls below use automatic options, which follow its choice
        tuned, tune_ms, _ = rsc.rsc_autotune_knn_batched(Xd, off, kw, kx, stream=stream, trials=1)
        for _ in range(args.warmup):
            rsc.rsc_knn_batched(Xd, off, kw, kx, stream=stream, workspace=ws, out=out)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(_smi_id(dev))
        sampler.__enter__()
        a.record(stream)
        for _ in range(args.steps):
            rsc.rsc_knn_batched(Xd, off, kw, kx, stream=stream, workspace=ws, out=out)
        b.record(stream)
        stream.synchronize()
        sampler.__exit__()
    if rsc.rsc_workspace_status(ws, stream) != rsc.RSC_OK:
        raise RuntimeError("a kernel recorded a failure status")
    ms = a.elapsed_time(b) / args.steps
    # pairs of (128-row query tile, 256-row database tile of one sample) the search computed
    scanned, total = rsc.rsc_knn_batched_scan_stats(n, 50, off, kw, kx, ws, stream=stream)
    flops = 2.0 * 50 * float(scanned) * 128.0 * 256.0
    peak = _peaks().get("bf16_tflops_sustained") or 1700.0
    line = {"metric": "batched kNN cells/s (64 samples, k_within=15, k_cross=3 from every sample)",
            "value": n / (ms / 1e3), "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "config": {"workload": BATCHED_WORKLOAD, "n": n, "samples": 64,
                                            "sizes_min_max": [int(sizes.min()), int(sizes.max())],
                                            "pruning": {"scanned_tile_pairs": scanned, "total_tile_pairs": total,
                                                        "frac": scanned / total}},
            "roofline": {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / peak, "traffic": None,
                         "kernel": "knn_tc_kernel (batched)",
                         "note": "whole call (prep + pruned search + both re-ranks) timed; 2*d flops per "
                                 "(query, row) pair computed: 128*256 per scanned tile pair"},
            # prep 3, ordering 36 + 2 chains + 5 (sample-preserving partition), BF16 operands 1,
            # pruned search 10 (2 sphere passes, nearest tiles, window pass, tau, count, scan (2),
            # fill, list pass), gather + within re-rank + cross re-rank 3; 7 without the ordering
            # (fewer than ORDER_MIN_ROWS rows)
            "gpu_launches": (60 if n >= ORDER_MIN_ROWS else 7) * args.steps, "clocks": sampler.summary(),
            "autotune": {"choice": tuned, "best_ms": tune_ms}}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batched_baseline(X, off, kw, kx, out)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_baseline(X, off, kw, kx, out):
    """The FP64 oracle on the five smallest samples (their rows against
    themselves, within and across those samples), with the recall of the GPU's
    lists for those rows: within-sample lists as they are, cross lists
    restricted to the five samples."""
    import numpy as np
    import oracle
    oracle.build()
    sizes = np.diff(off)
    pick = np.sort(np.argsort(sizes, kind="stable")[:5])
    rows = np.concatenate([np.arange(off[s], off[s + 1]) for s in pick])
    sub_off = np.concatenate([[0], np.cumsum(sizes[pick])])
    t0 = time.perf_counter()
    wi, wd, xi, xd = oracle.batched_knn(X[rows], sub_off, kw, kx)
    dt = time.perf_counter() - t0
    gw = out[1].cpu().numpy()[rows].astype(np.float64)
    within = float((gw <= wd[:, -1:] * (1 + 1e-6) + 1e-12).mean())
    # the GPU's k_cross nearest of each picked sample, for the picked rows
    gi_all = out[2].cpu().numpy()[rows]
    gd_all = out[3].cpu().numpy()[rows].astype(np.float64)
    ok = tot = 0
    for t, s in enumerate(pick):
        lo, hi = off[s], off[s + 1]
        # oracle distances of sample t's k_cross nearest (sorted rows mix samples: select by sample)
        sel = (xi >= sub_off[t]) & (xi < sub_off[t + 1])
        ref = np.where(sel, xd, np.inf)
        kth = np.sort(ref, axis=1)[:, kx - 1]
        mine = np.where((gi_all >= lo) & (gi_all < hi), gd_all, np.inf)
        got = np.sort(mine, axis=1)[:, :kx]
        ok += int((got <= kth[:, None] * (1 + 1e-6) + 1e-12).sum())
        tot += got.size
    return {"value": len(rows) / dt, "unit": "cells/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the 5 smallest samples ({len(rows)} rows): per-sample k={kw} and k_cross={kx} from each "
                      f"of the 5, FP64 brute force",
            "recall_within": within, "recall_cross": ok / max(tot, 1)}


PARTITION_WORKLOAD = ("Learned partitioner: 5,000,000 cells x 50 PCs fp32, 200-cluster mixture with random anisotropic "
                      "covariances (eigenvalues log-uniform 0.05-2), k=15; MLP 50->256->256->1024 parts (BF16 weights, "
                      "FP32 accumulation) trained on exact kNN lists of a 200k subsample; top-8 parts probed")


def run_partitioner(args):
    """Partitioned kNN graph of every cell (probe 8 of 1024 parts) + connectivities,
    against the exact BF16 path on the same GPU as the reference for recall."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n = args.n if args.n != 1_000_000 else 5_000_000
    k, probes = args.k, 8
    X = synth.anisotropic(n, 50, 200, seed=rank)
    Xd = torch.from_numpy(X).to(dev)
    train = torch.from_numpy(synth.query_sample(n, min(200_000, n // 5), seed=11).astype(np.int32)).to(dev)
    part = rsc.Partitioner(50, 1024, 256, bf16_weights=True, seed=rank)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record()
    loss = part.train(Xd, train, k=k, kmeans_iters=10, epochs=10, batch=1024, lr=1e-3)
    ev[1].record()
    torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    # exact BF16 path (the reference for recall)
    ws_exact = torch.empty(rsc.rsc_knn_workspace_size(n, 50, k, "euclidean", "bf16"), dtype=torch.uint8, device=dev)
    ev[2].record()
    ei, ed = rsc.rsc_knn(Xd, k, precision="bf16", workspace=ws_exact)
    ev[3].record()
    torch.cuda.synchronize()
    exact_ms = ev[2].elapsed_time(ev[3])
    del ws_exact
    ws = torch.empty(part.workspace_size(n, 0, k, n, probes), dtype=torch.uint8, device=dev)
    cap = rsc.rsc_connectivities_max_nnz(n, k)
    ws_conn = torch.empty(rsc.rsc_connectivities_workspace_size(n, k), dtype=torch.uint8, device=dev)
    out = (torch.empty((n, k), dtype=torch.int32, device=dev), torch.empty((n, k), device=dev))
    csr = (torch.empty(n + 1, dtype=torch.int64, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
           torch.empty(cap, device=dev), torch.empty(n, device=dev), torch.empty(n, device=dev))

    def step(routing="network"):
        part.knn(Xd, k=k, n_probe=probes, routing=routing, workspace=ws, out=out)
        rsc.rsc_connectivities(out[0], out[1], nnz_capacity=cap, workspace=ws_conn, out=csr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    ev[4].record()
    for _ in range(args.steps):
        step()
    ev[5].record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = ev[4].elapsed_time(ev[5]) / args.steps
    thr = ed[:, -1:] * (1 + 1e-6)
    recall = float((out[1] <= thr).float().mean())
    # recall against the exact path for 1, 2, 4 and 8 probed parts, with the
    # network's routing and with nearest-centroid routing (same parts, same
    # candidate budget: the method without the network)
    curves = {"network": {}, "centroids": {}}
    for routing in ("network", "centroids"):
        for pr in (1, 2, 4, 8):
            part.knn(Xd, k=k, n_probe=pr, routing=routing, workspace=ws, out=out)
            torch.cuda.synchronize()
            curves[routing][pr] = float((out[1] <= thr).float().mean())
    recall_c = curves["centroids"][probes]
    line = {"metric": "partitioned neighbors graph cells/s (5M cells, 50 PCs, k=15, 8 of 1024 parts probed)",
            "value": n / (ms / 1e3), "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "config": {"workload": PARTITION_WORKLOAD, "n": n, "k": k, "probes": probes},
            "recall_at_k_vs_exact": recall, "recall_at_k_centroid_routing": recall_c,
            "recall_vs_probes": curves,
            "exact_bf16_knn_ms": exact_ms, "exact_bf16_cells_per_s": n / (exact_ms / 1e3),
            "train_ms": train_ms, "train_final_loss": loss, "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


COSINE_WORKLOAD = ("Large exact graph: 11,000,000 cells x 50 PCs fp32 (~2.2 GB), 500-cluster mixture with PC variance "
                   "1/t, cosine metric (rows L2-normalised), k=30, BF16 candidates with FP32 re-rank of 128, "
                   "then the full connectivities CSR")


def run_cosine(args):
    """11M-cell cosine graph (k=30): one rsc_knn + rsc_connectivities per step."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n = args.n if args.n != 1_000_000 else 11_000_000
    k = 30
    X = synth.mixture(n, 50, n_comp=500, seed=rank)
    Xd = torch.from_numpy(X).to(dev)
    cands = args.candidates or 128   # 64 candidates give recall@30 ~0.97 here; 128 give ~0.998
    ws = torch.empty(rsc.rsc_knn_workspace_size(n, 50, k, "cosine", "bf16", cands), dtype=torch.uint8, device=dev)
    cap = rsc.rsc_connectivities_max_nnz(n, k)
    ws_conn = torch.empty(rsc.rsc_connectivities_workspace_size(n, k), dtype=torch.uint8, device=dev)
    out = (torch.empty((n, k), dtype=torch.int32, device=dev), torch.empty((n, k), device=dev))
    csr = (torch.empty(n + 1, dtype=torch.int64, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
           torch.empty(cap, device=dev), torch.empty(n, device=dev), torch.empty(n, device=dev))

    def step():
        rsc.rsc_knn(Xd, k, "cosine", "bf16", candidates=cands, workspace=ws, out=out)
        rsc.rsc_connectivities(out[0], out[1], nnz_capacity=cap, workspace=ws_conn, out=csr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    a.record()
    for _ in range(args.steps):
        step()
    b.record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = a.elapsed_time(b) / args.steps
    scanned, pairs_total = rsc.rsc_knn_scan_stats(n, 50, k, ws, "cosine", "bf16", candidates=cands)
    pairs = float(scanned) * 128.0 * 256.0 if scanned < pairs_total else float(n) * float(n)
    flops = 2.0 * 50 * pairs
    peak = _peaks().get("bf16_tflops_sustained") or 1700.0
    line = {"metric": "cosine neighbors graph cells/s (11M cells, 50 PCs, k=30)", "value": n / (ms / 1e3),
            "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": COSINE_WORKLOAD, "n": n, "k": k, "candidates": cands,
                       "nnz": int(csr[0][-1].item()),
                       "pruning": {"scanned_tile_pairs": scanned, "total_tile_pairs": pairs_total,
                                   "frac": scanned / pairs_total}},
            "roofline": {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / peak, "traffic": None,
                         "note": "whole step timed (ordering, search, re-rank, connectivities); 2*d flops per "
                                 "(query, row) pair computed: 128*256 per scanned tile pair"},
            "gpu_launches": launches_per_step("cosine", "bf16", n) * args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        q = synth.query_sample(n, 256, seed=5)   # about 30 s of the oracle on 16 cores
        t0 = time.perf_counter()
        oi, od, _ = oracle.knn(X, k, metric=oracle.COSINE, queries=q)
        dt = time.perf_counter() - t0
        gi = out[0].cpu().numpy()[q]
        gd = out[1].cpu().numpy()[q].astype(np.float64)
        dex = exact_distances(X, q, gi, "cosine")
        line["cpu_baseline"] = {"value": len(q) / dt, "unit": "cells/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"{len(q)} seeded query rows against all {n} rows"}
        line["recall_at_k_vs_oracle"] = recall_by_distance(dex, od[:, -1])
        line["max_abs_dist_err"] = float(np.abs(gd - dex).max())
    if rank == 0:
        print(json.dumps(line), flush=True)


UMAP_WORKLOAD = ("UMAP layout of the 1,000,000-cell graph (the headline workload's BF16+rerank kNN, k=15, and its "
                 "fuzzy union, built untimed): 200 epochs (scanpy's count above 10,000 cells), 2-D, 5 negatives "
                 "per sample, a, b from spread 1 / min_dist 0.5, learning rate 1, initial layout = the first two "
                 "PCs scaled to [-10, 10]")
UMAP_SOURCES = ("umap.cu",)


def run_umap(args):
    """UMAP layout workload: cells/s of one 200-epoch rsc_umap_layout call (one GPU; under torchrun each
    rank lays out its own graph and rank 0 reports its own)."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n, d, k, N, r = args.n, 50, args.k, args.epochs, 5
    X = synth.mixture(n, d, n_comp=100, seed=rank)
    Xd = torch.from_numpy(X).to(dev)
    idx, dst = rsc.rsc_knn(Xd, k, "euclidean", "bf16")
    ip, ind, dat, _, _ = rsc.rsc_connectivities(idx, dst)
    nnz = int(ip[-1].item())
    ind, dat = ind[:nnz].contiguous(), dat[:nnz].contiguous()
    del idx, dst
    a, b = rsc.rsc_umap_find_ab(1.0, 0.5)
    init = Xd[:, :2].contiguous()
    init = (init * (10.0 / init.abs().max())).contiguous()
    emb = torch.empty_like(init)
    ws = torch.empty(rsc.rsc_umap_workspace_size(n, nnz, 2), dtype=torch.uint8, device=dev)

    def step():
        emb.copy_(init)
        rsc.rsc_umap_layout(ip, ind, dat, emb, a, b, n_epochs=N, negative_sample_rate=r, nnz=nnz, seed=7,
                            workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    ev[0].record()
    for _ in range(args.steps):
        step()
    ev[1].record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = ev[0].elapsed_time(ev[1]) / args.steps

    # end to end through host buffers: graph and initial layout in from pinned memory, layout out
    h_ip, h_ind, h_dat = ip.cpu().pin_memory(), ind.cpu().pin_memory(), dat.cpu().pin_memory()
    h_init, h_out = init.cpu().pin_memory(), torch.empty_like(init, device="cpu").pin_memory()
    g_ip, g_ind, g_dat, g_emb = torch.empty_like(ip), torch.empty_like(ind), torch.empty_like(dat), torch.empty_like(init)

    def e2e_step():
        g_ip.copy_(h_ip, non_blocking=True)
        g_ind.copy_(h_ind, non_blocking=True)
        g_dat.copy_(h_dat, non_blocking=True)
        g_emb.copy_(h_init, non_blocking=True)
        rsc.rsc_umap_layout(g_ip, g_ind, g_dat, g_emb, a, b, n_epochs=N, negative_sample_rate=r, nnz=nnz, seed=7,
                            workspace=ws)
        h_out.copy_(g_emb, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 5))
    ev[0].record()
    for _ in range(e2e_steps):
        e2e_step()
    ev[1].record()
    torch.cuda.synchronize()
    e2e_ms = ev[0].elapsed_time(ev[1]) / e2e_steps
    assert torch.equal(h_out, emb.cpu()), "end-to-end layout differs from the device-resident one"
    h2d = 8 * (n + 1) + 8 * nnz + 8 * n
    d2h = 8 * n

    # roofline of the epoch kernel: streamed bytes per epoch (f and column per entry, row pointers,
    # positions read and written); the gathered positions come from L2 (8 MB of positions)
    h_w = dat.cpu().numpy()
    f = h_w / h_w.max()
    samples = float(np.floor(np.float32(N) * f.astype(np.float32)).sum())   # entries sampled over the N epochs
    per_epoch_bytes = 8.0 * nnz + 8.0 * (n + 1) + 2 * 8.0 * n
    achieved = per_epoch_bytes * N / (ms / 1e3) / 1e9
    peaks = _peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    sha = _kernel_sha(UMAP_SOURCES)
    tr = TRAFFIC.get(("umap.cu", "epoch"))
    traffic = tr["bytes_per_launch"] if tr and tr["kernel_sha"] == sha else None
    line = {"metric": "UMAP layout cells/s (1M-cell k=15 graph, 200 epochs, 2-D)", "value": n / (ms / 1e3),
            "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": UMAP_WORKLOAD, "n": n, "nnz": nnz, "epochs": N, "negative_sample_rate": r,
                       "dim": 2, "a": a, "b": b,
                       "l2": "graph streamed from HBM every epoch (8 B per entry, 182 MB > L2); the 8 MB of "
                             "positions stay in L2",
                       "samples_per_epoch": samples / N},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "kernel": "umap.cu (umap_epoch_kernel)",
                         "peak_source": "hbm_gbs of measured" if peaks.get("hbm_gbs") else "fallback",
                         "algorithmic": "per epoch 8 nnz + 8 (n + 1) + 16 n bytes (f and column per entry, row "
                                        "pointers, positions in and out) over the call's CUDA-event time / epochs",
                         "gathers_per_epoch": samples / N * (2 + r),
                         "ns_per_sample": ms * 1e6 / samples},
            "e2e": {"value": n / (e2e_ms / 1e3), "unit": "cells/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": (N + 4) * args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        h_ip, h_ind = ip.cpu().numpy(), ind.cpu().numpy()
        Y = init.cpu().numpy()
        e_run = 2
        t0 = time.perf_counter()
        oracle.umap_epochs(h_ip, h_ind, h_w, Y, a, b, neg_rate=r, n_epochs=N, first=100, last=100 + e_run - 1,
                           seed=7)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / (dt * N / e_run), "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": f"epochs 100-{100 + e_run - 1} of the {N} on the full graph (FP64, one "
                                          "thread), extrapolated to the whole layout"}
    if rank == 0:
        print(json.dumps(line), flush=True)


ED_WORKLOAD = ("E-distance of a perturbation screen: 300,000 cells x 50 PCs fp32 (60-cluster mixture), 2,000 "
               "groups of log-uniform sizes 20-2,000 in a permuted cell index, every group pair a <= b "
               "(4.5e10 cell pairs), split-BF16 tensor-core distances")


def run_edistance(args):
    """E-distance workload: cell-pair distances per second of one all-pairs rsc_edistance call."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n_cells = args.n if args.n != 1_000_000 else 300_000
    G = 2000
    sizes = synth.batched_sizes(G, lo=20, hi=2000, total=n_cells, seed=rank)
    n = int(sizes.sum())
    X = synth.mixture(n, 50, n_comp=60, seed=rank)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ci = np.random.default_rng(rank).permutation(n).astype(np.int32)
    Xd, cd = torch.from_numpy(X).to(dev), torch.from_numpy(ci).to(dev)
    ws = torch.empty(rsc.rsc_edistance_workspace_size(n, 50, off), dtype=torch.uint8, device=dev)
    pairs = float(n) * (n - 1) / 2   # every cell pair lies in exactly one group pair a <= b

    def step():
        return rsc.rsc_edistance(Xd, off, cd, workspace=ws, with_mean=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    ev[0].record()
    for _ in range(args.steps):
        sums, _, E = step()
    ev[1].record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = ev[0].elapsed_time(ev[1]) / args.steps

    # end to end: rows and cell index in from pinned memory, E out
    hX, hc = torch.from_numpy(X).pin_memory(), torch.from_numpy(ci).pin_memory()
    hE = torch.empty((G, G), dtype=torch.float64).pin_memory()
    gX, gc = torch.empty_like(Xd), torch.empty_like(cd)

    def e2e_step():
        gX.copy_(hX, non_blocking=True)
        gc.copy_(hc, non_blocking=True)
        _, _, Eo = rsc.rsc_edistance(gX, off, gc, workspace=ws, with_mean=False)
        hE.copy_(Eo, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 5))
    ev[0].record()
    for _ in range(k):
        e2e_step()
    ev[1].record()
    torch.cuda.synchronize()
    e2e_ms = ev[0].elapsed_time(ev[1]) / k

    peaks = _peaks()
    clk = (sampler.summary() or {}).get("sm_mhz") or 2070.0
    sfu_peak = 152 * 16 * clk * 1e6 / 1e12   # square roots per second (T/s): 16 per SM per clock
    achieved = pairs / (ms / 1e3) / 1e12
    tiles = 0
    T = (n + 127) // 128
    tiles = T * (T + 1) // 2
    tflops = 2.0 * 128 * 128 * 192 * tiles / (ms / 1e3) / 1e12
    line = {"metric": "E-distance cell-pair distances/s (300k cells, 2,000 groups, 50 PCs, all pairs)",
            "value": pairs / (ms / 1e3), "unit": "distances/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": ED_WORKLOAD, "n": n, "groups": G, "d": 50, "cell_pairs": pairs,
                       "tile_pairs": tiles,
                       "l2": "operands (230 MB) stream from HBM/L2 per query tile; the G x G sums stay in L2"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": sfu_peak, "unit": "Tsqrt/s",
                         "frac": achieved / sfu_peak,
                         "traffic": (TRAFFIC[("edist.cu", "screen")]["bytes_per_launch"]
                                     if n == 299977 and _kernel_sha(ED_SOURCES) == TRAFFIC[("edist.cu", "screen")]["kernel_sha"]
                                     else None),
                         "kernel": "edist.cu (edist_tc_kernel)",
                         "peak_source": "derived: 152 SMs x 16 special-function results per clock x median SM clock",
                         "algorithmic": "one square root per cell pair (n (n - 1) / 2) over the call's CUDA-event time",
                         "tensor_tflops_executed": tflops,
                         "tensor_frac_of_measured_bf16": tflops / (peaks.get("bf16_tflops_sustained") or 1729.0)},
            "e2e": {"value": pairs / (e2e_ms / 1e3), "unit": "distances/s",
                    "h2d_bytes_per_step": int(X.nbytes + ci.nbytes), "d2h_bytes_per_step": int(G * G * 8),
                    "ms_per_step": e2e_ms},
            "gpu_launches": 4 * args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rng = np.random.default_rng(3)
        a, b = rng.integers(0, G, 24), rng.integers(0, G, 24)
        pl = np.stack([np.minimum(a, b), np.maximum(a, b)], 1).astype(np.int32)
        cnt = sum(float(sizes[p]) * (sizes[q] if p != q else (sizes[p] - 1) / 2) for p, q in pl)
        t0 = time.perf_counter()
        ref = oracle.edistance_sums(X, off, ci, pairs=pl)
        dt = time.perf_counter() - t0
        got = sums.cpu().numpy()
        rel = max(abs(got[p, q] - ref[p, q]) / abs(ref[p, q]) for p, q in pl if ref[p, q] != 0)
        line["cpu_baseline"] = {"value": cnt / dt, "unit": "distances/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"24 seeded group pairs ({cnt:.3g} cell pairs, FP64 "
                                                            "direct differences)",
                                "max_rel_sum_diff": float(rel)}
    if rank == 0:
        print(json.dumps(line), flush=True)


NND_WORKLOAD = ("Approximate kNN by NN-descent: 1,000,000 cells x 50 PCs fp32 (100-cluster mixture, PC variance "
                "1/i), k=15 (self included), hashed initial lists, 15 new samples, 32 reverse and 64 candidate slots "
                "per cell, 8 iterations at most, stop below 0.001 n k changes; FP32 joins")


def run_nndescent(args):
    """NN-descent workload: cells/s of one rsc_knn_descent call (the paper's CPU
    neighbour search is PyNNDescent), with recall against the oracle's exact kNN."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n, k, d, T = args.n, args.k, 50, 8
    X = synth.mixture(n, d, n_comp=100, seed=rank)
    Xd = torch.from_numpy(X).to(dev)
    opts = rsc.nnd_opts(max_iters=T, delta=0.001, seed=0)
    ws = torch.empty(rsc.rsc_knn_descent_workspace_size(n, d, k, opts), dtype=torch.uint8, device=dev)

    def step():
        return rsc.rsc_knn_descent(Xd, k, max_iters=T, delta=0.001, seed=0, workspace=ws, with_changes=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    ev[0].record()
    for _ in range(args.steps):
        idx, dist, ch = step()
    ev[1].record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    pairs = rsc.rsc_knn_descent_pairs(ws)
    changes = ch.cpu().numpy()
    iters = int((changes > 0).sum())

    # end to end: rows in from pinned memory, lists out to pinned memory
    hX = torch.from_numpy(X).pin_memory()
    hI = torch.empty((n, k), dtype=torch.int32).pin_memory()
    hD = torch.empty((n, k), dtype=torch.float32).pin_memory()
    gX = torch.empty_like(Xd)

    def e2e_step():
        gX.copy_(hX, non_blocking=True)
        i2, d2 = rsc.rsc_knn_descent(gX, k, max_iters=T, delta=0.001, seed=0, workspace=ws)
        hI.copy_(i2, non_blocking=True)
        hD.copy_(d2, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ke = max(1, min(args.steps, 3))
    ev[0].record()
    for _ in range(ke):
        e2e_step()
    ev[1].record()
    torch.cuda.synchronize()
    e2e_ms = ev[0].elapsed_time(ev[1]) / ke

    clk = (sampler.summary() or {}).get("sm_mhz") or 2070.0
    lane_peak = 152 * 128 * clk * 1e6 / 1e12   # FP32 lane operations per second (T/s)
    lane_ops = float(pairs.sum()) * 2 * d      # a subtraction and a fused multiply-add per coordinate and pair
    line = {"metric": "approximate kNN cells/s by NN-descent (1M cells, 50 PCs, k=15)",
            "value": n / (ms / 1e3), "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": NND_WORKLOAD, "n": n, "k": k, "d": d, "iterations_run": iters,
                       "changes_per_iteration": changes[:T].tolist(), "pairs_joined": pairs[:T].tolist(),
                       "l2": "X (200 MB) exceeds L2; the slot arrays (768 MB) are touched at random"},
            "roofline": {"bound": "alu", "achieved": lane_ops / (ms / 1e3) / 1e12, "peak": lane_peak,
                         "unit": "T FP32 lane-ops/s", "frac": lane_ops / (ms / 1e3) / 1e12 / lane_peak,
                         "traffic": (TRAFFIC[("nndescent.cu", "call")]["bytes_per_launch"]
                                     if n == 1_000_000 and _kernel_sha(NND_SOURCES) == TRAFFIC[("nndescent.cu", "call")]["kernel_sha"]
                                     else None),
                         "traffic_note": "DRAM bytes of the call's eight join launches (ncu, cold cache): "
                                         "1.8 TB/s over the call, the join's staged rows and slot offers",
                         "kernel": "nndescent.cu (join_kernel)",
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x median SM clock",
                         "algorithmic": "2 d lane operations (subtract, fused multiply-add) per joined pair, "
                                        "pairs counted by the kernel, over the whole call's CUDA-event time "
                                        "(the join kernel is most of it: see the launch list)"},
            "e2e": {"value": n / (e2e_ms / 1e3), "unit": "cells/s", "h2d_bytes_per_step": int(X.nbytes),
                    "d2h_bytes_per_step": int(n * k * 8), "ms_per_step": e2e_ms},
            "gpu_launches": (2 + 3 * T) * args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # recall against the oracle's exact lists on a seeded query sample
        q = synth.query_sample(n, 1000, seed=5)
        want, wd, _ = oracle.knn(X, k, queries=q)
        gi = idx.cpu().numpy()[q]
        dex = exact_distances(X, q, gi)
        # the oracle's own NN-descent, timed on a bounded subset of the cells
        m = min(n, 40_000)
        t0 = time.perf_counter()
        oracle.nndescent(X[:m], k, iters=T, delta=0.001, seed=0)
        dt = time.perf_counter() - t0
        line["recall_at_k"] = recall_by_distance(dex, wd[:, -1])
        line["cpu_baseline"] = {"value": m / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": f"the oracle's NN-descent on the first {m} cells (same parameters; "
                                          "recall_at_k: 1,000 seeded queries against the oracle's exact kNN)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


LD_WORKLOAD = ("Leiden communities of the headline neighbourhood graph: 1,000,000 cells x 50 PCs (100-cluster "
               "mixture), k=15 BF16+re-rank kNN and fuzzy connectivities built untimed by the library "
               "(22.8M entries), modularity, resolution 1, two runs (scanpy's count)")


def run_leiden(args):
    """Leiden workload: cells/s of one rsc_leiden call on the 1M-cell graph."""
    import numpy as np
    import torch
    from paper_2603_02402_gb300 import rsc, synth

    world, rank, local = setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rsc.lib()
    n, k = args.n, args.k
    X = synth.mixture(n, 50, n_comp=100, seed=rank)
    idx, dist = rsc.rsc_knn(torch.from_numpy(X).to(dev), k, precision="bf16")
    ip, ind, dat, _, _ = rsc.rsc_connectivities(idx, dist)
    torch.cuda.synchronize()
    nnz = int(ip[-1])
    ind, dat = ind[:nnz].contiguous(), dat[:nnz].contiguous()
    del idx, dist
    ws = torch.empty(rsc.rsc_leiden_workspace_size(n, nnz), dtype=torch.uint8, device=dev)

    def step():
        return rsc.rsc_leiden(ip, ind, dat, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(_smi_id(dev))
    sampler.__enter__()
    ev[0].record()
    for _ in range(args.steps):
        mem, K, Q = step()
    ev[1].record()
    torch.cuda.synchronize()
    sampler.__exit__()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    st = rsc.rsc_leiden_last_stats()

    # end to end: the graph in from pinned memory, the membership out
    hip, hind, hdat = ip.cpu().pin_memory(), ind.cpu().pin_memory(), dat.cpu().pin_memory()
    hmem = torch.empty(n, dtype=torch.int32).pin_memory()
    gip, gind, gdat = torch.empty_like(ip), torch.empty_like(ind), torch.empty_like(dat)

    def e2e_step():
        gip.copy_(hip, non_blocking=True)
        gind.copy_(hind, non_blocking=True)
        gdat.copy_(hdat, non_blocking=True)
        m2, _, _ = rsc.rsc_leiden(gip, gind, gdat, workspace=ws)
        hmem.copy_(m2, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ke = max(1, min(args.steps, 3))
    ev[0].record()
    for _ in range(ke):
        e2e_step()
    ev[1].record()
    torch.cuda.synchronize()
    e2e_ms = ev[0].elapsed_time(ev[1]) / ke

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6787.6
    moved = 16.0 * st["entries"] + 32.0 * st["vertices"]   # bytes the rounds read at least
    achieved = moved / (ms / 1e3) / 1e9
    line = {"metric": "Leiden cells/s (1M-cell neighbourhood graph, modularity, resolution 1)",
            "value": n / (ms / 1e3), "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": LD_WORKLOAD, "n": n, "nnz": nnz, "communities": K, "modularity": Q,
                       "work": st, "l2": "the level-0 graph (273 MB with 64-bit weights) exceeds L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "leiden.cu (move_kernel, inner/pick_kernel)",
                         "peak_source": "hbm_gbs of measured",
                         "algorithmic": "16 bytes per graph entry (column, 64-bit weight, the neighbour's label) and "
                                        "32 per vertex (row pointers, strength, labels, totals) for every moving "
                                        "round, twice per refinement round, over the call's CUDA-event time"},
            "e2e": {"value": n / (e2e_ms / 1e3), "unit": "cells/s",
                    "h2d_bytes_per_step": int(hip.numel() * 8 + hind.numel() * 4 + hdat.numel() * 4),
                    "d2h_bytes_per_step": int(n * 4), "ms_per_step": e2e_ms},
            "gpu_launches": int(st["launches"]) * args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        from scipy import spatial
        oracle.build()
        m = 100_000
        Xs = synth.mixture(m, 8, n_comp=40, seed=11)
        dd, ii = spatial.cKDTree(Xs.astype(np.float64)).query(Xs.astype(np.float64), k, workers=-1)
        g = oracle.connectivities(ii.astype(np.int32), dd.astype(np.float32).astype(np.float64))
        t0 = time.perf_counter()
        oracle.leiden(g["indptr"], g["indices"], g["data"].astype(np.float32))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": f"the oracle's Leiden on a {m}-cell graph (k-d tree lists of an "
                                          "8-dimensional 40-cluster mixture, the oracle's connectivities)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "partitioner":
        run_partitioner(args)
    elif args.workload == "cosine":
        run_cosine(args)
    elif args.workload == "umap":
        run_umap(args)
    elif args.workload == "edistance":
        run_edistance(args)
    elif args.workload == "nndescent":
        run_nndescent(args)
    elif args.workload == "leiden":
        run_leiden(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
