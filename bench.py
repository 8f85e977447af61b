#!/usr/bin/env python
"""Benchmark of the CLR product (Calvin, Lewis & Valeev, Section 4.1) on one GB300.

Workload: the all-dense CLR product C = A B with N = 16384 split into 96 uneven clusters
(sizes U[128, 224] rescaled), A and B i.i.d. N(0,1) FP64 -- every block is dense, so the
product is ordinary dense matrix multiplication (the eps -> 0 limit, Section 4.3), computed in
split-precision bf16x3 on the tensor cores with FP32 accumulation in short segments and an
FP64 epilogue.  A step is one whole CLR product through the library (triple list, staging of
the bf16 term panels, the dense tile products, low-rank/recompression passes, norms).

Prints one JSON line (rank 0), which also carries Newton-Schulz timings (1D chain, 3D lattice
overlap and Coulomb-like matrices) and the batched configuration (64 chain products of uneven
size replayed as one CUDA graph, measured in a child process).  `--impl reference` times the
FP64 CPU oracle instead, on a bounded sample of the same workload.  Multi-GPU runs (torchrun) are independent replicas:
each rank multiplies its own matrices, nothing is exchanged between ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CLR multiply TFLOP/s and ms per Newton–Schulz S^-1/2 iteration at stated error"

# DRAM bytes (read + write) of one launch of the dense tile-product kernel at this workload,
# from ncu counters, keyed by the kernel source's hash so that the number is dropped
# (traffic: null) as soon as the kernel changes.  Counters are taken on the N = 8192 case of the
# same construction (48 clusters; 2.281 GB read, 0.896 GB written per launch) and scaled to
# N = 16384 by the units each part grows with: panel reads by the tile-k steps (N^3, x8), C
# writes by the output (N^2, x4).
MEASURED_TRAFFIC = {
    "a7f5dda373a2:bf16x3:16384:96": 8 * 2280723456 + 4 * 896034816,
}
# Truncation of the Newton-Schulz iterates on the lattice matrices: the matrix is built at
# eps_lr = 1e-6, but iterates truncated at 1e-6 hold the residual ||alpha Z S Z - I||_F/sqrt(N)
# near 1.8e-5 (the oracle floors at the same level); at 1e-8 the residual meets 1e-6.
EPS_NS_LATTICE = 1e-8
PAIRS = {"bf16x3": 3, "bf16x6": 6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "bf16x6", "fp64"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--clusters", type=int, default=96)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ns", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-products measurement (64 products, one CUDA graph)")
    ap.add_argument("--ns-prec", default="fp64", choices=["bf16x3", "bf16x6", "fp64"])
    ap.add_argument("--ns-lattice", default="8x8x4",
                    help="lattice sites of the 3D overlap NS measurement (16 points per site), "
                         "or 'none'")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain-FP64 product of the same workload")
    ap.add_argument("--no-chain", action="store_true",
                    help="skip the N = 2048 1D-chain product (FP64 and split)")
    ap.add_argument("--ns-lattice-large", default="8x8x8",
                    help="lattice sites of a second, larger overlap NS measurement (timed run "
                         "only), or 'none'")
    return ap.parse_args()


def workload(args, rank=0):
    from paper_1509_00309_gb300 import workloads as wl
    return wl.dense_normal(n=args.n, n_clusters=args.clusters, lo=128, hi=224,
                           seed=wl.default_seed(1) + 1000 * rank)


def config(args):
    """The workload (identical for both arms)."""
    return {"workload": "all-dense CLR product N=%d, %d uneven clusters U[128,224], "
                        "A,B ~ N(0,1) FP64" % (args.n, args.clusters),
            "n": args.n, "clusters": args.clusters, "precision": args.prec,
            "l2": "inputs larger than L2 (A, B 2.1 GB FP64 each + bf16 term panels); no flush",
            "parallelism": "replicas"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(backend=None):
    """One process per GPU under torchrun (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from the
    environment).  Returns (rank, world_size, local_rank)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if backend is None:
            backend = "nccl"
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        return dist.get_rank(), ws, local
    return 0, 1, 0


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device="cuda"):
    """The slowest rank's value (timings are taken as the max over ranks)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_rank_step, ws, steps, ms_max):
    """Whole-job throughput: every rank's flops over the slowest rank's time."""
    return flops_per_rank_step * ws * steps / (ms_max * 1e-3) / 1e12


# ------------------------------------------------------------------------------------------
# CPU oracle sample (the cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_sample(w, seconds: float):
    """Time the FP64 oracle's CLR product on whole block rows of C (all of K and all column
    clusters) until about ``seconds`` have elapsed.  Returns (flops, elapsed, rows_done)."""
    import numpy as np

    from oracle import clr_oracle as co
    rs = w.row_sizes
    off = np.concatenate([[0], np.cumsum(rs)])
    spec_b = [[(co.KIND_DENSE, w.b[off[k]:off[k + 1], off[j]:off[j + 1]])
               for j in range(len(rs))] for k in range(len(rs))]
    b = co.from_blocks(rs, rs, spec_b)
    flops, elapsed, rows = 0, 0.0, 0
    while elapsed < seconds and rows < len(rs):
        i = rows
        spec_a = [[(co.KIND_DENSE, w.a[off[i]:off[i + 1], off[k]:off[k + 1]])
                   for k in range(len(rs))]]
        a = co.from_blocks([rs[i]], rs, spec_a)
        t0 = time.perf_counter()
        co.multiply(a, b, 0.0)
        elapsed += time.perf_counter() - t0
        flops += 2 * rs[i] * w.n * w.n
        rows += 1
    return flops, elapsed, rows


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    # each step a bounded oracle sample: the whole run stays within about a minute or two
    per_step = getattr(args, "ref_seconds", None) or max(2.0, 60.0 / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(w, min(1.0, per_step))
    fl, el = 0, 0.0
    rows = 0
    for _ in range(args.steps):
        f, e, r = oracle_sample(w, per_step)
        fl += f
        el += e
        rows += r
    value = fl / el / 1e12
    cores = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(args),
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores,
                            "kind": "oracle",
                            "sample": "%d block rows of C (each: all 96 column clusters x all "
                                      "96 inner clusters) per %d steps" % (rows, args.steps)},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------

def sampled_accuracy(w, out_host_tiles, rng_seed=5, n_tiles=4):
    """Error of sampled C tiles against FP64 dot products of the inputs (numpy)."""
    import numpy as np
    off = np.concatenate([[0], np.cumsum(w.row_sizes)])
    rng = np.random.default_rng(rng_seed)
    num = den = ab = 0.0
    for _ in range(n_tiles):
        i, j = rng.integers(0, len(w.row_sizes), 2)
        r0, r1, c0, c1 = off[i], off[i + 1], off[j], off[j + 1]
        want = w.a[r0:r1] @ w.b[:, c0:c1]
        got = out_host_tiles(r0, r1, c0, c1)
        num += float(np.sum((got - want) ** 2))
        den += float(np.sum(want ** 2))
        ab += float(np.sum(np.linalg.norm(w.a[r0:r1], axis=1)[:, None] ** 2 *
                           np.linalg.norm(w.b[:, c0:c1], axis=0)[None, :] ** 2))
    return {"rel_frob_sampled": math.sqrt(num / den),
            "frob_over_normA_normB_sampled": math.sqrt(num / ab),
            "bound_10eps_eps1e-8": 1e-7, "tiles_sampled": n_tiles}


def dense_tiles_reader(gc, n):
    import torch
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    gc.to_dense(out)
    torch.cuda.synchronize()
    return lambda r0, r1, c0, c1: out[r0:r1, c0:c1].cpu().numpy()


def run_ours(args):
    import torch

    from paper_1509_00309_gb300 import build, clr
    rank, ws, local = dist_init()
    if ws == 1:
        torch.cuda.set_device(0)
    build.build()
    dev = torch.cuda.current_device()
    ctx = clr.Context(dev, precision=args.prec, eps_lr=1e-8)
    w = workload(args, rank)
    n = w.n
    stream = torch.cuda.current_stream()
    a_d = torch.from_numpy(w.a).cuda()
    b_d = torch.from_numpy(w.b).cuda()
    ga = ctx.from_dense(a_d, w.row_sizes)
    gb = ctx.from_dense(b_d, w.row_sizes)
    del a_d, b_d
    gc = ctx.zeros(w.row_sizes)
    stats = ctx.multiply_into(ga, gb, gc, stats=True)
    alg_flops = float(stats["flops"])
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] \
        if ws == 1 else str(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clk:
        for _ in range(args.warmup):
            ctx.multiply_into(ga, gb, gc)
        torch.cuda.synchronize()
        barrier(ws)
        clk.lines.clear()
        ctx.profile_enable(True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.multiply_into(ga, gb, gc)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    ctx.check()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms_total = max_over_ranks(e0.elapsed_time(e1), ws)
    ms_step = ms_total / args.steps
    value = job_tflops(alg_flops, ws, args.steps, ms_total)
    acc = sampled_accuracy(w, dense_tiles_reader(gc, n)) if rank == 0 else None

    # roofline of the dominant kernel (the split dense tile-product kernel)
    peaks, src = load_peaks()
    import hashlib
    with open(os.path.join(ROOT, "paper_1509_00309_gb300", "csrc", "k_split_gemm.cu"), "rb") as f:
        ksha = hashlib.sha256(f.read()).hexdigest()[:12]
    traffic = MEASURED_TRAFFIC.get("%s:%s:%d:%d" % (ksha, args.prec, args.n, args.clusters))
    # per launch of the dense kernel (one per product here)
    launches = max(1, prof["dense_launches"])
    per_product = launches / max(1, prof["products"])
    gemm_ms = prof["ms_dense"] / launches
    if args.prec in PAIRS:
        pairs = PAIRS[args.prec]
        achieved = alg_flops / per_product / (gemm_ms * 1e-3) / 1e12
        # the timed region is a burst of back-to-back products (well under a second): the
        # burst bf16 peak is the denominator; the sustained one is reported beside it
        peak = peaks["bf16_tflops"] / pairs
        peak_sus = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) / pairs
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "frac_sustained": achieved / peak_sus, "peak_sustained": peak_sus,
                # per launch: the bf16 term panels of A and of the launch's columns of B
                # read once, its FP64 columns of C written once
                "algorithmic_bytes": (2 if pairs == 3 else 3) * 2 * (n * n + n * n / per_product)
                + 8 * n * n / per_product,
                "launches_per_product": per_product,
                # the epilogue forms the dense tiles' norms when the clusters allow it
                "kernel": "split_gemm_kernel<%d, %d>" % (
                    2 if pairs == 3 else 3, 1 if min(w.row_sizes) >= 32 else 0),
                "kernel_ms": gemm_ms,
                "peak_basis": "%s burst bf16 %.1f TFLOP/s / %d term-pair products (sustained "
                              "%.1f / %d beside it)" % (
                                  src, peaks["bf16_tflops"], pairs,
                                  peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]),
                                  pairs),
                "tensor_tflops_issued": prof["dense_tensor_flops"] / (prof["ms_dense"] * 1e-3)
                / 1e12}
    else:
        roof = {"bound": "alu", "achieved": alg_flops / (gemm_ms * 1e-3) / 1e12,
                "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "kernel": "dd_fp64_kernel", "kernel_ms": gemm_ms}
    phases = {k: prof[k] / args.steps for k in ("ms_plan", "ms_stage", "ms_dense",
                                                "ms_lowrank", "ms_compress", "ms_finalize")}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        a_h = torch.from_numpy(w.a).pin_memory()
        b_h = torch.from_numpy(w.b).pin_memory()
        c_h = torch.empty((n, n), dtype=torch.float64).pin_memory()
        e2e_steps = max(3, min(args.steps, 10))
        ctx.multiply_host_stream(a_h, b_h, c_h, w.row_sizes, n_chunks=4)   # warm-up: buffers
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        marks = [t0]
        for _ in range(e2e_steps):
            # the streamed host product: A in 2 row chunks, B and C in 4 column chunks; the
            # copies overlap the 8 tile products (clr_multiply_host_stream, which returns
            # after synchronising)
            ctx.multiply_host_stream(a_h, b_h, c_h, w.row_sizes, n_chunks=4)
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, ws)
        each = [1e3 * (b - a) for a, b in zip(marks, marks[1:])]
        # the host side of the box is shared: the median step beside the mean shows whether
        # a few steps waited for the host link or host memory
        e2e = {"value": alg_flops * ws * e2e_steps / el / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8,
               "ms_per_step": 1e3 * el / e2e_steps, "steps": e2e_steps,
               "ms_each": [round(x, 2) for x in each],
               "ms_median": round(statistics.median(each), 2)}
        del a_h, b_h, c_h

    fp64_peak = clr.probe_fp64_rate(dev)

    # the plain form: the same product with FP64 tile products on the CUDA cores
    fp64 = ozaki = None
    if not args.no_fp64 and args.prec != "fp64":
        fp64 = fp64_product(ctx, ga, gb, gc, w, alg_flops, fp64_peak, value, acc, rank)
    if args.prec != "fp64":
        ozaki = ozaki_product(ctx, ga, gb, gc, w, alg_flops, fp64["tflops"] if fp64 else None,
                              rank)

    # the 1D-chain product (N = 2048, eps = 1e-8): FP64 against the split forms
    chain = None
    if not args.no_chain and rank == 0:
        chain = chain_product(clr, dev, fp64_peak)

    # Newton-Schulz S^-1/2 on the 1D-chain overlap matrix (N = 2048, 16 uneven clusters,
    # eps_lr = 1e-8): ms per iteration to ||X_n - I||_F/sqrt(N) <= 1e-6, and the residual
    # ||alpha Z S Z - I||_F / sqrt(N) of the result against the same tolerance
    ns = None
    if not args.no_ns:
        from paper_1509_00309_gb300 import workloads as wl
        wn = wl.chain_overlap()
        nctx = clr.Context(dev, precision=args.ns_prec,
                           eps_lr=wn.eps_lr, ns_tol=1e-6, ns_max_iter=60,
                           ns_fp64_tail=int(args.ns_prec != "fp64"), ns_ladder_switch=1e-3)
        sm = nctx.from_dense(torch.from_numpy(wn.a).cuda(), wn.row_sizes, eps_lr=wn.eps_lr,
                             drop_norm=wn.drop_norm)
        nctx.sqrt_inv(sm, allow_noconv=True)   # warm-up
        torch.cuda.synchronize()
        z, nst, _ = nctx.sqrt_inv(sm, allow_noconv=True)
        it = max(1, nst["iters"])
        ns = {"workload": "1D-chain overlap N=2048, 16 uneven clusters, eps_lr=1e-8",
              "ms_per_iteration": nst["ms_total"] / it, "iterations": nst["iters"],
              "residual_ZSZ_minus_I_rms": nst["residual"], "tol": 1e-6,
              "residual_met": nst["residual_met"], "proxy_final": nst["proxy"][-1],
              "ms_residual": nst["ms_residual"],
              "precision": args.ns_prec if args.ns_prec == "fp64" else
                           "%s, fp64 below proxy 1e-3" % args.ns_prec,
              "z_blocks_zero_dense_lr": z.info()["n_blocks"]}

    # Newton-Schulz on the 3D lattice matrices (16 points per jittered lattice site, clusters
    # of 64..256 points, built at eps_lr = 1e-6, drop 1e-10, eps_sp = 1e-13; iterates truncated
    # at EPS_NS_LATTICE), FP64 products, dense-accumulated tiles re-tested for low rank; with
    # the block-rank distribution of the 5th-iteration intermediates X, T, Y, Z (Section 5).
    # The same run with split products (bf16x6, FP64 from ||X - I|| <= 1e-3) shows the split
    # floor.  The overlap-like S has block sparsity; the Coulomb-like V (erf(r)/r) has only
    # block-rank sparsity (Section 4.2).
    ns_lat = ns_lat_split = ns_lat_ozaki = ns_coul = None
    if not args.no_ns and args.ns_lattice != "none":
        from paper_1509_00309_gb300 import workloads as wl
        shape = tuple(int(v) for v in args.ns_lattice.split("x"))
        wlat = wl.lattice_overlap(shape=shape)
        ns_lat = lattice_ns(clr, wlat, args.ns_lattice, "overlap", fp64_peak, "fp64")
        ns_lat_split = lattice_ns(clr, wlat, args.ns_lattice, "overlap", fp64_peak, "bf16x6",
                                  snapshot=False)
        ns_lat_ozaki = lattice_ns(clr, wlat, args.ns_lattice, "overlap", fp64_peak, "ozaki",
                                  snapshot=False)
        ns_coul = lattice_ns(clr, wl.lattice_coulomb(shape=shape), args.ns_lattice,
                             "Coulomb-like erf(r)/r", fp64_peak, "fp64", snapshot=False)
    ns_large = None
    if not args.no_ns and args.ns_lattice_large != "none":
        from paper_1509_00309_gb300 import workloads as wl
        shape = tuple(int(v) for v in args.ns_lattice_large.split("x"))
        wlarge = wl.lattice_overlap(shape=shape)
        ns_large = {p: lattice_ns_timed(clr, wlarge, args.ns_lattice_large, p)
                    for p in ("ozaki", "fp64")}

    # 64 independent 1D-chain products of uneven size in one CUDA graph (the batched
    # configuration), autotuned and FP64-only, each measured in a child process with its own
    # context and memory
    batch = None
    if rank == 0 and ws == 1 and not args.no_batch:
        batch = {"autotuned": batch_measure(64, "auto"), "fp64": batch_measure(64, "fp64")}
        for r in batch.values():
            if "error" not in r:
                r["roofline"] = batch_roofline(r, fp64_peak)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        fl, el, rows = oracle_sample(w, 15.0)
        cpu = {"value": fl / el / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "%d block rows of C (all 96 column clusters x all 96 inner clusters, "
                         "%.1f GFLOP) of the same workload" % (rows, fl / 1e9)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.prec, "data": "synthetic", "config": config(args),
                "accuracy": acc, "phases_ms_per_step": phases,
                "algorithmic_flops_per_step": alg_flops,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_dense": fp64,
                "fp64_accurate_tensor": ozaki,
                "chain_product": chain, "ns": ns, "ns_lattice": ns_lat,
                "ns_lattice_split": ns_lat_split, "ns_lattice_ozaki": ns_lat_ozaki,
                "ns_coulomb": ns_coul,
                "ns_lattice_large": ns_large, "batch": batch,
                "gpu_launches": int(prof["launches"]), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ozaki_product(ctx, ga, gb, gc, w, alg_flops, fp64_value, rank, warmup=2, steps=5):
    """The same workload with FP64-accurate dense products on the tensor cores (exact slices,
    precision "ozaki"): TFLOP/s over `steps` products after `warmup`, the exact-slice kernel's
    time, and the accuracy beside the FP64 form's."""
    import torch
    prev = ctx.get_opts().precision
    ctx.set_opts(precision="ozaki")
    for _ in range(warmup):
        ctx.multiply_into(ga, gb, gc)
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(steps):
        ctx.multiply_into(ga, gb, gc)
    e[1].record()
    torch.cuda.synchronize()
    ctx.check()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.set_opts(precision=prev)
    ms = e[0].elapsed_time(e[1]) / steps
    tf = alg_flops / (ms * 1e-3) / 1e12
    kern_ms = prof["ms_dense"] / steps
    acc = sampled_accuracy(w, dense_tiles_reader(gc, w.n)) if rank == 0 else None
    return {"ms_per_product": ms, "tflops": tf, "kernel": "ozaki_gemm_kernel",
            "kernel_ms": kern_ms, "kernel_tflops": alg_flops / (kern_ms * 1e-3) / 1e12,
            "staging_ms": prof["ms_stage"] / steps,
            "tensor_products_per_flop": 36,
            "accuracy": acc, "over_fp64_speedup": tf / fp64_value if fp64_value else None,
            "steps": steps, "warmup": warmup}


def fp64_product(ctx, ga, gb, gc, w, alg_flops, fp64_peak, split_value, split_acc, rank):
    """One product of the same workload with FP64 tile products (dd_fp64_kernel on the CUDA
    cores; ~7 s at N = 16384), after the split run sized every workspace: TFLOP/s, the
    fraction of the measured FP64 FMA rate, and its accuracy beside the split form's."""
    import torch
    prev = ctx.get_opts().precision
    ctx.set_opts(precision="fp64")
    ctx.profile_enable(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    ctx.multiply_into(ga, gb, gc)
    e[1].record()
    torch.cuda.synchronize()
    ctx.check()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.set_opts(precision=prev)
    ms = e[0].elapsed_time(e[1])
    tf = alg_flops / (ms * 1e-3) / 1e12
    kern = alg_flops / (prof["ms_dense"] * 1e-3) / 1e12
    acc = sampled_accuracy(w, dense_tiles_reader(gc, w.n)) if rank == 0 else None
    return {"ms_per_product": ms, "tflops": tf, "kernel": "dd_fp64_kernel",
            "kernel_ms": prof["ms_dense"], "kernel_tflops": kern,
            "peak_fp64_measured": fp64_peak, "frac": kern / fp64_peak, "bound": "alu",
            "peak_basis": "measured FP64 FMA rate of this GPU (clr_probe_fp64_rate)",
            "accuracy": acc, "split_over_fp64_speedup": split_value / tf,
            "split_accuracy_within_bound": bool(split_acc and
                                                split_acc["frob_over_normA_normB_sampled"] <=
                                                split_acc["bound_10eps_eps1e-8"]),
            "steps": 1}


def chain_product(clr, dev, fp64_peak, warmup=3, steps=15):
    """The 1D-chain CLR product S S (N = 2048, 16 uneven clusters, built and recompressed at
    eps = 1e-8; Section 4.1) in FP64 and in the split forms: microseconds per product (median
    of `steps` after `warmup`), algorithmic TFLOP/s, and ||C - A A||_F against the FP64 dense
    product of the reconstructed operand with the bound 10 eps ||A||_F^2."""
    import numpy as np
    import torch
    from paper_1509_00309_gb300 import workloads as wl
    wn = wl.chain_overlap()
    out = {"workload": "1D-chain overlap product S S, N=2048, 16 uneven clusters, eps=1e-8"}
    ctx = clr.Context(dev, precision="fp64", eps_lr=wn.eps_lr)
    sm = ctx.from_dense(torch.from_numpy(wn.a).cuda(), wn.row_sizes, eps_lr=wn.eps_lr,
                        drop_norm=wn.drop_norm)
    a = sm.to_dense()
    want = a @ a
    bound = 10.0 * wn.eps_lr * float(np.linalg.norm(a)) ** 2
    for prec in ("fp64", "bf16x6", "bf16x3"):
        ctx.set_opts(precision=prec)
        gc = ctx.zeros(wn.row_sizes)
        st = ctx.multiply_into(sm, sm, gc, stats=True)
        for _ in range(warmup):
            ctx.multiply_into(sm, sm, gc)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record()
        for i in range(steps):
            ctx.multiply_into(sm, sm, gc)
            ev[i + 1].record()
        torch.cuda.synchronize()
        ctx.check()
        ms = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
        med = ms[steps // 2]
        err = float(np.linalg.norm(gc.to_dense() - want))
        out[prec] = {"us_per_product": 1e3 * med, "tflops": st["flops"] / (med * 1e-3) / 1e12,
                     "err_frob": err, "bound_10eps_normA2": bound,
                     "within_bound": err <= bound, "triples": st["n_triples"],
                     "tiles_dense_lr": st["n_tiles"][1:]}
        gc.close()
    fast = [p for p in ("bf16x3", "bf16x6") if out[p]["within_bound"]]
    if fast:
        best = min(fast, key=lambda p: out[p]["us_per_product"])
        out["fastest_split_within_bound"] = best
        out["split_over_fp64_speedup"] = out["fp64"]["us_per_product"] / out[best]["us_per_product"]
    return out


FP32_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def batch_measure(n: int, precision: str, timeout: int = 420):
    """products/s and algorithmic TFLOP/s of n batched chain products replayed as one CUDA graph
    (`python -m paper_1509_00309_gb300.diagnostics --batch n --batch-precision P`), or
    {"error": ...}."""
    cmd = [sys.executable, "-m", "paper_1509_00309_gb300.diagnostics", "--batch", str(n),
           "--batch-precision", precision]
    try:
        r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": "did not finish within %d s" % timeout}
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        tail = (r.stderr or "").strip().splitlines()[-1:] or [""]
        return {"error": "exit %d: %s" % (r.returncode, tail[0][:200])}
    try:
        return json.loads(lines[-1])
    except ValueError:
        return {"error": "unreadable output"}


def lattice_ns(clr, w, shape_txt, what, fp64_peak, precision, snapshot=True):
    """NS on one lattice matrix through the C ABI: the iterates truncated at EPS_NS_LATTICE,
    stopped at ||X - I||_F/sqrt(N) <= 1e-6 and judged by the residual ||alpha Z S Z - I||_F /
    sqrt(N) <= 1e-6 (the stated error).  One profiled run (the iteration's two products one
    after the other, so that the phase intervals time their own kernels) gives the phase split,
    the SVD counters, the recompression kernels' ALU rooflines and the rank distribution; a
    second, unprofiled run (the two products on two streams, as in production) gives the time
    per iteration."""
    import torch
    from paper_1509_00309_gb300 import diagnostics
    split = precision in ("bf16x3", "bf16x6")
    ctx = clr.Context(torch.cuda.current_device(), precision=precision, eps_lr=EPS_NS_LATTICE,
                      eps_sp=w.eps_sp, ns_tol=1e-6, ns_max_iter=40, recompress_dense=1,
                      ns_fp64_tail=int(split), ns_ladder_switch=1e-3)
    sm = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                        drop_norm=w.drop_norm)
    ctx.set_opts(ns_max_iter=1, ns_tol=0.0)
    ctx.sqrt_inv(sm, allow_noconv=True)   # warm-up: workspaces
    ctx.set_opts(ns_max_iter=40, ns_tol=1e-6)
    torch.cuda.synchronize()
    d = diagnostics.ns_rank_distribution(ctx, sm, 5 if snapshot else 0)
    torch.cuda.synchronize()
    _, st, _ = ctx.sqrt_inv(sm, allow_noconv=True)
    prof = d["profile"]
    out = {"workload": "3D lattice %s matrix, %s sites x 16 points, N=%d, %d clusters of "
                       "64..256, built at eps_lr=%g, iterates truncated at %g" % (
                           what, shape_txt, w.n, len(w.row_sizes), w.eps_lr, EPS_NS_LATTICE),
           "ms_per_iteration": st["ms_total"] / max(1, st["iters"]),
           "iterations": st["iters"], "ms_residual": st["ms_residual"],
           "proxy_final": st["proxy"][-1],
           "residual_ZSZ_minus_I_rms": st["residual"], "tol": 1e-6,
           "residual_met": st["residual_met"], "proxy_met": st["proxy_met"],
           "precision": precision if precision in ("fp64", "ozaki") else
                        "%s, fp64 below proxy 1e-3" % precision,
           "recompress_dense": True,
           "profiled_run": {
               "ms_per_iteration_serial": d["ns"]["ms_per_iter"],
               "phases_ms_total": {k: prof[k] for k in
                                   ("ms_dense", "ms_lowrank", "ms_compress_qr",
                                    "ms_compress_dense")},
               "svd": {k: prof[k] for k in ("svd_blocks", "svd_sweeps_fp32",
                                            "svd_sweeps_fp64", "svd_early_dense",
                                            "svd_prereduced")},
               "compress_dense_paths": {
                   name: {"blocks": prof["svd_path_blocks"][i],
                          "mcycles_per_block": prof["svd_path_cycles"][i] / 1e6 /
                          max(1, prof["svd_path_blocks"][i])}
                   for i, name in enumerate(("pivoted_qr_svd_of_r_low_rank",
                                             "certified_dense_without_svd", "full_svd",
                                             "pivoted_qr_svd_of_r_dense"))},
               "full_svd_stages_mcycles": dict(
                   zip(("pivoted_qr_attempt", "fp32_sweeps_on_a", "fp64_orthonormalise_project",
                        "fp32_sweeps_on_g", "fp64_orthonormalise_multiply", "fp64_sweeps",
                        "truncate_store"),
                       (round(c / 1e6, 1) for c in prof["svd_full_cycles"])),
                   blocks_all_stages=prof["svd_full_blocks"],
                   blocks_stored_dense=prof["svd_full_dense"]),
               "pre_reduced_stages_mcycles": dict(
                   zip(("pivoted_qr", "fp32_sweeps_on_rt", "fp64_orthonormalise_project",
                        "fp32_sweeps_on_g", "fp64_orthonormalise_multiply", "fp64_sweeps",
                        "truncate_recover_store"),
                       (round(c / 1e6, 1) for c in prof["svd_pre_cycles"])),
                   blocks=prof["svd_pre_blocks"]),
               "roofline_recompress": recompress_roofline(prof, fp64_peak)}}
    if snapshot:
        out["rank_distribution_iter5"] = {
            k: {f: d[k][f] for f in ("zero", "dense", "low_rank", "lr_rank_mean", "lr_rank_max")}
            for k in ("S", "X_5", "T_5", "Y_5", "Z_5", "Z_final") if d.get(k)}
    return out


def lattice_ns_timed(clr, w, shape_txt, precision="fp64"):
    """NS on a larger lattice overlap matrix at the stated error: one unprofiled run (after a
    one-iteration warm-up that sizes the workspaces), FP64 products, iterates truncated at
    EPS_NS_LATTICE, dense-accumulated tiles re-tested."""
    import torch
    ctx = clr.Context(torch.cuda.current_device(), precision=precision,
                      eps_lr=EPS_NS_LATTICE, eps_sp=w.eps_sp, ns_tol=1e-6, ns_max_iter=40,
                      recompress_dense=1)
    sm = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                        drop_norm=w.drop_norm)
    ctx.set_opts(ns_max_iter=1, ns_tol=0.0)
    ctx.sqrt_inv(sm, allow_noconv=True)
    ctx.set_opts(ns_max_iter=40, ns_tol=1e-6)
    torch.cuda.synchronize()
    z, st, _ = ctx.sqrt_inv(sm, allow_noconv=True)
    info = z.info()
    return {"workload": "3D lattice overlap matrix, %s sites x 16 points, N=%d, %d clusters of "
                        "64..256, built at eps_lr=%g, iterates truncated at %g" % (
                            shape_txt, w.n, len(w.row_sizes), w.eps_lr, EPS_NS_LATTICE),
            "ms_per_iteration": st["ms_total"] / max(1, st["iters"]),
            "iterations": st["iters"], "ms_residual": st["ms_residual"],
            "proxy_final": st["proxy"][-1], "residual_ZSZ_minus_I_rms": st["residual"],
            "tol": 1e-6, "residual_met": st["residual_met"], "proxy_met": st["proxy_met"],
            "precision": precision, "recompress_dense": True,
            "z_blocks_zero_dense_lr": info["n_blocks"]}


def _alu_roofline(f64, f32, ms, fp64_peak):
    t = ms * 1e-3
    if not t > 0:
        return None
    a64, a32 = f64 / t / 1e12, f32 / t / 1e12
    # time the two pipes would need at their peaks, as a fraction of the measured time
    return {"bound": "alu", "achieved_fp64": a64, "peak_fp64": fp64_peak,
            "achieved_fp32": a32, "peak_fp32": FP32_TFLOPS_NOMINAL, "unit": "TFLOP/s",
            "frac": a64 / fp64_peak + a32 / FP32_TFLOPS_NOMINAL, "kernel_ms": ms,
            "traffic": None}


def recompress_roofline(prof, fp64_peak):
    """ALU rooflines of the two recompression kernels from the library's algorithmic flop
    counters and their device times: FP64 flops against the measured FMA rate, FP32 flops
    against the nominal rate."""
    qr = _alu_roofline(prof["svd_flops_fp64_qr"], prof["svd_flops_fp32_qr"],
                       prof["ms_compress_qr"], fp64_peak)
    dn = _alu_roofline(prof["svd_flops_fp64"] - prof["svd_flops_fp64_qr"],
                       prof["svd_flops_fp32"] - prof["svd_flops_fp32_qr"],
                       prof["ms_compress_dense"], fp64_peak)
    return {"compress_qr_kernel": qr, "compress_dense_kernel": dn,
            "peak_basis": "FP64: measured FMA rate (clr_probe_fp64_rate); FP32: 152 SMs x 128 "
                          "lanes x 2 x 2.07 GHz (nominal)"}


def batch_roofline(r, fp64_peak):
    """ALU rooflines of a batch run's dominant kernels, from its uncaptured pass: the two
    recompression kernels, and for FP64 products the dense x dense kernel (its flops counted
    from the operands' block kinds) against the measured FP64 FMA rate.  {"error": ...} when
    an input is missing."""
    try:
        p = r["roofline_inputs"]
        out = {"recompression": recompress_roofline(p, fp64_peak)}
        if r.get("precision_mode") == "fp64" and p.get("dense_dd_flops"):
            dense = _alu_roofline(p["dense_dd_flops"], 0.0, p["ms_dense"], fp64_peak)
            if dense is not None:
                dense["kernel"] = "dd_fp64_kernel"
            out["dense_fp64"] = dense
        return out
    except (KeyError, TypeError, ZeroDivisionError) as e:
        return {"error": "roofline inputs incomplete: %r" % (e,)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
