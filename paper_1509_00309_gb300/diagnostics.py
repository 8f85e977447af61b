"""Block-rank diagnostics of the Newton–Schulz iterates (Section 5, the distribution of block
ranks of the 5th-iteration intermediates X, Y, Z, T and of the input S).

    python -m paper_1509_00309_gb300.diagnostics --shape 8x8x4 --iter 5 [--matrix coulomb]
    python -m paper_1509_00309_gb300.diagnostics --adjoint --shape 8x8x8 --max-iter 20
    python -m paper_1509_00309_gb300.diagnostics --batch 64

builds the 3D lattice overlap matrix (16 points per site, clusters of 64..256 points, eps_lr
1e-6, drop 1e-10, eps_sp 1e-13), or the Coulomb-like erf(r)/r matrix on the same lattice, on
the GPU, runs clr_sqrt_inv with the snapshot option and
prints one JSON object: per matrix its block counts by kind and the rank histogram (entry 0:
zero blocks, entry r: low-rank blocks of rank r, last entry: dense blocks), plus the NS timing
and the SVD counters of the library's profile.  Everything runs through the C ABI."""
import argparse
import json
import time
from typing import Dict

import numpy as np

from . import clr
from . import workloads as wl


def histogram_summary(m: "clr.Matrix") -> Dict:
    info = m.info()
    h = np.asarray(info["rank_hist"], dtype=np.int64)
    lr_ranks = np.repeat(np.arange(len(h) - 2) + 1, h[1:-1])
    return {"zero": int(h[0]), "dense": int(h[-1]), "low_rank": int(h[1:-1].sum()),
            "lr_rank_mean": float(lr_ranks.mean()) if lr_ranks.size else 0.0,
            "lr_rank_max": int(lr_ranks.max()) if lr_ranks.size else 0,
            "hist": {int(r): int(c) for r, c in enumerate(h) if c}}


def ns_rank_distribution(ctx: "clr.Context", s: "clr.Matrix", k: int = 5) -> Dict:
    """Run NS on s with the k-th iteration snapshot on; histograms of S and of X, T, Y, Z."""
    ctx.set_opts(ns_snapshot_iter=k)
    ctx.profile_enable(True)
    t0 = time.time()
    z, st, _ = ctx.sqrt_inv(s, allow_noconv=True)
    wall = time.time() - t0
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    out = {"S": histogram_summary(s)}
    for name in "XTYZ":
        try:
            out[name + "_%d" % k] = histogram_summary(ctx.ns_snapshot(name, s))
        except clr.ClrError:   # the iteration was not reached
            out[name + "_%d" % k] = None
    out["Z_final"] = histogram_summary(z)
    out["ns"] = {"iters": st["iters"], "residual": st["residual"], "wall_s": wall,
                 "ms_per_iter": st["ms_total"] / max(1, st["iters"]),
                 "proxy": st["proxy"], "status": st["status"]}
    out["profile"] = {key: prof[key] for key in ("products", "ms_dense", "ms_lowrank",
                                                  "ms_compress", "svd_blocks", "svd_sweeps_fp32",
                                                  "svd_sweeps_fp64", "svd_early_dense",
                                                  "svd_flops_fp64", "svd_flops_fp32")}
    ctx.set_opts(ns_snapshot_iter=0)
    return out


def adjoint_run(shape, precision: str = "fp64", iters: int = 20, eps: float = 1e-8) -> Dict:
    """The differentiation configuration: loss = trace(W S^-1/2) on the 3D lattice overlap
    matrix (eps_lr = 1e-8, 20 checkpointed NS iterations), gradient dL/dS by the hand-written
    adjoint (clr_sqrt_inv_backward); device times of the forward and backward sweeps."""
    import torch
    w = wl.adjoint_lattice(n_sites_shape=shape)
    ctx = clr.Context(0, precision=precision, eps_lr=eps, ns_tol=0.0, ns_max_iter=iters)
    s = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=eps)
    zb = ctx.from_dense(torch.from_numpy(np.ascontiguousarray(w.extra["w"].T)).cuda(),
                        w.row_sizes, eps_lr=0.0)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    z, st, tape = ctx.sqrt_inv(s, keep_tape=True)
    ev[1].record()
    g = ctx.sqrt_inv_backward(tape, zb)
    ev[2].record()
    torch.cuda.synchronize()
    gi = g.info()
    return {"workload": w.name, "n": w.n, "clusters": len(w.row_sizes), "eps_lr": eps,
            "iterations": st["iters"], "residual": st["residual"],
            "ms_forward": ev[0].elapsed_time(ev[1]), "ms_backward": ev[1].elapsed_time(ev[2]),
            "grad_frob": gi["frob_norm"], "grad_blocks": gi["n_blocks"]}


def batch_run(n_instances: int = 64, steps: int = 10, warmup: int = 3) -> Dict:
    """The batched configuration: n_instances independent 1D-chain products S S of uneven size
    (N ~ U[1024, 8192], clusters U[48, 256], eps from {1e-6, 1e-8}) captured into one CUDA graph
    with the autotuner's per-shape choice (clr_batch_*); products/s and algorithmic TFLOP/s of
    graph replays timed with CUDA events."""
    import torch
    ws = wl.batched_chains(n_instances=n_instances)
    ctx = clr.Context(0, precision="auto", eps_lr=1e-8)
    mats = [ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                           drop_norm=w.drop_norm) for w in ws]
    torch.cuda.synchronize()
    # algorithmic flops of every product (the library's triple statistics), untimed
    flops = 0.0
    for m, w in zip(mats, ws):
        ctx.set_opts(eps_lr=w.eps_lr)
        out = ctx.zeros(w.row_sizes)
        flops += float(ctx.multiply_into(m, m, out, stats=True)["flops"])
        out.close()
    ctx.set_opts(eps_lr=1e-8)
    batch = ctx.batch(mats, mats, eps=[w.eps_lr for w in ws], tune=True)
    for _ in range(warmup):
        batch.run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(steps):
        batch.run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    prec = {}
    for i in range(batch.n):
        t = batch.tuning(i)["precision"]
        prec[t] = prec.get(t, 0) + 1
    batch.close()
    return {"workload": "%d batched 1D-chain products S S, N ~ U[1024,8192], clusters U[48,256], "
                        "eps in {1e-6, 1e-8}, one CUDA graph" % n_instances,
            "instances": n_instances, "sum_n": int(sum(w.n for w in ws)),
            "ms_per_batch": ms, "products_per_s": n_instances / (ms * 1e-3),
            "tflops": flops / (ms * 1e-3) / 1e12, "algorithmic_flops_per_batch": flops,
            "precisions": prec, "steps": steps, "warmup": warmup}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="8x8x4", help="lattice sites, e.g. 16x16x8 (N = 16 x sites)")
    ap.add_argument("--iter", type=int, default=5)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--max-iter", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-recompress-dense", action="store_true")
    ap.add_argument("--matrix", default="overlap", choices=["overlap", "coulomb"])
    ap.add_argument("--adjoint", action="store_true",
                    help="time forward + adjoint of trace(W S^-1/2) instead (eps_lr 1e-8, "
                         "--max-iter iterations)")
    ap.add_argument("--batch", type=int, default=0, metavar="N",
                    help="time N batched 1D-chain products in one CUDA graph instead")
    args = ap.parse_args()
    import torch
    shape = tuple(int(v) for v in args.shape.split("x"))
    if args.batch:
        print(json.dumps(batch_run(args.batch)))
        return
    if args.adjoint:
        print(json.dumps(adjoint_run(shape, args.precision, min(args.max_iter, 40))))
        return
    w = wl.lattice_overlap(shape=shape) if args.matrix == "overlap" else \
        wl.lattice_coulomb(shape=shape)
    ctx = clr.Context(0, precision=args.precision, eps_lr=w.eps_lr, eps_sp=w.eps_sp,
                      ns_tol=args.tol, ns_max_iter=args.max_iter,
                      recompress_dense=0 if args.no_recompress_dense else 1)
    s = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                       drop_norm=w.drop_norm)
    out = {"workload": w.name, "n": w.n, "clusters": len(w.row_sizes),
           "precision": args.precision, "recompress_dense": not args.no_recompress_dense}
    out.update(ns_rank_distribution(ctx, s, args.iter))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
