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
                 "ms_residual": st["ms_residual"], "proxy": st["proxy"],
                 "proxy_met": st["proxy_met"], "residual_met": st["residual_met"],
                 "converged": st["converged"], "status": st["status"]}
    out["profile"] = {key: prof[key] for key in ("products", "ms_dense", "ms_lowrank",
                                                  "ms_compress", "ms_compress_qr",
                                                  "ms_compress_dense", "svd_blocks",
                                                  "svd_sweeps_fp32", "svd_sweeps_fp64",
                                                  "svd_early_dense", "svd_prereduced",
                                                  "svd_flops_fp64", "svd_flops_fp32",
                                                  "svd_flops_fp64_qr", "svd_flops_fp32_qr",
                                                  "svd_path_cycles", "svd_path_blocks",
                                                  "svd_full_cycles", "svd_full_blocks",
                                                  "svd_full_dense", "svd_pre_cycles",
                                                  "svd_pre_blocks")}
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


def batch_run(n_instances: int = 64, steps: int = 10, warmup: int = 3,
              precision: str = "auto", n_check: int = 8) -> Dict:
    """The batched configuration: n_instances independent 1D-chain products S S of uneven size
    (N ~ U[1024, 8192], clusters U[48, 256], eps from {1e-6, 1e-8}) captured into one CUDA graph
    (clr_batch_*), with the autotuner's per-shape choice of precision and CTAs per SM
    (precision "auto") or FP64 products throughout (precision "fp64", tuned CTAs per SM only);
    products/s and algorithmic TFLOP/s of graph replays timed with CUDA events.  Also: the
    device-time split of one uncaptured pass over all products (the dominant kernel and its
    share), and for n_check instances spread over the batch the error of the replayed output
    against the FP64 dense product of the reconstructed operand (10 eps ||A||_F^2 bound)."""
    import torch
    ws = wl.batched_chains(n_instances=n_instances)
    ctx = clr.Context(0, precision=precision, eps_lr=1e-8)
    mats = [ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                           drop_norm=w.drop_norm) for w in ws]
    torch.cuda.synchronize()
    try:
        dd_flops = sum(dense_product_flops(m.get_blocks(pool=False)[0], w.row_sizes)
                       for m, w in zip(mats, ws))
    except Exception:   # noqa: BLE001 -- the count only feeds a roofline figure
        dd_flops = None
    batch = ctx.batch(mats, mats, eps=[w.eps_lr for w in ws], tune=True)
    tuned = [batch.tuning(i) for i in range(batch.n)]
    # algorithmic flops of every product (the library's triple statistics) and the device-time
    # split of one uncaptured pass with the tuned precisions, untimed
    flops = 0.0
    outs = []
    ctx.profile_enable(True)
    for m, w, t in zip(mats, ws, tuned):
        ctx.set_opts(eps_lr=w.eps_lr, precision=t["precision"])
        out = ctx.zeros(w.row_sizes)
        flops += float(ctx.multiply_into(m, m, out, stats=True)["flops"])
        outs.append(out)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    for o in outs:
        o.close()
    ctx.set_opts(eps_lr=1e-8, precision=precision)
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
    for t in tuned:
        prec[t["precision"]] = prec.get(t["precision"], 0) + 1
    # per-instance error of the replayed outputs
    errs = []
    for i in np.linspace(0, n_instances - 1, min(n_check, n_instances)).astype(int):
        a = mats[i].to_dense()
        c = batch.output(int(i)).to_dense()
        nrm = float(np.linalg.norm(a))
        err = float(np.linalg.norm(c - a @ a))
        errs.append({"instance": int(i), "n": ws[i].n, "eps": ws[i].eps_lr,
                     "precision": tuned[i]["precision"], "err_frob": err,
                     "bound_10eps_normA2": 10.0 * ws[i].eps_lr * nrm * nrm,
                     "within_bound": err <= 10.0 * ws[i].eps_lr * nrm * nrm})
    batch.close()
    phases = {k: prof[k] for k in ("ms_plan", "ms_stage", "ms_dense", "ms_lowrank",
                                   "ms_compress", "ms_finalize")}
    tot = sum(phases.values())
    top = max(phases, key=phases.get)
    names = {"ms_plan": "plan kernels", "ms_stage": "split_stage kernels",
             "ms_dense": "dense tile products (split_gemm_kernel / dd_fp64_kernel)",
             "ms_lowrank": "lr_products_kernel",
             "ms_compress": "compress_qr_kernel + compress_dense_kernel",
             "ms_finalize": "norms / scaling"}
    return {"workload": "%d batched 1D-chain products S S, N ~ U[1024,8192], clusters U[48,256], "
                        "eps in {1e-6, 1e-8}, one CUDA graph" % n_instances,
            "precision_mode": precision,
            "instances": n_instances, "sum_n": int(sum(w.n for w in ws)),
            "ms_per_batch": ms, "products_per_s": n_instances / (ms * 1e-3),
            "tflops": flops / (ms * 1e-3) / 1e12, "algorithmic_flops_per_batch": flops,
            "precisions": prec, "steps": steps, "warmup": warmup,
            "uncaptured_pass_ms": phases, "dominant": {"phase": names[top],
                                                       "share": phases[top] / tot if tot else None},
            "svd": {k: prof[k] for k in ("svd_blocks", "svd_sweeps_fp32", "svd_sweeps_fp64",
                                         "svd_flops_fp64", "svd_flops_fp32")},
            # the uncaptured pass's kernel times and algorithmic flops, for the rooflines
            "roofline_inputs": dict({k: prof[k] for k in (
                "ms_dense", "ms_compress_qr", "ms_compress_dense", "svd_flops_fp64",
                "svd_flops_fp32", "svd_flops_fp64_qr", "svd_flops_fp32_qr")},
                dense_dd_flops=dd_flops),
            "errors": errs, "all_within_bound": all(e["within_bound"] for e in errs)}


def dense_product_flops(kinds, sizes) -> float:
    """Flops of the dense x dense tile products of M M for a square CLR matrix M with block
    kinds `kinds` and cluster sizes `sizes`: 2 m_I m_K m_J for every (I, K, J) whose blocks
    M_IK and M_KJ are both dense, i.e. 2 s^T (D diag(s) D) s with D the dense indicator."""
    d = (np.asarray(kinds) == clr.KIND_DENSE).astype(np.float64)
    sz = np.asarray(sizes, dtype=np.float64)
    return 2.0 * float(sz @ ((d * sz[None, :]) @ d) @ sz)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="8x8x4", help="lattice sites, e.g. 16x16x8 (N = 16 x sites)")
    ap.add_argument("--iter", type=int, default=5)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--max-iter", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--eps-ns", type=float, default=0.0,
                    help="truncation of the NS iterates (default: the matrix's build eps_lr, "
                         "1e-6)")
    ap.add_argument("--no-recompress-dense", action="store_true")
    ap.add_argument("--matrix", default="overlap", choices=["overlap", "coulomb"])
    ap.add_argument("--adjoint", action="store_true",
                    help="time forward + adjoint of trace(W S^-1/2) instead (eps_lr 1e-8, "
                         "--max-iter iterations)")
    ap.add_argument("--batch", type=int, default=0, metavar="N",
                    help="time N batched 1D-chain products in one CUDA graph instead")
    ap.add_argument("--batch-precision", default="auto", choices=["auto", "fp64"])
    args = ap.parse_args()
    import torch
    shape = tuple(int(v) for v in args.shape.split("x"))
    if args.batch:
        print(json.dumps(batch_run(args.batch, precision=args.batch_precision)))
        return
    if args.adjoint:
        print(json.dumps(adjoint_run(shape, args.precision, min(args.max_iter, 40))))
        return
    w = wl.lattice_overlap(shape=shape) if args.matrix == "overlap" else \
        wl.lattice_coulomb(shape=shape)
    eps_ns = args.eps_ns if args.eps_ns > 0 else w.eps_lr
    ctx = clr.Context(0, precision=args.precision, eps_lr=eps_ns, eps_sp=w.eps_sp,
                      ns_tol=args.tol, ns_max_iter=args.max_iter,
                      recompress_dense=0 if args.no_recompress_dense else 1,
                      ns_fp64_tail=int(args.precision in ("bf16x3", "bf16x6")),
                      ns_ladder_switch=1e-3)
    s = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                       drop_norm=w.drop_norm)
    out = {"workload": w.name, "n": w.n, "clusters": len(w.row_sizes),
           "precision": args.precision, "eps_build": w.eps_lr, "eps_ns": eps_ns,
           "recompress_dense": not args.no_recompress_dense}
    out.update(ns_rank_distribution(ctx, s, args.iter))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
