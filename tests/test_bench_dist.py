"""The multi-rank path of bench.py (independent replicas, one process per GPU) on CPU with
the gloo backend, world size 2: the rendezvous, the max-over-ranks timing, the whole-job
throughput, and the reference arm running on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, root, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, root)
    import bench
    import torch.distributed as dist
    r, ws, local = bench.dist_init("gloo")
    assert (r, ws, local) == (rank, world, rank)
    bench.barrier(ws)
    slowest = bench.max_over_ranks(100.0 + 10.0 * rank, ws, device="cpu")
    value = bench.job_tflops(1e12, ws, 5, slowest)
    out.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo(repo_root):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, repo_root, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 110.0                      # max over ranks
        assert abs(value - 1e12 * 2 * 5 / 0.110 / 1e12) < 1e-9
    

def test_reference_arm_other_ranks_do_no_work(repo_root, monkeypatch):
    sys.path.insert(0, repo_root)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "n": 256, "clusters": 2, "gpus": 2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_reference_arm_rank0_prints_one_line(repo_root, monkeypatch):
    import json
    sys.path.insert(0, repo_root)
    import bench
    monkeypatch.setenv("RANK", "0")
    args = type("A", (), {"steps": 2, "warmup": 1, "n": 512, "clusters": 3, "gpus": 1,
                          "prec": "bf16x3", "ref_seconds": 0.2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "TFLOP/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
