"""Batched CLR products captured into one CUDA graph (clr_batch_*) and the autotuner."""
import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clr():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr


def _instances(n=8):
    # the batched 1D-chain workload, scaled down (N ~ U[1024,8192] * 0.12)
    return wl.batched_chains(n_instances=n, n_scale=0.12)


def test_batch_graph_matches_individual_products_and_oracle(clr, tmp_path):
    ws = _instances()
    ctx = clr.Context(0, precision="auto", eps_lr=1e-8)
    mats = [ctx.from_dense(w.a, w.row_sizes, eps_lr=w.eps_lr, drop_norm=w.drop_norm) for w in ws]
    eps = [w.eps_lr for w in ws]
    batch = ctx.batch(mats, mats, eps=eps, tune=True)
    assert ctx.autotune_entries() >= 1
    batch.run()
    outs = [batch.output(i).to_dense() for i in range(batch.n)]
    batch.run()   # graph replay gives the same bits
    for i in range(batch.n):
        assert np.array_equal(batch.output(i).to_dense(), outs[i])
    for i, w in enumerate(ws):
        t = batch.tuning(i)
        # the same product through the regular entry point with the chosen configuration
        single = clr.Context(0, precision=t["precision"], eps_lr=eps[i])
        si = single.from_dense(w.a, w.row_sizes, eps_lr=w.eps_lr, drop_norm=w.drop_norm)
        ref = single.multiply(si, si).to_dense()
        assert np.array_equal(outs[i], ref), (i, t)
    for i in (0, len(ws) - 1):
        w = ws[i]
        s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
        want = co.multiply(s_or, s_or, w.eps_lr).to_dense()
        tol = co.product_tolerance(w.a, w.a, w.eps_lr)
        assert np.linalg.norm(outs[i] - want) <= tol
    # the autotuner cache survives a save / load round trip
    path = str(tmp_path / "tune.txt")
    ctx.autotune_save(path)
    ctx2 = clr.Context(0, precision="auto")
    ctx2.autotune_load(path)
    assert ctx2.autotune_entries() == ctx.autotune_entries()
    batch.close()


def test_multiply_batched_hands_out_outputs(clr):
    ws = _instances(5)
    ctx = clr.Context(0, precision="fp64", eps_lr=1e-8)
    mats = [ctx.from_dense(w.a, w.row_sizes, eps_lr=1e-8, drop_norm=1e-12) for w in ws]
    outs = ctx.multiply_batched(mats, mats)
    for m, o in zip(mats, outs):
        assert np.array_equal(o.to_dense(), ctx.multiply(m, m).to_dense())
