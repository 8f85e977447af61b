"""Failure detection on the GPU without a fault: a bounded device-side wait of the tensor-core
pipeline is given a limit it must overrun (1 us, shorter than one accumulation segment of 96
MMAs), so the kernel gives up, drains its own copies and MMAs, frees its tensor memory and
returns.  The host then reads the error flag: CLR_ETIMEOUT at the next synchronising call, and
the context stays usable."""
import numpy as np
import pytest

from paper_1509_00309_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    ctx = clr.Context(0, precision="bf16x6", eps_lr=1e-8)
    w = wl.dense_normal(n=1024, n_clusters=6, lo=128, hi=224, seed=77)
    ga = ctx.from_dense(w.a, w.row_sizes)
    gb = ctx.from_dense(w.b, w.row_sizes)
    return clr, ctx, w, ga, gb


def _check_product(gc, w):
    want = w.a @ w.b
    err = np.linalg.norm(gc.to_dense() - want)
    assert err <= 1e-7 * np.linalg.norm(w.a) * np.linalg.norm(w.b)


def test_wait_timeout_is_reported_by_the_stats_call(setup):
    clr, ctx, w, ga, gb = setup
    gc = ctx.zeros(w.row_sizes)
    ctx.set_opts(wait_timeout_us=1)
    with pytest.raises(clr.ClrError) as e:
        ctx.multiply_into(ga, gb, gc, stats=True)
    assert e.value.status == clr.CLR_ETIMEOUT
    # the flag was cleared by that report; with the default limit the context works again
    ctx.set_opts(wait_timeout_us=0)
    ctx.multiply_into(ga, gb, gc, stats=True)
    _check_product(gc, w)


def test_wait_timeout_of_an_async_product_is_reported_by_check(setup):
    clr, ctx, w, ga, gb = setup
    gc = ctx.zeros(w.row_sizes)
    ctx.set_opts(wait_timeout_us=1)
    ctx.multiply_into(ga, gb, gc)          # asynchronous: cannot report
    ctx.set_opts(wait_timeout_us=0)
    with pytest.raises(clr.ClrError) as e:
        ctx.check()
    assert e.value.status == clr.CLR_ETIMEOUT
    ctx.check()                            # reported once, then cleared
    ctx.multiply_into(ga, gb, gc)
    ctx.check()
    _check_product(gc, w)
