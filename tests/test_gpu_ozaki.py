"""GPU parity of the FP64-accurate dense x dense tile products on the tensor cores (exact
slices, precision "ozaki"): against the exact value of the sliced product (oracle/ozaki_oracle.py:
only the FP64 accumulation order of the seven group sums separates the two), against the FP64
product within the scheme's error bound, across K segments and ragged clusters, inside mixed CLR
products, and in Newton–Schulz at the stated error."""
import numpy as np
import pytest

from oracle import clr_oracle as co
from oracle import ozaki_oracle as oz
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr.Context(0, precision="ozaki", eps_lr=1e-8)


def _operands(rng, n, spread=4.0):
    a = rng.standard_normal((n, n)) * np.exp(rng.uniform(-spread, spread, (n, 1)))
    b = rng.standard_normal((n, n)) * np.exp(rng.uniform(-spread, spread, (1, n)))
    return a, b


@pytest.mark.parametrize("n,sizes", [
    (1100, None),                                   # 6 uneven clusters, one K segment
    (2300, [256, 1, 7, 200, 33, 256, 256, 191, 100, 256, 256, 256, 232]),  # 2 segments, ragged
])
def test_ozaki_matches_sliced_product_and_fp64(ctx, n, sizes):
    rng = np.random.default_rng(n)
    if sizes is None:
        sizes = wl.dense_normal(n=n, n_clusters=6, lo=128, hi=224, seed=77).row_sizes
    assert sum(sizes) == n
    a, b = _operands(rng, n)
    gc = ctx.multiply(ctx.from_dense(a, sizes), ctx.from_dense(b, sizes))
    got = gc.to_dense()
    want = oz.sliced_product(a, b)
    # the group sums are exact on both sides; the FP64 sums over g and over K segments differ
    # only in rounding order
    scale = np.ldexp(1.0, oz.row_exponents(a)[:, None] + oz.row_exponents(b.T)[None, :])
    assert np.all(np.abs(got - want) <= 1e-14 * n * scale)
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)
    # and the FP64 product within the scheme's bound
    assert np.all(np.abs(got - a @ b) <= oz.error_bound(a, b))
    k, _, _, _ = gc.get_blocks(pool=False)
    assert (k == co.KIND_DENSE).all()


def test_ozaki_inside_mixed_clr_product(ctx):
    # the 1D-chain product: dense x dense on the tensor cores by exact slices, low-rank
    # contributions in FP64; every dense tile within the slices' error of the oracle's FP64 sum
    from tests.test_gpu_product import _check_product
    w = wl.chain_overlap()
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    gs = clr_pack.to_library(ctx, s_or)
    gc = ctx.zeros(w.row_sizes)
    st = ctx.multiply_into(gs, gs, gc, stats=True)
    assert st["precision"] == "ozaki" and st["n_tiles_tensor"] == st["n_tiles"][1]
    # K ~ 2048 terms of 2^-39-relative truncation: 1e-10 |A||B| per tile bounds it
    _check_product(ctx, s_or, s_or, w.eps_lr, gc, st, dense_rel=1e-10)
