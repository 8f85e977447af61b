"""GPU parity of the FP64-accurate tile products on the tensor cores (exact slices, precision
"ozaki"): against the exact value of the segmented sliced product (oracle/ozaki_oracle.py: only
the FP64 accumulation order of the eight group sums and of the K segments separates the two),
against the FP64 product within the scheme's error bound, across K segments and ragged clusters,
inside mixed CLR products (low-rank blocks staged as reconstructions, densely accumulated
low-rank sums on the tensor cores), and in Newton–Schulz at the stated error."""
import numpy as np
import pytest

from oracle import clr_oracle as co
from oracle import ozaki_oracle as oz
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu

SEG = 1024   # the library's K segment (exponents per segment)


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
    (1100, None),                                   # 6 uneven clusters, 2 K segments
    (2300, [256, 1, 7, 200, 33, 256, 256, 191, 100, 256, 256, 256, 232]),  # 3 segments, ragged
])
def test_ozaki_matches_sliced_product_and_fp64(ctx, n, sizes):
    rng = np.random.default_rng(n)
    if sizes is None:
        sizes = wl.dense_normal(n=n, n_clusters=6, lo=128, hi=224, seed=77).row_sizes
    assert sum(sizes) == n
    a, b = _operands(rng, n)
    gc = ctx.multiply(ctx.from_dense(a, sizes), ctx.from_dense(b, sizes))
    got = gc.to_dense()
    want = oz.sliced_product(a, b, seg=SEG)
    # the group sums are exact on both sides; the FP64 sums over g and over K segments differ
    # only in rounding order
    scale = np.ldexp(1.0, oz.row_exponents(a)[:, None] + oz.row_exponents(b.T)[None, :])
    assert np.all(np.abs(got - want) <= 1e-14 * n * scale)
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)
    # and the FP64 product within the scheme's bound
    assert np.all(np.abs(got - a @ b) <= oz.error_bound(a, b, seg=SEG))
    k, _, _, _ = gc.get_blocks(pool=False)
    assert (k == co.KIND_DENSE).all()


def test_ozaki_inside_mixed_clr_product(ctx):
    # the 1D-chain product: every tile with a dense x dense product formed whole on the tensor
    # cores (low-rank operand blocks staged as reconstructions); each dense tile within the
    # slices' error of the oracle's FP64 sum
    from tests.test_gpu_product import _check_product
    w = wl.chain_overlap()
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    gs = clr_pack.to_library(ctx, s_or)
    gc = ctx.zeros(w.row_sizes)
    st = ctx.multiply_into(gs, gs, gc, stats=True)
    assert st["precision"] == "ozaki" and st["n_tiles_tensor"] >= st["n_tiles"][1]
    # K = 2048 terms, 2^-48-relative per term to the segment's largest entries; a densely
    # accumulated sum goes to the tensor cores with an expected error within eps / 64
    _check_product(ctx, s_or, s_or, w.eps_lr, gc, st, dense_rel=1e-12, lr_slack=w.eps_lr / 16)


def test_ozaki_densely_accumulated_low_rank_sums(ctx):
    # Dense diagonal blocks, low-rank off-diagonal blocks of rank 13 (3 clusters): an
    # off-diagonal C tile gets DL, LD and LL products of concatenated rank 39 > min/2, so it is
    # accumulated densely.  Its expected sliced error, 1.2 2^-48 sqrt(K_seg sum 4^e_i sum 4^f_j)
    # ~ 1.5e-10 here, times 4 is within eps/16 at eps = 1e-6 (the tensor cores sum it, DACC_G)
    # but not at eps = 1e-12 (FP64 low-rank products).  Either way the result matches the
    # oracle: dense tiles at the slices' accuracy, low-rank ones within eps (plus the sum's
    # error budget eps/16 where it was formed on the tensor cores).
    from tests.test_gpu_product import _check_product
    rng = np.random.default_rng(23)
    sizes = [64, 80, 72]
    for eps, want_gemm in ((1e-6, True), (1e-12, False)):
        def spec():
            out = []
            for i, m in enumerate(sizes):
                row = []
                for j, n in enumerate(sizes):
                    if i == j:
                        row.append((co.KIND_DENSE, rng.standard_normal((m, n))))
                    else:
                        row.append((co.KIND_LR, (rng.standard_normal((m, 13)),
                                                 rng.standard_normal((n, 13)))))
                out.append(row)
            return out
        a_or = co.from_blocks(sizes, sizes, spec())
        b_or = co.from_blocks(sizes, sizes, spec())
        ctx.set_opts(eps_lr=eps)
        gc = ctx.zeros(sizes)
        st = ctx.multiply_into(clr_pack.to_library(ctx, a_or), clr_pack.to_library(ctx, b_or),
                               gc, stats=True)
        # diagonal tiles hold a dense x dense product (tensor cores in both cases); the six
        # off-diagonal tiles are densely accumulated low-rank sums
        assert st["n_tiles_tensor"] == (9 if want_gemm else 3), st
        _check_product(ctx, a_or, b_or, eps, gc, dense_rel=1e-12,
                       lr_slack=eps / 16 if want_gemm else 0.0)
    ctx.set_opts(eps_lr=1e-8)
