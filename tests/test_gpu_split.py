"""GPU parity of the split-precision (bf16 terms on tcgen05 tensor cores) dense x dense tile
products against the oracle: the exact value of the split product (oracle/split_oracle.py,
which isolates the FP32 accumulation), the FP64 product at the product tolerance
10 eps ||A||_F ||B||_F, and sampled tiles at the full 16384 size."""
import math

import numpy as np
import pytest

from oracle import clr_oracle as co
from oracle import split_oracle as so
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr.Context(0, precision="bf16x3", eps_lr=1e-8)


@pytest.fixture(scope="module")
def dense_case():
    # ragged against the 128 x 256 GEMM tiles and the 32-wide k chunks
    return wl.dense_normal(n=1100, n_clusters=6, lo=128, hi=224, seed=77)


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
def test_split_matches_exact_split_product(ctx, dense_case, mode):
    w = dense_case
    ctx.set_opts(precision=mode)
    ga, gb = ctx.from_dense(w.a, w.row_sizes), ctx.from_dense(w.b, w.row_sizes)
    gc = ctx.zeros(w.row_sizes)
    st = ctx.multiply_into(ga, gb, gc, stats=True)
    assert st["precision"] == mode
    got = gc.to_dense()
    want = so.split_product(w.a, w.b, mode)
    # only FP32 accumulation separates the two: far below the 2^-16 effect of a dropped
    # bf16x6 term pair and the 2^-8 effect of a wrong bf16x3 pair
    assert np.linalg.norm(got - want) <= 2.0 ** -18 * np.linalg.norm(want)


def test_bf16x6_meets_product_tolerance(ctx, dense_case):
    w = dense_case
    ctx.set_opts(precision="bf16x6")
    gc = ctx.multiply(ctx.from_dense(w.a, w.row_sizes), ctx.from_dense(w.b, w.row_sizes))
    err = np.linalg.norm(gc.to_dense() - w.a @ w.b)
    assert err <= co.product_tolerance(w.a, w.b, 1e-8)


@pytest.mark.parametrize("mode,rel", [("bf16x3", 2.0 ** -16), ("bf16x6", 2.0 ** -23)])
def test_product_with_identity_returns_split_of_a(ctx, mode, rel):
    # A I = A up to the split's truncation: |C - A| <= 2^-16 |A| (bf16x3), 2^-24-ish (bf16x6)
    rng = np.random.default_rng(3)
    sizes = [200, 56, 256, 17]
    n = sum(sizes)
    a = rng.standard_normal((n, n)) * np.exp(rng.uniform(-3, 3, (n, n)))
    ctx.set_opts(precision=mode)
    ga = ctx.from_dense(a, sizes)
    gi = ctx.from_dense(np.eye(n), sizes)
    got = ctx.multiply(ga, gi).to_dense()
    assert np.all(np.abs(got - a) <= rel * np.abs(a) + 1e-300)
    if mode == "bf16x3":
        # where a_0 + a_1 is an FP32 value the tensor-core sum is exact, so the GPU's integer
        # bf16 rounding must reproduce the oracle's terms bit for bit there
        t = so.split_terms(a, 2)
        s2 = t[0] + t[1]
        exact = s2.astype(np.float32).astype(np.float64) == s2
        assert exact.mean() > 0.99
        assert np.array_equal(got[exact], s2[exact])


def test_split_inside_mixed_clr_product(ctx):
    # chain overlap: dense x dense products on the tensor cores, low-rank products in FP64
    w = wl.chain_overlap()
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    ctx.set_opts(precision="bf16x6")
    gs = clr_pack.to_library(ctx, s_or)
    gc = ctx.zeros(w.row_sizes)
    st = ctx.multiply_into(gs, gs, gc, stats=True)
    tl = co.triple_list(s_or, s_or)
    assert st["n_triples"] == [int(v) for v in np.bincount(tl.triples[:, 3], minlength=4)]
    want = co.multiply(s_or, s_or, w.eps_lr)
    g = clr_pack.from_library(gc)
    assert np.array_equal(g.kinds(), want.kinds())
    err = np.linalg.norm(g.to_dense() - want.to_dense())
    assert err <= co.product_tolerance(w.a, w.a, w.eps_lr)
    # every dense tile is summed entirely by the tensor cores (low-rank operand blocks staged as
    # their reconstructions): it equals the exact split product of the reconstructed block row
    # and column up to the FP32 accumulation
    sd = s_or.to_dense()
    for i in range(len(w.row_sizes)):
        for j in range(len(w.row_sizes)):
            if g.kinds()[i, j] != co.KIND_DENSE:
                continue
            rows = slice(s_or.row_off[i], s_or.row_off[i + 1])
            cols = slice(s_or.col_off[j], s_or.col_off[j + 1])
            exact = so.split_product(sd[rows], sd[:, cols], "bf16x6")
            d = np.linalg.norm(g.block_dense(i, j) - exact)
            assert d <= 2.0 ** -18 * np.linalg.norm(exact), (i, j, d)


def test_full_size_sampled_tiles(ctx):
    # the all-dense workload at full size (N = 16384, 96 uneven clusters, bf16x3), in the
    # launch configuration the benchmark times; sampled C tiles against FP64 dot products
    import torch
    w = wl.dense_normal()
    ctx.set_opts(precision="bf16x3")
    ga = ctx.from_dense(w.a, w.row_sizes)
    gb = ctx.from_dense(w.b, w.row_sizes)
    gc = ctx.zeros(w.row_sizes)
    ctx.multiply_into(ga, gb, gc)
    out = torch.empty((w.n, w.n), dtype=torch.float64, device="cuda")
    gc.to_dense(out)
    torch.cuda.synchronize()
    off = np.concatenate([[0], np.cumsum(w.row_sizes)])
    num, den, ab = 0.0, 0.0, 0.0
    # whole block rows (every column cluster) and whole block columns (every row cluster):
    # the first and last, the ones across the middle of the 128 x 256 GEMM grid, and two more
    j_mid = int(np.searchsorted(off, (w.n // 256) // 2 * 256, side="right")) - 1
    i_mid = int(np.searchsorted(off, (w.n // 128) // 2 * 128, side="right")) - 1
    host = out.cpu().numpy()
    for i in (0, 95, i_mid, 33):
        r0, r1 = off[i], off[i + 1]
        want = w.a[r0:r1] @ w.b
        got = host[r0:r1]
        num += float(np.sum((got - want) ** 2))
        den += float(np.sum(want ** 2))
        ab += float(np.sum(np.linalg.norm(w.a[r0:r1], axis=1)[:, None] ** 2 *
                           np.linalg.norm(w.b, axis=0)[None, :] ** 2))
    for j in (0, 95, j_mid, 61):
        c0, c1 = off[j], off[j + 1]
        want = w.a @ w.b[:, c0:c1]
        got = host[:, c0:c1]
        num += float(np.sum((got - want) ** 2))
        den += float(np.sum(want ** 2))
        ab += float(np.sum(np.linalg.norm(w.a, axis=1)[:, None] ** 2 *
                           np.linalg.norm(w.b[:, c0:c1], axis=0)[None, :] ** 2))
    # per-sample form of ||dC||_F <= 10 eps ||A||_F ||B||_F with eps = 1e-8:
    # sum over sampled entries of dC^2 <= (10 eps)^2 * sum ||a_i||^2 ||b_j||^2
    assert num <= (10 * 1e-8) ** 2 * ab
    assert math.sqrt(num / den) < 3e-5
    # the whole matrix: every block is dense, and the block norms (formed in the GEMM's
    # epilogue) add up to ||C||_F
    k, _, _, _ = gc.get_blocks(pool=False)
    assert (k == co.KIND_DENSE).all()
    del host
    fro = float(torch.linalg.norm(out))
    assert abs(gc.info()["frob_norm"] - fro) <= 1e-12 * fro


def test_low_rank_sums_on_tensor_cores_follow_error_bound(ctx):
    # Dense diagonal blocks, low-rank off-diagonal blocks of rank 13 (3 clusters): an
    # off-diagonal C tile gets DL, LD and LL products of concatenated rank 39 > min/2, so it is
    # accumulated densely.  With the off-diagonal blocks scaled to 1e-10 its split error bound
    # u sum_K ||A_IK|| ||B_KJ|| is below eps/16 and the tensor-core GEMM sums it; at scale 1 the
    # low-rank products stay in FP64.  Either way the result matches the oracle.
    from tests.test_gpu_product import _check_product
    rng = np.random.default_rng(21)
    sizes = [64, 80, 72]
    eps = 1e-8
    for scale, want_gemm in ((1e-10, True), (1.0, False)):
        def spec():
            out = []
            for i, m in enumerate(sizes):
                row = []
                for j, n in enumerate(sizes):
                    if i == j:
                        row.append((co.KIND_DENSE, rng.standard_normal((m, n))))
                    else:
                        row.append((co.KIND_LR, (scale * rng.standard_normal((m, 13)),
                                                 rng.standard_normal((n, 13)))))
                out.append(row)
            return out
        a_or = co.from_blocks(sizes, sizes, spec())
        b_or = co.from_blocks(sizes, sizes, spec())
        # bf16x6: at K ~ 200 the bf16x3 error 2^-16 ||A|| ||B|| / sqrt(K) exceeds the product
        # tolerance 10 eps ||A|| ||B|| for eps = 1e-8
        ctx.set_opts(precision="bf16x6", eps_lr=eps)
        gc = ctx.zeros(sizes)
        st = ctx.multiply_into(clr_pack.to_library(ctx, a_or), clr_pack.to_library(ctx, b_or),
                               gc, stats=True)
        # diagonal tiles hold a dense x dense product (tensor cores in both cases); the six
        # off-diagonal tiles are densely accumulated low-rank sums
        assert st["n_tiles_tensor"] == (9 if want_gemm else 3)
        _check_product(ctx, a_or, b_or, eps, gc, split_mode="bf16x6")
    ctx.set_opts(precision="bf16x3", eps_lr=1e-8)


@pytest.mark.parametrize("mode", ["bf16x3", "fp64"])
def test_streamed_host_product_equals_regular_product(ctx, mode):
    # C = A B for page-locked host matrices, A in 2 row chunks and B in 3 column chunks, the 6
    # tile products on two streams (each row chunk's panels staged once): every entry equals
    # the regular product's, which runs the same k order
    import torch
    from paper_1509_00309_gb300 import clr
    rng = np.random.default_rng(71)
    rs, ks, cs = [130, 77, 200], [64, 190, 33, 90], [100, 60, 150, 41, 90]
    m, k, n = sum(rs), sum(ks), sum(cs)
    a = torch.from_numpy(rng.standard_normal((m, k))).pin_memory()
    b = torch.from_numpy(rng.standard_normal((k, n))).pin_memory()
    c = torch.full((m, n), np.nan, dtype=torch.float64).pin_memory()
    ctx.set_opts(precision=mode)
    ctx.multiply_host_stream(a, b, c, rs, ks, cs, n_chunks=3)
    ga = ctx.from_dense(a.numpy(), rs, ks)
    gb = ctx.from_dense(b.numpy(), ks, cs)
    want = ctx.multiply(ga, gb).to_dense()
    assert np.array_equal(c.numpy(), want)
    ref = a.numpy() @ b.numpy()
    an, bn = np.linalg.norm(a.numpy()), np.linalg.norm(b.numpy())
    # fp64: the product tolerance at eps 1e-8; bf16x3 at K ~ 400: its ~2^-16 / sqrt(K) error
    bound = co.product_tolerance(a.numpy(), b.numpy(), 1e-8) if mode == "fp64" else \
        2.0 ** -16 * an * bn
    assert np.linalg.norm(c.numpy() - ref) <= bound
    with pytest.raises(clr.ClrError) as e:   # pageable buffers are refused
        ctx.multiply_host_stream(torch.zeros((m, k)), b, c, rs, ks, cs)
    assert e.value.status == clr.CLR_EINVAL
    a[m - 1, 5] = float("nan")                 # a non-finite value in A's second row chunk
    with pytest.raises(clr.ClrError) as e:
        ctx.multiply_host_stream(a, b, c, rs, ks, cs, n_chunks=3)
    assert e.value.status == clr.CLR_EINVAL
    ctx.set_opts(precision="bf16x3")


@pytest.mark.parametrize("terms", [2, 3])
def test_device_split_terms_bit_exact(ctx, terms):
    """The device's bf16 term split (the staging kernels' paired split, with its hardware
    bf16x2 conversion) bit for bit against the oracle's split from the bf16 format's
    definition, on values over the whole range and the rounding edge cases."""
    import torch
    from paper_1509_00309_gb300 import clr
    from tests.test_split_rounding_host import bf16_bits, cases
    rng = np.random.default_rng(1510)
    x = cases(rng)
    x = np.concatenate([x, rng.permutation(x), x[:1]])   # odd count: a lone last value
    got = clr.split_bf16(torch.from_numpy(x).cuda(), terms).cpu().numpy().view(np.uint16)
    for t, want in enumerate(so.split_terms(x, terms)):
        w = bf16_bits(want)
        bad = np.nonzero(got[t] != w)[0]
        assert bad.size == 0, (t, x[bad[:5]], got[t, bad[:5]], w[bad[:5]])


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("sizes", [None, [40, 17, 200, 64, 33, 250]])
def test_block_norms_after_split_product(ctx, dense_case, mode, sizes):
    # The dense tiles' norms of a split product (formed in the dense kernel's epilogue when every
    # row cluster has >= 32 rows and every column cluster >= 16, else by a separate pass) equal
    # the norms of the stored blocks: sqrt(sum of squared block norms) = ||C||_F
    w = dense_case
    rs = w.row_sizes if sizes is None else sizes
    a, b = w.a[:sum(rs), :sum(rs)], w.b[:sum(rs), :sum(rs)]
    ctx.set_opts(precision=mode)
    gc = ctx.multiply(ctx.from_dense(a, rs), ctx.from_dense(b, rs))
    c = gc.to_dense()
    assert abs(gc.info()["frob_norm"] - np.linalg.norm(c)) <= 1e-13 * np.linalg.norm(c)
    ctx.set_opts(precision="bf16x3")


def test_block_norms_mixed_routes_split(ctx):
    # a product with dense and low-rank C tiles (1D chain overlap, bf16x6): the dense tiles'
    # epilogue norms and the recompressed tiles' norms together give ||C||_F
    w = wl.chain_overlap()
    ctx.set_opts(precision="bf16x6", eps_lr=w.eps_lr)
    s = ctx.from_dense(w.a, w.row_sizes, eps_lr=w.eps_lr, drop_norm=w.drop_norm)
    gc = ctx.multiply(s, s)
    c = gc.to_dense()
    nb = gc.info()["n_blocks"]     # zero, dense, low rank
    assert nb[1] > 0 and nb[2] > 0
    assert abs(gc.info()["frob_norm"] - np.linalg.norm(c)) <= 1e-12 * np.linalg.norm(c)
    ctx.set_opts(precision="bf16x3", eps_lr=1e-8)
