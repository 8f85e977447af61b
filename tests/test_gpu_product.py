"""GPU parity of the CLR product (FP64 path) against the FP64 oracle, through the C ABI."""
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
    return clr.Context(0, precision="fp64", eps_lr=1e-8)


def _check_product(ctx, a_or, b_or, eps, got, stats=None, split_mode=None, dense_rel=1e-13,
                   lr_slack=0.0):
    """Compare a GPU product with the oracle's: reconstruction within the truncation bound,
    kinds equal (ranks within one of the oracle's at the threshold), and every dense tile
    against its exact value.  FP64 tile products (split_mode None): the oracle's FP64 tile sum
    up to rounding -- the two sum the same exact products in different orders (dense x dense
    blocks whole, low-rank ones in factored form), so they differ by a few units of
    u |A_I*| |B_*J| (bound 1e-13 |A||B|, about 450 u, far below any dropped or misplaced
    contribution).  Split precision: a dense tile is summed entirely by the tensor cores (the
    low-rank operand blocks staged as their reconstructions), so it equals the exact split
    product of the reconstructed block row and column up to the FP32 accumulation (2^-18).
    lr_slack: what a low-rank tile may exceed its truncation bound by when the sum it truncates
    carries a product error (densely accumulated sums formed on the tensor cores)."""
    want = co.multiply(a_or, b_or, eps)
    g = clr_pack.from_library(got)
    da, db = a_or.to_dense(), b_or.to_dense()
    ref = da @ db
    absab = so.abs_product(da, db)
    err = np.linalg.norm(g.to_dense() - want.to_dense())
    tol = co.product_tolerance(da, db, max(eps, 1e-12))
    assert err <= tol, (err, tol)
    # every low-rank tile is within eps of the exact tile sum (truncation bound)
    gk, wk = g.kinds(), want.kinds()
    gr, wr = g.ranks(), want.ranks()
    for i in range(len(a_or.row_sizes)):
        for j in range(len(b_or.col_sizes)):
            if gk[i, j] == wk[i, j] == co.KIND_DENSE:
                rows = slice(a_or.row_off[i], a_or.row_off[i + 1])
                cols = slice(b_or.col_off[j], b_or.col_off[j + 1])
                if split_mode is None:
                    d = np.linalg.norm(g.block_dense(i, j) - want.block_dense(i, j))
                    assert d <= dense_rel * np.linalg.norm(absab[rows, cols]) + 1e-300, \
                        (i, j, d)
                else:
                    exact = so.split_product(da[rows], db[:, cols], split_mode)
                    d = np.linalg.norm(g.block_dense(i, j) - exact)
                    assert d <= 2.0 ** -18 * np.linalg.norm(exact) + 1e-300, (i, j, d)
            if gk[i, j] != wk[i, j]:
                # a kind may only differ at the dense/low-rank threshold
                lim = co.dense_rank_limit(a_or.row_sizes[i], b_or.col_sizes[j])
                assert {gk[i, j], wk[i, j]} <= {co.KIND_DENSE, co.KIND_LR}
                assert max(gr[i, j], wr[i, j]) >= lim
                continue
            if gk[i, j] == co.KIND_LR:
                assert abs(int(gr[i, j]) - int(wr[i, j])) <= 1
                blk = ref[a_or.row_off[i]:a_or.row_off[i + 1], b_or.col_off[j]:b_or.col_off[j + 1]]
                scale = np.abs(blk).sum() + 1.0
                assert (np.linalg.norm(g.block_dense(i, j) - blk) <=
                        eps * (1 + 1e-6) + lr_slack + 1e-13 * scale)
    if stats is not None:
        tl = co.triple_list(a_or, b_or)
        kinds = np.bincount(tl.triples[:, 3], minlength=4) if len(tl.triples) else np.zeros(4)
        assert stats["n_triples"] == [int(v) for v in kinds]
        assert stats["flops"] == int(tl.flops.sum())
        modes = np.bincount(tl.tile_mode.ravel(), minlength=3)
        assert stats["n_tiles"] == [int(v) for v in modes]
    return err


@pytest.mark.parametrize("seed", range(8))
def test_random_structures_all_kinds(ctx, seed):
    rng = np.random.default_rng(1000 + seed)
    nb = int(rng.integers(2, 5))
    sizes = [int(s) for s in rng.integers(1, 40, size=nb)]
    if seed == 0:
        sizes = [1, 7, 33]
    a = co.from_blocks(sizes, sizes, wl.random_blocks_spec(rng, sizes, sizes))
    b = co.from_blocks(sizes, sizes, wl.random_blocks_spec(rng, sizes, sizes))
    ga, gb = clr_pack.to_library(ctx, a), clr_pack.to_library(ctx, b)
    gc = ctx.zeros(sizes, sizes)
    stats = ctx.multiply_into(ga, gb, gc, stats=True)
    _check_product(ctx, a, b, 1e-8, gc, stats)


def test_rectangular_and_max_cluster(ctx):
    rng = np.random.default_rng(7)
    rs, ks, cs = [256, 5], [200, 256, 3], [17, 256]
    a = co.from_blocks(rs, ks, wl.random_blocks_spec(rng, rs, ks, p_zero=0.1))
    b = co.from_blocks(ks, cs, wl.random_blocks_spec(rng, ks, cs, p_zero=0.1))
    gc = ctx.multiply(clr_pack.to_library(ctx, a), clr_pack.to_library(ctx, b))
    _check_product(ctx, a, b, 1e-8, gc)


def test_low_rank_sum_recompression_ranks(ctx):
    # a tile fed only by low-rank products: ranks after recompression equal the oracle's
    rng = np.random.default_rng(11)
    sizes = [48, 40, 56]
    spec = [[(2, (rng.standard_normal((m, 3)), rng.standard_normal((n, 3)))) for n in sizes]
            for m in sizes]
    a = co.from_blocks(sizes, sizes, spec)
    gc = ctx.multiply(clr_pack.to_library(ctx, a), clr_pack.to_library(ctx, a))
    g = clr_pack.from_library(gc)
    want = co.multiply(a, a, 1e-8)
    assert np.array_equal(g.kinds(), want.kinds())
    assert np.array_equal(g.ranks(), want.ranks())
    ref = a.to_dense() @ a.to_dense()
    for i in range(3):
        for j in range(3):
            blk = ref[a.row_off[i]:a.row_off[i + 1], a.col_off[j]:a.col_off[j + 1]]
            s_ref = np.linalg.svd(blk, compute_uv=False)
            r = want.ranks()[i, j]
            s_got = np.linalg.svd(g.block_dense(i, j), compute_uv=False)[:r]
            assert np.allclose(s_got, s_ref[:r], rtol=1e-11, atol=1e-12 * s_ref[0])


def test_all_zero_product(ctx):
    sizes = [5, 9]
    a = co.CLR(sizes, sizes)
    gc = ctx.multiply(clr_pack.to_library(ctx, a), clr_pack.to_library(ctx, a))
    k, r, n, _ = gc.get_blocks(pool=False)
    assert not k.any() and not r.any() and not n.any()
    assert not gc.to_dense().any()


def test_from_dense_matches_oracle_build(ctx):
    w = wl.chain_overlap(n=512, n_clusters=4, lo=96, hi=160)
    m = ctx.from_dense(w.a, w.row_sizes, eps_lr=w.eps_lr, drop_norm=w.drop_norm)
    want = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    g = clr_pack.from_library(m)
    assert np.array_equal(g.kinds(), want.kinds())
    assert np.abs(g.ranks().astype(int) - want.ranks().astype(int)).max() <= 1
    for (i, j) in want.blocks:
        blk = w.a[want.row_off[i]:want.row_off[i + 1], want.col_off[j]:want.col_off[j + 1]]
        assert np.linalg.norm(g.block_dense(i, j) - blk) <= w.eps_lr * (1 + 1e-6) + 1e-14
    # device input path gives the same matrix
    import torch
    m2 = ctx.from_dense(torch.from_numpy(w.a).cuda(), w.row_sizes, eps_lr=w.eps_lr,
                        drop_norm=w.drop_norm)
    assert np.array_equal(m2.to_dense(), m.to_dense())


def test_chain_overlap_product_full_size(ctx):
    # the 1D-chain workload at its full size: N = 2048, 16 uneven clusters, eps = 1e-8
    w = wl.chain_overlap()
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    gs = clr_pack.to_library(ctx, s_or)
    gc = ctx.zeros(w.row_sizes)
    stats = ctx.multiply_into(gs, gs, gc, stats=True)
    err = _check_product(ctx, s_or, s_or, w.eps_lr, gc, stats)
    assert err <= co.product_tolerance(w.a, w.a, w.eps_lr)


def test_all_dense_product_matches_gemm(ctx):
    w = wl.dense_normal(n=1100, n_clusters=6)
    ga = ctx.from_dense(w.a, w.row_sizes)
    gb = ctx.from_dense(w.b, w.row_sizes)
    gc = ctx.multiply(ga, gb)
    ref = w.a @ w.b
    got = gc.to_dense()
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref) * math.sqrt(1100)
    k, _, _, _ = gc.get_blocks(pool=False)
    assert (k == co.KIND_DENSE).all()


def test_lincomb_matches_oracle(ctx):
    rng = np.random.default_rng(21)
    sizes = [30, 45, 20]
    x = co.from_blocks(sizes, sizes, wl.random_blocks_spec(rng, sizes, sizes, max_rank=4))
    y = co.from_blocks(sizes, sizes, wl.random_blocks_spec(rng, sizes, sizes, max_rank=4))
    out = ctx.lincomb(-1.25, clr_pack.to_library(ctx, x), 0.375, clr_pack.to_library(ctx, y),
                      1.875)
    want = co.lincomb(-1.25, x, 0.375, y, 1.875, 1e-8)
    g = clr_pack.from_library(out)
    assert np.array_equal(g.kinds(), want.kinds())
    assert np.linalg.norm(g.to_dense() - want.to_dense()) <= 1e-12 * np.linalg.norm(want.to_dense()) + 9e-8


def test_transpose_and_matvec(ctx):
    rng = np.random.default_rng(5)
    rs, cs = [12, 30], [7, 25, 9]
    a = co.from_blocks(rs, cs, wl.random_blocks_spec(rng, rs, cs))
    ga = clr_pack.to_library(ctx, a)
    at = ctx.transpose(ga)
    assert np.array_equal(at.to_dense(), a.to_dense().T)
    import torch
    x = torch.randn(sum(cs), dtype=torch.float64, device="cuda")
    y = torch.empty(sum(rs), dtype=torch.float64, device="cuda")
    ctx.matvec(ga, x, y)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy(), a.to_dense() @ x.cpu().numpy(), rtol=1e-13, atol=1e-12)


def test_errors_are_reported(ctx):
    from paper_1509_00309_gb300 import clr
    a = ctx.zeros([4, 5], [3, 3])
    b = ctx.zeros([4, 2], [3])
    with pytest.raises(clr.ClrError) as e:
        ctx.multiply(a, b)
    assert e.value.status == clr.CLR_EINVAL
    with pytest.raises(clr.ClrError) as e:
        ctx.zeros([257])
    assert e.value.status == clr.CLR_EINVAL
    bad = np.ones((8, 8))
    bad[3, 4] = np.nan
    with pytest.raises(clr.ClrError) as e:
        ctx.from_dense(bad, [8], eps_lr=1e-8)
    assert e.value.status == clr.CLR_EINVAL
    c = ctx.zeros([4, 5], [4, 5])
    with pytest.raises(clr.ClrError):
        ctx.multiply_into(c, c, c)


@pytest.mark.parametrize("no_prereduce", [0, 1])
def test_build_svd_shared_memory_placements(ctx, no_prereduce):
    # clusters of 256 (FP32 copies of the SVD in global scratch), 200 (G32 in shared memory,
    # V32 in scratch) and 37 (both in shared memory), on a smooth kernel whose blocks need
    # both FP32 stages and the FP64 clean-up to reach eps = 1e-8; with the pivoted-QR
    # pre-reduction (the SVD of R) and without it (the full SVD of every block)
    sizes = [256, 200, 37]
    n = sum(sizes)
    r = np.linspace(0.0, 0.02 * n, n) + np.random.default_rng(3).uniform(-0.004, 0.004, n)
    a = np.exp(-(r[:, None] - r[None, :]) ** 2 / 2.0) + 1e-3 * np.eye(n)
    eps = 1e-8
    ctx.set_opts(svd_no_prereduce=no_prereduce)
    try:
        m = ctx.from_dense(a, sizes, eps_lr=eps)
    finally:
        ctx.set_opts(svd_no_prereduce=0)
    want = co.build(a, sizes, sizes, eps)
    g = clr_pack.from_library(m)
    gk, wk, gr, wr = g.kinds(), want.kinds(), g.ranks(), want.ranks()
    assert (wk == co.KIND_LR).sum() >= 4
    for i in range(3):
        for j in range(3):
            blk = a[want.row_off[i]:want.row_off[i + 1], want.col_off[j]:want.col_off[j + 1]]
            if gk[i, j] != wk[i, j]:
                lim = co.dense_rank_limit(sizes[i], sizes[j])
                assert max(gr[i, j], wr[i, j]) >= lim
                continue
            if gk[i, j] == co.KIND_LR:
                assert abs(int(gr[i, j]) - int(wr[i, j])) <= 1
                assert np.linalg.norm(g.block_dense(i, j) - blk) <= eps * (1 + 1e-6)
            elif gk[i, j] == co.KIND_DENSE:
                assert np.array_equal(g.block_dense(i, j), blk)


def _spectrum_block(m, n, lead, tail_top, eps, seed):
    """U diag(s) V^T with orthonormal U, V: `lead` singular values from 1 down to 1e-2, then a
    geometric tail of the remaining min(m, n) - lead values from tail_top eps down to
    2e-3 tail_top eps."""
    rng = np.random.default_rng(seed)
    q = min(m, n)
    u, _ = np.linalg.qr(rng.standard_normal((m, q)))
    v, _ = np.linalg.qr(rng.standard_normal((n, q)))
    rho = (2e-3) ** (1.0 / (q - lead - 1))
    s = np.concatenate([np.logspace(0, -2, lead), tail_top * eps * rho ** np.arange(q - lead)])
    return (u * s) @ v.T, s


@pytest.mark.parametrize("m,n", [(200, 200), (150, 230)])
def test_build_pivoted_qr_past_three_fifths_takes_svd_of_r(ctx, m, n):
    # Tiles whose column-pivoted QR needs more than 3q/5 steps to reach eps/16 (the geometric
    # tail: about 160 of 200 and 120 of 150 steps) and whose rank the QR's triangles cannot
    # certify (sigma_min(R_11) ~ 0.02-0.16 eps, the tail bound ~ 0.02-0.2 eps^2): the SVD of
    # the QR's factor R decides.  With 0.45 q leading values and the tail from 0.3 eps the
    # tail beyond them holds ~0.2 eps^2: low rank at the oracle's rank (within one), within
    # eps.  With q/2 leading values and the tail from 0.5 eps the tail beyond q/2 holds
    # ~1.6-2.1 eps^2: dense, stored as the block itself.  The profile counters show the path
    # (pivoted QR and the SVD of R, stored low rank / stored dense).
    eps = 1e-8
    q = min(m, n)
    for lead, top, want_dense in ((int(0.45 * q), 0.3, False), (q // 2, 0.5, True)):
        a, s = _spectrum_block(m, n, lead, top, eps, seed=11)
        r_or = co.compress_block(a, eps).rank
        assert (r_or > co.dense_rank_limit(m, n)) == want_dense
        ctx.profile_enable(True)
        try:
            mat = ctx.from_dense(a, [m], [n], eps_lr=eps)
            prof = ctx.profile_read()
        finally:
            ctx.profile_enable(False)
        g = clr_pack.from_library(mat)
        paths = prof["svd_path_blocks"]
        if want_dense:
            assert g.kinds()[0, 0] == co.KIND_DENSE
            assert np.array_equal(g.block_dense(0, 0), a)
            assert paths == [0, 0, 0, 1], paths
        else:
            assert g.kinds()[0, 0] == co.KIND_LR
            assert abs(int(g.ranks()[0, 0]) - r_or) <= 1 and r_or == lead
            assert np.linalg.norm(g.block_dense(0, 0) - a) <= eps * (1 + 1e-6)
            assert paths == [1, 0, 0, 0], paths


def test_rrqr_build_matches_oracle(ctx):
    # the paper's construction (Section 4.1): rank-revealing QR with greedy column pivoting,
    # truncated at ||R_22||_F <= eps; ranks as the oracle's step-by-step pivoted QR (within one
    # where a pivot is decided by rounding), errors within eps, never below the SVD's rank
    w = wl.chain_overlap(n=640, n_clusters=5, lo=96, hi=160)
    eps = 1e-8
    ctx.set_opts(build_rrqr=1)
    try:
        m = ctx.from_dense(w.a, w.row_sizes, eps_lr=eps, drop_norm=w.drop_norm)
    finally:
        ctx.set_opts(build_rrqr=0)
    want = co.build(w.a, w.row_sizes, w.col_sizes, eps, w.drop_norm, rrqr=True)
    svd = co.build(w.a, w.row_sizes, w.col_sizes, eps, w.drop_norm)
    g = clr_pack.from_library(m)
    gk, wk, gr, wr = g.kinds(), want.kinds(), g.ranks(), want.ranks()
    assert (wk == co.KIND_LR).sum() >= 6
    for (i, j) in want.blocks:
        blk = w.a[want.row_off[i]:want.row_off[i + 1], want.col_off[j]:want.col_off[j + 1]]
        if gk[i, j] != wk[i, j]:
            lim = co.dense_rank_limit(blk.shape[0], blk.shape[1])
            assert max(gr[i, j], wr[i, j]) >= lim
            continue
        if gk[i, j] == co.KIND_LR:
            assert abs(int(gr[i, j]) - int(wr[i, j])) <= 1
            assert gr[i, j] >= svd.ranks()[i, j]
            assert np.linalg.norm(g.block_dense(i, j) - blk) <= eps * (1 + 1e-6)
            x = g.blocks[(i, j)].x
            assert np.allclose(x.T @ x, np.eye(x.shape[1]), atol=1e-12)   # X = Q_r


@pytest.mark.parametrize("no_prereduce", [0, 1])
def test_build_tight_cluster_least_squares_factor(ctx, no_prereduce):
    # A tight cluster of kept singular values (40 values 1 + 1e-12 k) keeps the FP64 Jacobi from
    # converging within its sweep cap; the right factor is then the least-squares one and X W^T
    # must still be within eps of the block, with the oracle's rank.  Square and wide blocks,
    # through the SVD of the pivoted QR's R and through the full SVD of the block.
    rng = np.random.default_rng(17)
    eps = 1e-6
    for m, n in ((200, 200), (120, 230)):
        k = min(m, n)
        u, _ = np.linalg.qr(rng.standard_normal((m, k)))
        v, _ = np.linalg.qr(rng.standard_normal((n, k)))
        s = np.concatenate([1.0 + 1e-12 * np.arange(40), 1e-9 * rng.uniform(0.5, 1.0, k - 40)])
        a = (u * s) @ v.T
        ctx.set_opts(svd_no_prereduce=no_prereduce)
        try:
            mat = ctx.from_dense(a, [m], [n], eps_lr=eps)
        finally:
            ctx.set_opts(svd_no_prereduce=0)
        g = clr_pack.from_library(mat)
        assert g.kinds()[0, 0] == co.KIND_LR
        assert g.ranks()[0, 0] == co.compress_block(a, eps).rank == 40
        assert np.linalg.norm(g.block_dense(0, 0) - a) <= eps


def test_pinned_host_buffers_read_and_written_in_place(ctx):
    # page-locked host input and output go through the host-device link without staging; the
    # results equal those of pageable buffers bit for bit (ragged 32-wide tiles)
    import torch
    rng = np.random.default_rng(31)
    sizes = [70, 33, 130]
    n = sum(sizes)
    a = rng.standard_normal((n, n))
    ref = ctx.from_dense(a, sizes)                       # pageable: staged
    pin = torch.from_numpy(a).pin_memory()
    m = ctx.from_dense(pin, sizes)                       # pinned: read in place
    assert np.array_equal(m.to_dense(), ref.to_dense())
    out = torch.empty((n, n), dtype=torch.float64).pin_memory()
    m.to_dense(out)                                      # pinned: written in place
    assert np.array_equal(out.numpy(), a)
    # a strided (ld > n) pinned output
    wide = torch.zeros((n, n + 5), dtype=torch.float64).pin_memory()
    m.to_dense(wide[:, :n])
    assert np.array_equal(wide[:, :n].numpy(), a) and not wide[:, n:].numpy().any()
