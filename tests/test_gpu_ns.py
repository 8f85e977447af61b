"""GPU parity of the Newton–Schulz S^-1/2 driver (Section 4.2) against the oracle."""
import math

import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr.Context(0, precision="fp64", eps_lr=1e-8)


def test_ns_chain_matches_oracle_and_eigh(ctx):
    w = wl.chain_overlap(n=768, n_clusters=6, lo=96, hi=160)
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    gs = clr_pack.to_library(ctx, s_or)
    # with eps = 1e-8 the proxy floors near 2e-9; 1e-8 is reached one iteration after 2e-4.
    # The residual of the returned Z is held near the truncation level, which may lie above
    # this tolerance: then the proxy is met and the stated error is not
    from paper_1509_00309_gb300 import clr
    ctx.set_opts(ns_tol=1e-8, ns_max_iter=60, ns_alpha=0.0, eps_lr=1e-8)
    z, st, _ = ctx.sqrt_inv(gs, allow_noconv=True)
    alpha_or = co.alpha_estimate(s_or.to_dense())
    assert abs(st["alpha"] - alpha_or) <= 1e-12 * alpha_or
    ref = co.ns_clr(s_or, alpha_or, 1e-8, max_iter=60, tol=1e-8)
    assert st["proxy_met"] and ref.converged and st["iters"] == ref.iters
    assert st["converged"] == st["residual_met"] == (st["residual"] <= 1e-8)
    assert st["status"] == (clr.CLR_OK if st["converged"] else clr.CLR_ENOCONV)
    assert np.allclose(st["proxy"], ref.proxy, rtol=1e-6, atol=2e-8)
    zd = z.to_dense()
    exact = co.inv_sqrt_eigh(s_or.to_dense())
    assert np.linalg.norm(zd - exact) / np.linalg.norm(exact) < 1e-6
    assert np.linalg.norm(zd - ref.z.to_dense()) / np.linalg.norm(exact) < 1e-7
    assert st["residual"] < 1e-7
    # the library's residual runs through two FP64 CLR products truncated at
    # min(eps_lr, ns_tol / 100) = 1e-10, the oracle's is exact: they agree to that level
    assert abs(st["residual"] - co.residual(s_or.to_dense(), zd)) < 0.01 * st["residual"] + 1e-10


def test_ns_fixed_iterations_and_noconv(ctx):
    from paper_1509_00309_gb300 import clr
    w = wl.chain_overlap(n=384, n_clusters=3, lo=96, hi=160)
    gs = ctx.from_dense(w.a, w.row_sizes, eps_lr=1e-10, drop_norm=1e-12)
    ctx.set_opts(ns_tol=0.0, ns_max_iter=3, ns_alpha=0.05, eps_lr=1e-10)
    z, st, _ = ctx.sqrt_inv(gs)
    assert st["iters"] == 3 and len(st["proxy"]) == 4
    d = co.ns_dense(clr_pack.from_library(gs).to_dense(), 0.05, 3)
    assert np.linalg.norm(z.to_dense() - d.inv_sqrt) <= 1e-8 * np.linalg.norm(d.inv_sqrt)
    ctx.set_opts(ns_tol=1e-12, ns_max_iter=2, ns_alpha=0.0)
    with pytest.raises(clr.ClrError) as e:
        ctx.sqrt_inv(gs)
    assert e.value.status == clr.CLR_ENOCONV
    ctx.set_opts(ns_tol=1e-6, ns_max_iter=50)


def test_ns_fp64_meets_residual_and_split_floor(ctx):
    from paper_1509_00309_gb300 import clr
    # FP64 products reach the residual tolerance 1e-6 on the 1D chain (kappa ~ 8400).  Split
    # products (bf16x6, FP64 from ||X - I|| <= 1e-3 on) stop at the floor ~ u_split * kappa:
    # early absolute rounding errors are large relative to the small-eigenvalue components of
    # X and the coupled iteration carries them to the end.
    w = wl.chain_overlap()
    gs = ctx.from_dense(w.a, w.row_sizes, eps_lr=w.eps_lr, drop_norm=w.drop_norm)
    ctx.set_opts(precision="fp64", ns_tol=1e-6, ns_max_iter=60, ns_alpha=0.0, eps_lr=1e-8,
                 ns_fp64_tail=0)
    z_64, st_64, _ = ctx.sqrt_inv(gs)
    assert st_64["converged"] and st_64["residual_met"] and st_64["residual"] < 1e-6
    exact = co.inv_sqrt_eigh(w.a)
    assert np.linalg.norm(z_64.to_dense() - exact) / np.linalg.norm(exact) < 1e-6
    ctx.set_opts(precision="bf16x6", ns_fp64_tail=1, ns_ladder_switch=1e-3)
    z_lad, st_lad, _ = ctx.sqrt_inv(gs, allow_noconv=True)
    assert st_lad["proxy_met"]
    lam = np.linalg.eigvalsh(w.a)
    floor = 2.0 ** -24 * lam[-1] / lam[0]
    assert st_lad["residual"] < 30 * floor
    # the split floor is far above the tolerance: not reported as converged
    assert not st_lad["converged"] and not st_lad["residual_met"]
    assert st_lad["status"] == clr.CLR_ENOCONV
    ctx.set_opts(precision="fp64", ns_fp64_tail=0)


def test_ns_snapshot_rank_distribution_matches_oracle(ctx):
    # Section 5's distribution of block ranks of the 5th-iteration intermediates, on the 3D
    # lattice overlap construction scaled down to 16x8x2 sites x 4 points (N = 1024, eps
    # 1e-6), with dense-accumulated tiles re-tested for low rank so that the iterates keep
    # low-rank blocks
    w = wl.lattice_overlap(shape=(16, 8, 2), points_per_site=4, min_points=32, max_points=96)
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    alpha = co.alpha_estimate(s_or.to_dense())
    ref = co.ns_clr(s_or, alpha, w.eps_lr, max_iter=5, eps_sp=w.eps_sp, snapshot_iter=5,
                    recompress_dense=True)
    gs = clr_pack.to_library(ctx, s_or)
    ctx.set_opts(precision="fp64", eps_lr=w.eps_lr, eps_sp=w.eps_sp, ns_tol=0.0,
                 ns_max_iter=5, ns_alpha=alpha, ns_snapshot_iter=5, recompress_dense=1)
    ctx.sqrt_inv(gs)
    sizes = np.asarray(w.row_sizes)
    full = np.minimum.outer(sizes, sizes)
    nb = full.size
    for name in "XTYZ":
        g = ctx.ns_snapshot(name, gs)
        want = ref.snapshot[name]
        k, r, _, _ = g.get_blocks(pool=False)
        h = np.asarray(g.info()["rank_hist"])
        # the library's histogram is its own block table counted
        assert h[0] == np.sum(k == co.KIND_ZERO) and h[-1] == np.sum(k == co.KIND_DENSE), name
        assert h[1:-1].sum() == np.sum(k == co.KIND_LR), name
        # per block: rank (full for dense) within one of the oracle's, the tie rule at eps
        rk_g = np.where(k == co.KIND_DENSE, full, r)
        rk_o = np.where(want.kinds() == co.KIND_DENSE, full, want.ranks())
        close = (np.abs(rk_g - rk_o) <= 1) | ((k == co.KIND_DENSE) & (rk_o > full // 2 - 1)) | \
            ((want.kinds() == co.KIND_DENSE) & (rk_g > full // 2 - 1))
        assert close.all(), name
        assert np.mean(k == want.kinds()) >= 0.95, name
        # values: equal up to truncations at eps that land on different sides of a tie
        diff = np.linalg.norm(clr_pack.from_library(g).to_dense() - want.to_dense())
        assert diff <= 100 * w.eps_lr * math.sqrt(nb), name
        # distribution has the paper's shape: low ranks and full-rank blocks side by side
        if name in "YZ":
            assert h[-1] > 0 and h[1:-1].sum() > 0
    from paper_1509_00309_gb300 import clr
    with pytest.raises(clr.ClrError):
        ctx.ns_snapshot("X", gs)   # ownership was passed on: nothing left to take
    ctx.set_opts(ns_snapshot_iter=0, eps_sp=0.0, ns_alpha=0.0, eps_lr=1e-8, recompress_dense=0)
