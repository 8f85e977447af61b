"""GPU parity on the Coulomb-like matrix (no block sparsity, only block-rank sparsity) against the
oracle: the CLR product V V and the Newton–Schulz iteration for V^-1/2."""
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
    return clr.Context(0, precision="fp64", eps_lr=1e-6)


@pytest.fixture(scope="module")
def coulomb():
    w = wl.lattice_coulomb(shape=(4, 4, 2), min_points=32, max_points=96)
    return w, co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_coulomb_product_matches_oracle(ctx, coulomb, prec):
    w, v_or = coulomb
    ctx.set_opts(precision=prec, eps_lr=w.eps_lr, eps_sp=w.eps_sp)
    gv = clr_pack.to_library(ctx, v_or)
    gc = ctx.zeros(w.row_sizes)
    ctx.multiply_into(gv, gv, gc)
    want = co.multiply(v_or, v_or, w.eps_lr, w.eps_sp)
    got = clr_pack.from_library(gc)
    vd = v_or.to_dense()
    assert np.linalg.norm(got.to_dense() - want.to_dense()) <= \
        co.product_tolerance(vd, vd, w.eps_lr)
    # kinds agree except where a rank sits at the dense threshold (ranks within one)
    full = np.minimum.outer(np.asarray(w.row_sizes), np.asarray(w.row_sizes))
    rk_g = np.where(got.kinds() == co.KIND_DENSE, full, got.ranks())
    rk_o = np.where(want.kinds() == co.KIND_DENSE, full, want.ranks())
    assert np.all((np.abs(rk_g - rk_o) <= 1) | ((rk_g > full // 2 - 1) & (rk_o > full // 2 - 1)))


def test_coulomb_ns_matches_oracle(ctx, coulomb):
    w, v_or = coulomb
    alpha = co.alpha_estimate(v_or.to_dense())
    ctx.set_opts(precision="fp64", eps_lr=w.eps_lr, eps_sp=w.eps_sp, ns_tol=0.0,
                 ns_max_iter=8, ns_alpha=alpha)
    gv = clr_pack.to_library(ctx, v_or)
    z, st, _ = ctx.sqrt_inv(gv)
    ref = co.ns_clr(v_or, alpha, w.eps_lr, max_iter=8, eps_sp=w.eps_sp)
    assert st["iters"] == ref.iters == 8
    assert np.allclose(st["proxy"], ref.proxy, rtol=1e-6, atol=1e-7)
    zd, zo = z.to_dense(), ref.z.to_dense()
    assert np.linalg.norm(zd - zo) <= 1e-5 * np.linalg.norm(zo)
    ctx.set_opts(ns_tol=1e-6, ns_max_iter=60, ns_alpha=0.0, eps_sp=0.0)
