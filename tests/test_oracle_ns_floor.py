"""Where the Newton–Schulz residual floors, and why (Section 4.2's iteration, Section 4.1's
truncation), pinned on the oracle alone.

In exact arithmetic Y_n = S Z_n, so X_n = alpha Y_n Z_n = alpha Z_n S Z_n: the loop's proxy
||X_n - I||_F / sqrt(N) IS the residual of the Z it returns.  Dense FP64 NS keeps that identity
to rounding.  With every product truncated at eps, Y_n drifts from S Z_n by the accumulated
truncation, and the residual of the returned Z settles at a floor proportional to eps while the
proxy keeps falling.  On the 3D lattice overlap matrix built at eps_lr = 1e-6 (4x4x4 sites x 16
points, N = 1024, kappa ~ 4e4), iterates truncated at 1e-6 leave the residual above the stated
tolerance 1e-6; truncated at 1e-8 they meet it."""
import numpy as np

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl


def test_dense_ns_residual_equals_its_proxy():
    w = wl.lattice_overlap(shape=(4, 4, 4))
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm).to_dense()
    alpha = co.alpha_estimate(s)
    r = co.ns_dense(s, alpha, 40, tol=1e-6)
    assert r.converged and r.proxy[-1] <= 1e-6
    res = co.residual(s, r.inv_sqrt)
    assert abs(res - r.proxy[-1]) <= 1e-3 * r.proxy[-1] + 1e-12


def test_truncated_ns_residual_floor_scales_with_eps():
    w = wl.lattice_overlap(shape=(4, 4, 4))
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    sd = s.to_dense()
    alpha = co.alpha_estimate(sd)
    res, proxy = {}, {}
    for eps in (1e-6, 1e-8):
        r = co.ns_clr(s, alpha, eps, 40, tol=1e-6, eps_sp=w.eps_sp, recompress_dense=True)
        assert r.converged                      # the proxy met the tolerance
        proxy[eps] = r.proxy[-1]
        res[eps] = co.residual(sd, r.z.to_dense())
    # truncation at the build threshold: the proxy is met, the residual is not
    assert proxy[1e-6] <= 1e-6 < res[1e-6]
    assert res[1e-6] > 3 * proxy[1e-6]
    # truncation at 1e-8: the stated error is met
    assert res[1e-8] <= 1e-6
    # the floor follows eps (a hundredfold smaller eps, a far smaller floor)
    assert res[1e-6] / res[1e-8] > 20
    assert np.isfinite(res[1e-8])
