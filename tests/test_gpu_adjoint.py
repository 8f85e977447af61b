"""GPU parity of the hand-written adjoints: of the Newton–Schulz iteration (loss
trace(W S^-1/2)) against the oracle's reverse sweep, the Daleckii–Krein eigen-gradient and
finite differences; and of the CLR product C = A B against the oracle's products of the
transposed operands and finite differences."""
import math

import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clr():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr


def test_adjoint_fixed_iterations_matches_oracle_reverse_sweep(clr):
    w = wl.chain_overlap(n=384, n_clusters=3, lo=96, hi=160)
    s = w.a
    wmat = wl.symmetric_normal(3, s.shape[0])
    alpha = co.alpha_estimate(s)
    ctx = clr.Context(0, precision="fp64", eps_lr=1e-13, ns_tol=0.0, ns_max_iter=6,
                      ns_alpha=alpha)
    sm = ctx.from_dense(s, w.row_sizes, eps_lr=1e-13)
    z, st, tape = ctx.sqrt_inv(sm, keep_tape=True)
    assert st["iters"] == 6
    zb = ctx.from_dense(np.ascontiguousarray(wmat.T), w.row_sizes, eps_lr=0.0)
    g = ctx.sqrt_inv_backward(tape, zb).to_dense()
    want = co.ns_adjoint_dense(s, wmat, alpha, 6)
    assert np.linalg.norm(g - want) <= 1e-9 * np.linalg.norm(want)


def test_adjoint_converged_matches_daleckii_krein(clr):
    # the 3D lattice construction at N = 512 (4 x 4 x 2 sites x 16 points)
    w = wl.adjoint_lattice(n_sites_shape=(4, 4, 2), min_points=32, max_points=128)
    s, wmat = w.a, w.extra["w"]
    ctx = clr.Context(0, precision="fp64", eps_lr=1e-10, ns_tol=1e-11, ns_max_iter=80)
    sm = ctx.from_dense(s, w.row_sizes, eps_lr=1e-10)
    z, st, tape = ctx.sqrt_inv(sm, keep_tape=True, allow_noconv=True)
    assert st["proxy_met"] and st["residual"] < 1e-8
    zb = ctx.from_dense(np.ascontiguousarray(wmat.T), w.row_sizes, eps_lr=0.0)
    g = ctx.sqrt_inv_backward(tape, zb).to_dense()
    want = co.grad_trace_inv_sqrt(s, wmat)
    assert np.linalg.norm(g - want) <= 1e-5 * np.linalg.norm(want)


def test_autograd_function_vs_finite_differences(clr):
    import torch
    from paper_1509_00309_gb300.autograd import sqrt_inv
    w = wl.chain_overlap(n=256, n_clusters=2, lo=96, hi=160)
    ctx = clr.Context(0, precision="fp64", eps_lr=1e-12, ns_tol=1e-12, ns_max_iter=80)
    s = torch.from_numpy(w.a).cuda().requires_grad_(True)
    wm = torch.from_numpy(wl.symmetric_normal(5, 256)).cuda()
    loss = torch.trace(wm @ sqrt_inv(s, ctx, w.row_sizes, eps_lr=1e-12))
    loss.backward()
    g = s.grad.cpu().numpy()

    def f(mat):
        z = sqrt_inv(torch.from_numpy(mat).cuda(), ctx, w.row_sizes, eps_lr=1e-12)
        return float(torch.trace(wm @ z))

    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(3):
        i, j = rng.integers(0, 256, 2)
        e = np.zeros_like(w.a)
        e[i, j] = h
        fd = (f(w.a + e) - f(w.a - e)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-4 * max(1.0, abs(g[i, j])), (i, j, fd, g[i, j])


@pytest.mark.parametrize("eps", [1e-8, 0.0])
def test_adjoint_lattice_finite_differences_32_entries(clr, eps):
    # the differentiation configuration scaled to N = 512 (4x4x2 sites x 16 points): 20
    # Newton-Schulz iterations at eps_lr, gradient of trace(W S^-1/2) by the adjoint against
    # central differences (h = 1e-6) on 32 seeded entries.  With eps = 1e-8 the truncation noise
    # in L (~1e-8) limits the difference quotient to ~1e-2 absolute: tolerance
    # max(1e-2 |g|, 1e-3); exact arithmetic (eps = 0, dense tiles): 1e-6 relative.
    w = wl.adjoint_lattice(n_sites_shape=(4, 4, 2), min_points=32, max_points=128)
    s, wmat = w.a, w.extra["w"]
    alpha = co.alpha_estimate(s)
    ctx = clr.Context(0, precision="fp64", eps_lr=eps, ns_tol=0.0, ns_max_iter=20,
                      ns_alpha=alpha)

    def loss(mat, tape=False):
        sm = ctx.from_dense(mat, w.row_sizes, eps_lr=eps)
        z, st, tp = ctx.sqrt_inv(sm, keep_tape=tape)
        assert st["iters"] == 20
        return float(np.sum(wmat * z.to_dense().T)), z, tp   # trace(W Z)

    _, z, tape = loss(s, tape=True)
    zb = ctx.from_dense(np.ascontiguousarray(wmat.T), w.row_sizes, eps_lr=0.0)
    g = ctx.sqrt_inv_backward(tape, zb).to_dense()
    h = 1e-6
    rng = np.random.default_rng(44)

    def central(i, j, step):
        e = np.zeros_like(s)
        e[i, j] = step
        return (loss(s + e)[0] - loss(s - e)[0]) / (2 * step)

    for i, j in rng.integers(0, w.n, size=(32, 2)):
        fd = central(i, j, h)
        if eps > 0:
            tol = max(1e-2 * abs(g[i, j]), 1e-3)
        else:
            # exact arithmetic: 1e-6 relative plus the difference quotient's own O(h^2) error,
            # estimated by Richardson from the step 2h (|fd(h) - fd(2h)| / 3); the small
            # eigenvalues (1e-2) make the third derivative large enough for that term to matter
            tol = 1e-6 * max(1.0, abs(g[i, j])) + abs(fd - central(i, j, 2 * h)) / 3 * 1.5
        assert abs(fd - g[i, j]) <= tol, (i, j, fd, g[i, j])


def test_multiply_backward_matches_oracle(clr):
    # the adjoint of C = A B (Section 4.1's block product reversed, truncation as the identity):
    # Abar = Cbar B^T and Bbar = A^T Cbar, each the oracle's CLR product of the transposed
    # operand, on rectangular clusterings with every block kind
    rng = np.random.default_rng(404)
    rs, ks, cs = [30, 45, 20], [25, 40], [33, 17, 28, 9]
    eps = 1e-10
    a = co.from_blocks(rs, ks, wl.random_blocks_spec(rng, rs, ks, max_rank=4))
    b = co.from_blocks(ks, cs, wl.random_blocks_spec(rng, ks, cs, max_rank=4))
    cb = co.from_blocks(rs, cs, wl.random_blocks_spec(rng, rs, cs, max_rank=4))
    ctx = clr.Context(0, precision="fp64", eps_lr=eps)
    ga, gb, gcb = (clr_pack.to_library(ctx, m) for m in (a, b, cb))
    abar, bbar = ctx.multiply_backward(ga, gb, gcb)
    want_a = co.multiply(cb, co.transpose(b), eps)
    want_b = co.multiply(co.transpose(a), cb, eps)
    for got, want, l, r in ((abar, want_a, cb, co.transpose(b)),
                            (bbar, want_b, co.transpose(a), cb)):
        g = clr_pack.from_library(got)
        assert g.to_dense().shape == want.to_dense().shape
        err = np.linalg.norm(g.to_dense() - want.to_dense())
        assert err <= co.product_tolerance(l.to_dense(), r.to_dense(), eps)
        ex = l.to_dense() @ r.to_dense()
        assert np.linalg.norm(g.to_dense() - ex) <= 2 * eps * math.sqrt(g.kinds().size) + \
            1e-13 * np.linalg.norm(ex)
    # one adjoint alone
    only_b = ctx.multiply_backward(ga, gb, gcb, need_a=False)
    assert only_b[0] is None and np.array_equal(only_b[1].to_dense(), bbar.to_dense())
    with pytest.raises(clr.ClrError) as e:
        ctx.multiply_backward(ga, gb, ga)   # Cbar with the wrong clusters
    assert e.value.status == clr.CLR_EINVAL


def test_autograd_multiply_gradients_and_finite_differences(clr):
    # loss = sum(W o (A B)) through the autograd Function: dL/dA = W B^T, dL/dB = A^T W (exact
    # products of the dense operands within the truncation eps), and central differences on 8
    # entries of each operand (the loss is bilinear: the quotient is exact up to rounding)
    import torch
    from paper_1509_00309_gb300.autograd import multiply
    w = wl.chain_overlap(n=384, n_clusters=3, lo=96, hi=160)
    eps = 1e-12
    ctx = clr.Context(0, precision="fp64", eps_lr=eps)
    a = torch.from_numpy(w.a).cuda().requires_grad_(True)
    bnp = w.a @ np.diag(np.linspace(0.5, 1.5, w.n))
    b = torch.from_numpy(bnp).cuda().requires_grad_(True)
    wm = torch.from_numpy(np.random.default_rng(9).standard_normal((w.n, w.n))).cuda()
    loss = torch.sum(wm * multiply(a, b, ctx, w.row_sizes, eps_lr=eps))
    loss.backward()
    ga, gb = a.grad.cpu().numpy(), b.grad.cpu().numpy()
    wn = wm.cpu().numpy()
    assert np.linalg.norm(ga - wn @ bnp.T) <= 1e-9 * np.linalg.norm(wn @ bnp.T)
    assert np.linalg.norm(gb - w.a.T @ wn) <= 1e-9 * np.linalg.norm(w.a.T @ wn)

    def f(am, bm):
        c = multiply(torch.from_numpy(am).cuda(), torch.from_numpy(bm).cuda(), ctx, w.row_sizes,
                     eps_lr=eps)
        return float(torch.sum(wm * c))

    h = 1e-4
    rng = np.random.default_rng(2)
    for _ in range(8):
        i, j = rng.integers(0, w.n, 2)
        e = np.zeros_like(w.a)
        e[i, j] = h
        fda = (f(w.a + e, bnp) - f(w.a - e, bnp)) / (2 * h)
        fdb = (f(w.a, bnp + e) - f(w.a, bnp - e)) / (2 * h)
        assert abs(fda - ga[i, j]) <= 1e-6 * max(1.0, abs(ga[i, j])), (i, j, fda, ga[i, j])
        assert abs(fdb - gb[i, j]) <= 1e-6 * max(1.0, abs(gb[i, j])), (i, j, fdb, gb[i, j])
