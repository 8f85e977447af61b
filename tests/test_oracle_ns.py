"""Pins of the oracle's Newton–Schulz S^-1/2 iteration (Section 4.2)."""
import json
import math
import os

import numpy as np

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl


def scalar_map(x):
    """On an eigenvalue x of alpha*S the iteration acts as x -> x f(x)^2 with
    f(x) = (15 - 10 x + 3 x^2) / 8 (X = x, T = f(x), Z and Y pick up one factor each)."""
    f = (15.0 - 10.0 * x + 3.0 * x * x) / 8.0
    return x * f * f


def test_polynomial_coefficients_match_paper(repo_root):
    facts = json.load(open(os.path.join(repo_root, "tests", "golden", "paper_facts.json")))
    p = facts["ns_polynomial"]
    x = np.diag([0.3, 0.7, 1.0])
    t = co.ns_poly(x)
    want = (p["c0"] * np.eye(3) + p["c1"] * x + p["c2"] * x @ x) / p["den"]
    assert np.allclose(t, want, rtol=0, atol=1e-15)
    # fixed point: f(1) = 1
    assert (p["c0"] + p["c1"] + p["c2"]) / p["den"] == 1.0


def test_scalar_map_cubic_convergence():
    # x = 1 - e  ->  1 - (5/8) e^3 + O(e^4)
    for e in [1e-2, 3e-3, 1e-3]:
        e_next = 1.0 - scalar_map(1.0 - e)
        assert abs(e_next / e ** 3 - 5.0 / 8.0) < 4 * e
    x = 1e-4
    for _ in range(40):
        x = scalar_map(x)
    assert abs(x - 1.0) < 1e-15


def test_diagonal_matrix_reduces_to_scalar_map():
    lam = np.array([0.01, 0.3, 1.0, 4.0, 9.0])
    s = np.diag(lam)
    alpha = 1.0 / 9.5
    res = co.ns_dense(s, alpha, max_iter=6, tol=0.0)
    z = np.ones_like(lam)
    x = alpha * lam
    for _ in range(6):
        f = (15.0 - 10.0 * x + 3.0 * x * x) / 8.0
        z = z * f
        x = x * f * f
    assert np.allclose(np.diag(res.inv_sqrt), math.sqrt(alpha) * z, rtol=1e-14, atol=0)
    conv = co.ns_dense(s, alpha, max_iter=60, tol=1e-14)
    assert conv.converged
    assert np.allclose(np.diag(conv.inv_sqrt), lam ** -0.5, rtol=1e-12)


def test_alpha_estimate_on_known_spectrum():
    lam = np.array([1.0, 2.0, 5.0, 7.0])
    a = co.alpha_estimate(np.diag(lam), steps=200)
    assert abs(a - 1.0 / (1.01 * 7.0)) < 1e-12


def test_dense_ns_matches_eigh_and_invariants():
    w = wl.chain_overlap(n=256, n_clusters=4, lo=48, hi=80)
    s = w.a
    alpha = co.alpha_estimate(s)
    lam = np.linalg.eigvalsh(s)
    assert alpha * lam.max() <= 1.0 and alpha * lam.min() > 0
    res = co.ns_dense(s, alpha, max_iter=60, tol=1e-12, keep_tape=True)
    assert res.converged
    ref = co.inv_sqrt_eigh(s)
    kappa = lam.max() / lam.min()
    assert np.linalg.norm(res.inv_sqrt - ref) / np.linalg.norm(ref) < 1e-15 * kappa * 10
    assert co.residual(s, res.inv_sqrt) < 1e-11
    # Y_n and Z_n are polynomials in S: they commute and Y_n = S Z_n
    for y, z in res.tape[::4]:
        assert np.linalg.norm(y @ z - z @ y) <= 1e-10 * np.linalg.norm(y) * np.linalg.norm(z)
        assert np.linalg.norm(y - s @ z) <= 1e-10 * np.linalg.norm(y)


def test_clr_ns_exact_limit_equals_dense():
    # eps -> 0: CLR arithmetic is exact (Section 4.1), so CLR NS equals dense NS
    w = wl.chain_overlap(n=192, n_clusters=3, lo=48, hi=80)
    s = co.build(w.a, w.row_sizes, w.col_sizes, 0.0)
    alpha = co.alpha_estimate(w.a)
    d = co.ns_dense(w.a, alpha, max_iter=5)
    c = co.ns_clr(s, alpha, 0.0, max_iter=5)
    assert np.linalg.norm(c.z.to_dense() - d.inv_sqrt) <= 1e-12 * np.linalg.norm(d.inv_sqrt)
    assert np.allclose(c.proxy, d.proxy, rtol=1e-10, atol=1e-14)


def test_clr_ns_truncated_converges():
    w = wl.lattice_overlap(shape=(2, 2, 2), points_per_site=16, min_points=32, max_points=64,
                           eps_lr=1e-7)
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    alpha = co.alpha_estimate(s.to_dense())
    c = co.ns_clr(s, alpha, w.eps_lr, max_iter=40, tol=1e-6)
    assert c.converged
    ref = co.inv_sqrt_eigh(w.a)
    assert co.residual(w.a, c.z.to_dense()) < 1e-5
    assert np.linalg.norm(c.z.to_dense() - ref) / np.linalg.norm(ref) < 1e-4


def test_clr_ns_snapshot_on_diagonal_follows_scalar_recurrence():
    # S diagonal in three dense diagonal blocks, eps = 0: the k-th iteration's X, T, Y, Z are
    # diagonal with the scalar recurrence x = alpha y z, t = f(x), z <- z t, y <- t y
    lam = np.array([0.02, 0.5, 1.0, 2.0, 3.5, 5.0, 6.0, 8.0, 9.0])
    sizes = [2, 4, 3]
    s = co.build(np.diag(lam), sizes, sizes, 0.0)
    alpha = 1.0 / 9.5
    k = 3
    res = co.ns_clr(s, alpha, 0.0, max_iter=6, snapshot_iter=k)
    y, z = lam.copy(), np.ones_like(lam)
    for _ in range(k):
        x = alpha * y * z
        t = (15.0 - 10.0 * x + 3.0 * x * x) / 8.0
        z, y = z * t, t * y
    for name, want in (("X", x), ("T", t), ("Y", y), ("Z", z)):
        got = res.snapshot[name].to_dense()
        assert np.allclose(got, np.diag(want), rtol=1e-14, atol=1e-15), name
    assert co.ns_clr(s, alpha, 0.0, max_iter=2, snapshot_iter=k).snapshot == {}


def test_rank_histogram_counts_kinds_and_ranks():
    rng = np.random.default_rng(4)
    sizes = [6, 5, 7]

    def lr(m, n, r):
        return (co.KIND_LR, (rng.standard_normal((m, r)), rng.standard_normal((n, r))))

    spec = [[(co.KIND_DENSE, rng.standard_normal((6, 6))), lr(6, 5, 2), (co.KIND_ZERO, None)],
            [lr(5, 6, 1), (co.KIND_DENSE, rng.standard_normal((5, 5))), lr(5, 7, 2)],
            [(co.KIND_ZERO, None), lr(7, 5, 3), (co.KIND_ZERO, None)]]
    h = co.rank_histogram(co.from_blocks(sizes, sizes, spec))
    want = np.zeros(130, dtype=np.int64)
    want[0], want[1], want[2], want[3], want[-1] = 3, 1, 2, 1, 2
    assert np.array_equal(h, want)
