"""Pins of the oracle's gradient of L = trace(W S^-1/2) and of the NS adjoint."""
import math

import numpy as np

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl


def _spd(rng, n, cond=50.0):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (q * lam) @ q.T


def loss_exact(s, w):
    return float(np.trace(w @ co.inv_sqrt_eigh(0.5 * (s + s.T)))) if np.allclose(s, s.T) \
        else float(np.trace(w @ _inv_sqrt_general(s)))


def _inv_sqrt_general(s):
    # principal inverse square root of a (possibly nonsymmetric) matrix with positive
    # eigenvalues, through its eigendecomposition
    lam, v = np.linalg.eig(s)
    return np.real((v * lam ** -0.5) @ np.linalg.inv(v))


def test_diagonal_closed_form():
    lam = np.array([0.5, 1.0, 3.0, 8.0])
    wd = np.array([1.0, -2.0, 0.5, 4.0])
    g = co.grad_trace_inv_sqrt(np.diag(lam), np.diag(wd))
    assert np.allclose(np.diag(g), -0.5 * wd * lam ** -1.5, rtol=1e-14)
    assert np.allclose(g - np.diag(np.diag(g)), 0.0, atol=1e-15)


def test_daleckii_krein_vs_central_differences():
    rng = np.random.default_rng(2)
    n = 6
    s = _spd(rng, n)
    w = wl.symmetric_normal(rng, n)
    g = co.grad_trace_inv_sqrt(s, w)
    h = 1e-6
    for i, j in [(0, 0), (1, 3), (4, 2), (5, 5), (2, 0)]:
        e = np.zeros((n, n))
        e[i, j] = h
        fd = (loss_exact(s + e, w) - loss_exact(s - e, w)) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-7 * max(1.0, abs(g[i, j]))


def test_ns_adjoint_vs_differences_of_the_iteration():
    # the reverse sweep differentiates exactly the finite NS map (alpha fixed)
    rng = np.random.default_rng(7)
    n = 5
    s = _spd(rng, n, cond=20.0)
    w = wl.symmetric_normal(rng, n)
    alpha = co.alpha_estimate(s)
    iters = 4

    def f(mat):
        return float(np.trace(w @ co.ns_dense(mat, alpha, iters).inv_sqrt))

    g = co.ns_adjoint_dense(s, w, alpha, iters)
    h = 1e-6
    for i, j in [(0, 0), (1, 2), (3, 1), (4, 4)]:
        e = np.zeros((n, n))
        e[i, j] = h
        fd = (f(s + e) - f(s - e)) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-7 * max(1.0, abs(g[i, j]))


def test_ns_adjoint_converges_to_daleckii_krein():
    rng = np.random.default_rng(11)
    n = 8
    s = _spd(rng, n, cond=100.0)
    w = wl.symmetric_normal(rng, n)
    alpha = co.alpha_estimate(s)
    g_ns = co.ns_adjoint_dense(s, w, alpha, 30)
    g_dk = co.grad_trace_inv_sqrt(s, w)
    assert np.linalg.norm(g_ns - g_dk) <= 1e-10 * np.linalg.norm(g_dk)
