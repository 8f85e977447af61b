"""Pins of the oracle's block compression (Section 4.1) against closed forms."""
import math

import numpy as np
import pytest

from oracle import clr_oracle as co


def _orth(rng, n):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return q


def _with_singular_values(rng, m, n, s):
    u, v = _orth(rng, m)[:, :len(s)], _orth(rng, n)[:, :len(s)]
    return (u * np.asarray(s)) @ v.T


def test_truncation_rank_hand_values():
    s = np.array([3.0, 2.0, 1.0])
    # tails: r=0 -> sqrt(14), r=1 -> sqrt(5), r=2 -> 1, r=3 -> 0
    assert co.truncation_rank(s, 1.0) == 2
    assert co.truncation_rank(s, 0.999) == 3
    assert co.truncation_rank(s, math.sqrt(5.0) + 1e-12) == 1
    assert co.truncation_rank(s, math.sqrt(14.0) + 1e-12) == 0
    assert co.truncation_rank(s, 0.0) == 3
    assert co.truncation_rank(np.array([1.0, 0.0, 0.0]), 0.0) == 1


def test_dense_rank_limit():
    assert co.dense_rank_limit(7, 9) == 3
    assert co.dense_rank_limit(8, 8) == 4
    assert co.dense_rank_limit(1, 5) == 0


def test_compress_2x2_closed_form():
    # For a 2x2 block, s1^2 + s2^2 = ||M||_F^2 and s1 s2 = |det M| give both singular values
    # without an SVD; a rank-1 block keeps low-rank form (1 <= floor(2/2)), rank 2 is dense.
    rng = np.random.default_rng(1)
    for _ in range(20):
        m = rng.standard_normal((2, 2))
        f2 = float(np.sum(m * m))
        det = abs(m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0])
        s1 = math.sqrt(0.5 * (f2 + math.sqrt(f2 * f2 - 4 * det * det)))
        s2 = det / s1
        b = co.compress_block(m, eps=s2 * 1.001)
        assert b.kind == co.KIND_LR and b.rank == 1
        assert abs(np.linalg.norm(m - b.x @ b.w.T) - s2) < 1e-12 * s1
        assert co.compress_block(m, eps=s2 * 0.999).kind == co.KIND_DENSE
        assert co.compress_block(m, eps=math.sqrt(f2) * 1.001).kind == co.KIND_ZERO


@pytest.mark.parametrize("m,n", [(9, 7), (12, 12), (5, 11)])
def test_compress_known_spectrum(m, n):
    rng = np.random.default_rng(m * 100 + n)
    s = np.array([4.0, 1.0, 0.25, 1e-3, 1e-5, 1e-9])[:min(m, n)]
    mat = _with_singular_values(rng, m, n, s)
    for eps, want_rank in [(1e-10, 6), (2e-5, 4), (1.1e-3, 3), (0.3, 2), (1.1, 1)]:
        b = co.compress_block(mat, eps)
        tail = math.sqrt(float(np.sum(s[want_rank:] ** 2)))
        if want_rank > co.dense_rank_limit(m, n):
            assert b.kind == co.KIND_DENSE
            continue
        assert b.kind == co.KIND_LR and b.rank == want_rank
        err = np.linalg.norm(mat - b.x @ b.w.T)
        assert abs(err - tail) < 1e-12 * 4.0
        # singular values sit on the left factor: W has orthonormal columns
        assert np.allclose(b.w.T @ b.w, np.eye(want_rank), atol=1e-12)
        assert np.allclose(np.linalg.norm(b.x, axis=0), s[:want_rank], rtol=1e-12)


def test_drop_norm_and_zero_block():
    m = np.full((3, 4), 1e-13)
    assert co.compress_block(m, eps=0.0, drop_norm=1e-12).kind == co.KIND_ZERO
    assert co.compress_block(m, eps=0.0, drop_norm=1e-13).kind != co.KIND_ZERO
    assert co.compress_block(np.zeros((4, 4)), eps=0.0).kind == co.KIND_ZERO


def test_build_and_reconstruct_block_errors():
    rng = np.random.default_rng(5)
    sizes = [3, 5, 4]
    n = sum(sizes)
    pts = np.sort(rng.uniform(0, 6, n))
    a = np.exp(-(pts[:, None] - pts[None, :]) ** 2)
    c = co.build(a, sizes, sizes, eps=1e-6)
    for i in range(3):
        for j in range(3):
            blk = a[c.row_off[i]:c.row_off[i + 1], c.col_off[j]:c.col_off[j + 1]]
            assert np.linalg.norm(blk - c.block_dense(i, j)) <= 1e-6 * (1 + 1e-9)
    assert np.linalg.norm(c.to_dense() - a) <= 3e-6


def test_rrqr_build_error_rank_and_exact_low_rank():
    rng = np.random.default_rng(12)
    eps = 1e-8
    # exact rank 6 (generic): the pivoted QR's trailing block vanishes after 6 steps
    a = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 25))
    b = co.compress_block_rrqr(a, eps)
    assert b.kind == co.KIND_LR and b.rank == 6
    assert np.linalg.norm(b.x @ b.w.T - a) <= 1e-12 * np.linalg.norm(a)
    assert np.allclose(b.x.T @ b.x, np.eye(6), atol=1e-13)         # X = Q_r orthonormal
    # graded spectrum: error <= eps and rank >= the SVD's minimal rank
    u, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    v, _ = np.linalg.qr(rng.standard_normal((32, 32)))
    s = 10.0 ** (-0.5 * np.arange(32))
    g = (u[:, :32] * s) @ v.T
    for e in (1e-4, 1e-6):
        br = co.compress_block_rrqr(g, e)
        bs = co.compress_block(g, e)
        assert br.kind == co.KIND_LR
        assert np.linalg.norm(br.x @ br.w.T - g) <= e * (1 + 1e-9)
        assert br.rank >= bs.rank
    # dense and zero rules as for the SVD build
    assert co.compress_block_rrqr(rng.standard_normal((8, 8)), eps).kind == co.KIND_DENSE
    assert co.compress_block_rrqr(np.full((4, 5), 1e-12), 1e-8).kind == co.KIND_ZERO


def test_rrqr_matches_lapack_pivoted_qr_rank():
    # the step-by-step pivoted QR selects the same columns as LAPACK's xGEQP3 on generic input,
    # so the truncation ranks agree
    from scipy.linalg import qr
    rng = np.random.default_rng(13)
    for trial in range(5):
        m, n = rng.integers(10, 40, size=2)
        k = min(m, n)
        s = 10.0 ** (-rng.uniform(0.2, 0.8) * np.arange(k))
        u, _ = np.linalg.qr(rng.standard_normal((m, k)))
        v, _ = np.linalg.qr(rng.standard_normal((n, k)))
        g = (u * s) @ v.T
        _, r_l, piv = qr(g, pivoting=True, mode="economic")
        tails = [np.linalg.norm(r_l[j:, j:]) for j in range(k)] + [0.0]
        want = next(j for j in range(k + 1) if tails[j] <= 1e-7)
        b = co.compress_block_rrqr(g, 1e-7)
        got = b.rank if b.kind == co.KIND_LR else (0 if b.kind == co.KIND_ZERO else -1)
        if b.kind == co.KIND_DENSE:
            assert want > co.dense_rank_limit(m, n)
        else:
            assert got == want
