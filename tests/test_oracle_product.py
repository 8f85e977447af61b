"""Pins of the oracle's CLR product (Section 4.1) against dense GEMM, brute force and
hand-enumerated work lists."""
import itertools
import math

import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl


def brute_matmul(a, b):
    """Triple loop in pure Python: the definition of the matrix product."""
    m, k = a.shape
    _, n = b.shape
    out = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            s = 0.0
            for t in range(k):
                s += float(a[i, t]) * float(b[t, j])
            out[i, j] = s
    return out


def test_full_rank_equals_dense_gemm():
    # eps -> 0: every block is dense and the CLR product is ordinary matrix multiplication
    # (Section 4.3).
    rng = np.random.default_rng(0)
    sizes = [7, 13, 5, 11]
    n = sum(sizes)
    a, b = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    ca, cb = co.build(a, sizes, sizes, 0.0), co.build(b, sizes, sizes, 0.0)
    assert set(ca.kinds().ravel()) == {co.KIND_DENSE}
    c = co.multiply(ca, cb, 0.0)
    ref = a @ b
    assert np.linalg.norm(c.to_dense() - ref) <= 1e-14 * np.linalg.norm(ref) * math.sqrt(n)
    tl = co.triple_list(ca, cb)
    assert len(tl.triples) == 4 ** 3 and set(tl.triples[:, 3]) == {co.T_DD}


@pytest.mark.parametrize("seed", range(6))
def test_tiny_brute_force_all_kinds(seed):
    rng = np.random.default_rng(100 + seed)
    nb = int(rng.integers(2, 4))
    sizes = [int(s) for s in rng.integers(1, 10, size=nb)]
    spec_a = wl.random_blocks_spec(rng, sizes, sizes)
    spec_b = wl.random_blocks_spec(rng, sizes, sizes)
    a, b = co.from_blocks(sizes, sizes, spec_a), co.from_blocks(sizes, sizes, spec_b)
    da, db = a.to_dense(), b.to_dense()
    ref = brute_matmul(da, db)
    eps = 1e-9
    c = co.multiply(a, b, eps)
    tl = co.triple_list(a, b)
    for i in range(nb):
        for j in range(nb):
            r0, r1 = c.row_off[i], c.row_off[i + 1]
            c0, c1 = c.col_off[j], c.col_off[j + 1]
            got, want = c.block_dense(i, j), ref[r0:r1, c0:c1]
            scale = max(1.0, float(np.abs(want).sum()))
            if tl.tile_mode[i, j] == co.MODE_DENSE:
                assert c.get(i, j).kind == co.KIND_DENSE
                assert np.abs(got - want).max() <= 1e-13 * scale
            else:
                # truncation error of at most eps (plus rounding)
                assert np.linalg.norm(got - want) <= eps + 1e-13 * scale


def test_low_rank_side_choice():
    assert co.lr_output_rank(3, 5) == (3, 1)
    assert co.lr_output_rank(5, 3) == (3, 0)
    assert co.lr_output_rank(4, 4) == (4, 0)


def test_triple_flops_hand_values():
    m, k, n = 10, 20, 30
    assert co.triple_flops(co.T_DD, m, k, n, 0, 0) == 2 * 10 * 20 * 30
    assert co.triple_flops(co.T_DL, m, k, n, 0, 4) == 2 * 10 * 20 * 4
    assert co.triple_flops(co.T_LD, m, k, n, 3, 0) == 2 * 20 * 30 * 3
    # LL, r_A = 3 < r_B = 4: Z (3x4) then W_B Z^T (n x 3)
    assert co.triple_flops(co.T_LL, m, k, n, 3, 4) == 2 * 20 * 3 * 4 + 2 * 30 * 3 * 4
    # LL, r_A = 4 >= r_B = 2: Z (4x2) then X_A Z (m x 2)
    assert co.triple_flops(co.T_LL, m, k, n, 4, 2) == 2 * 20 * 4 * 2 + 2 * 10 * 4 * 2


def test_triple_list_hand_enumerated():
    # A: dense diagonal, LR (0,1); B: dense diagonal, LR (1,0), zero elsewhere.
    sizes = [4, 6]
    rng = np.random.default_rng(3)
    d0, d1 = rng.standard_normal((4, 4)), rng.standard_normal((6, 6))
    xa, wa = rng.standard_normal((4, 2)), rng.standard_normal((6, 2))
    xb, wb = rng.standard_normal((6, 1)), rng.standard_normal((4, 1))
    a = co.from_blocks(sizes, sizes, [[(1, d0), (2, (xa, wa))], [(0, None), (1, d1)]])
    b = co.from_blocks(sizes, sizes, [[(1, d0), (0, None)], [(2, (xb, wb)), (1, d1)]])
    tl = co.triple_list(a, b)
    want = [(0, 0, 0, co.T_DD), (0, 0, 1, co.T_LL), (0, 1, 1, co.T_LD),
            (1, 0, 1, co.T_DL), (1, 1, 1, co.T_DD)]
    assert [tuple(int(v) for v in t) for t in tl.triples] == want
    assert tl.tile_mode.tolist() == [[co.MODE_DENSE, co.MODE_LR], [co.MODE_LR, co.MODE_DENSE]]
    assert tl.tile_rank_sum.tolist() == [[1, 2], [1, 0]]
    assert tl.flops.tolist() == [2 * 4 * 4 * 4, 2 * 6 * 2 * 1 + 2 * 4 * 2 * 1,
                                 2 * 6 * 6 * 2, 2 * 6 * 6 * 1, 2 * 6 * 6 * 6]


def test_screening_drops_small_tiles():
    sizes = [2, 2]
    a = co.from_blocks(sizes, sizes, [[(1, np.eye(2)), (1, 1e-9 * np.ones((2, 2)))],
                                      [(0, None), (1, np.eye(2))]])
    # C_01 estimate: ||A_00|| ||A_01|| + ||A_01|| ||A_11|| = 2 * sqrt(2) * 2e-9
    est = 2 * math.sqrt(2.0) * 2e-9
    keep = co.triple_list(a, a, eps_sp=0.99 * est / 4)
    drop = co.triple_list(a, a, eps_sp=1.01 * est / 4)
    assert keep.tile_count[0, 1] == 2 and drop.tile_count[0, 1] == 0
    assert drop.tile_count[0, 0] == 1 and drop.tile_count[1, 1] == 1


def test_screening_uses_the_low_rank_blocks_reconstruction_norm():
    # A low-rank operand block enters the estimate with ||X W^T||_F (here diag(3, 4, 0, 0): 5),
    # not with the bound ||X||_F ||W||_F (sqrt(2) 5): the threshold between keeping and
    # dropping C_01 sits at the estimate 2 * 5e-9 + 5e-9 * 2 = 2e-8 over its 16 entries
    sizes = [4, 4]
    x = np.zeros((4, 2))
    x[0, 0] = x[1, 1] = 1.0
    w = np.zeros((4, 2))
    w[0, 0], w[1, 1] = 3e-9, 4e-9
    a = co.from_blocks(sizes, sizes, [[(1, np.eye(4)), (2, (x, w))],
                                      [(0, None), (1, np.eye(4))]])
    assert abs(co.block_norm(a.get(0, 1)) - 5e-9) <= 1e-24
    est = 2.0 * 5e-9 + 5e-9 * 2.0
    keep = co.triple_list(a, a, eps_sp=0.99 * est / 16)
    drop = co.triple_list(a, a, eps_sp=1.01 * est / 16)
    assert keep.tile_count[0, 1] == 2 and drop.tile_count[0, 1] == 0


def test_triple_output_rank_hand_values():
    # DD has no low-rank form; DL keeps B's rank, LD keeps A's; LL the smaller of the two, and
    # on a tie the X_A side (Eq. 1 as printed)
    assert co.triple_out_rank(co.T_DD, 5, 7) == 0
    assert co.triple_out_rank(co.T_DL, 5, 7) == 7
    assert co.triple_out_rank(co.T_LD, 5, 7) == 5
    assert co.triple_out_rank(co.T_LL, 5, 7) == 5
    assert co.triple_out_rank(co.T_LL, 9, 3) == 3
    assert co.lr_output_rank(4, 4) == (4, 0)
    assert co.lr_output_rank(3, 8) == (3, 1) and co.lr_output_rank(8, 3) == (3, 0)


def test_recompressed_singular_values_are_those_of_the_sum():
    # Invariant of recompression: the kept singular values of C_IJ are the leading singular
    # values of the exact block sum, and the rank is the count from the sigma tail.
    rng = np.random.default_rng(9)
    sizes = [12, 10]
    spec = [[(2, (rng.standard_normal((12, 2)), rng.standard_normal((12, 2)))),
             (2, (rng.standard_normal((12, 1)), rng.standard_normal((10, 1))))],
            [(2, (rng.standard_normal((10, 1)), rng.standard_normal((12, 1)))),
             (2, (rng.standard_normal((10, 2)), rng.standard_normal((10, 2))))]]
    a = co.from_blocks(sizes, sizes, spec)
    c = co.multiply(a, a, 1e-8)
    ref = a.to_dense() @ a.to_dense()
    for i, j in itertools.product(range(2), range(2)):
        blk = ref[c.row_off[i]:c.row_off[i + 1], c.col_off[j]:c.col_off[j + 1]]
        s_ref = np.linalg.svd(blk, compute_uv=False)
        got = c.get(i, j)
        r = co.truncation_rank(s_ref, 1e-8)
        assert 0 < r <= co.dense_rank_limit(*blk.shape)
        assert got.kind == co.KIND_LR and got.rank == r
        s_got = np.linalg.svd(got.dense(*blk.shape), compute_uv=False)[:r]
        assert np.allclose(s_got, s_ref[:r], rtol=1e-12, atol=1e-12 * s_ref[0])


def test_chain_product_structure():
    # the 1D chain overlap: only nearest-neighbour off-diagonal blocks survive the drop
    # threshold, so C = S S has at most three nonzero block diagonals after truncation at
    # 1e-8 (the next diagonal's norm is far below eps).
    w = wl.chain_overlap(n=512, n_clusters=8, lo=48, hi=80)
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    k = s.kinds()
    nb = len(w.row_sizes)
    for i in range(nb):
        for j in range(nb):
            if abs(i - j) > 1:
                assert k[i, j] == co.KIND_ZERO
    assert all(k[i, i] == co.KIND_DENSE for i in range(nb))
    c = co.multiply(s, s, w.eps_lr)
    ref = w.a @ w.a
    assert np.linalg.norm(c.to_dense() - ref) <= co.product_tolerance(w.a, w.a, w.eps_lr)


def test_lincomb_against_dense():
    rng = np.random.default_rng(21)
    sizes = [5, 7, 4]
    spec_x = wl.random_blocks_spec(rng, sizes, sizes)
    spec_y = wl.random_blocks_spec(rng, sizes, sizes)
    x, y = co.from_blocks(sizes, sizes, spec_x), co.from_blocks(sizes, sizes, spec_y)
    eps = 1e-10
    t = co.lincomb(-1.25, x, 0.375, y, 1.875, eps)
    ref = -1.25 * x.to_dense() + 0.375 * y.to_dense() + 1.875 * np.eye(16)
    assert np.linalg.norm(t.to_dense() - ref) <= 9 * eps + 1e-12 * np.linalg.norm(ref)
    for i in range(3):
        assert t.get(i, i).kind == co.KIND_DENSE


def test_transpose_and_scale():
    rng = np.random.default_rng(4)
    sizes = [3, 4]
    a = co.from_blocks(sizes, [5, 2], wl.random_blocks_spec(rng, sizes, [5, 2]))
    assert np.array_equal(co.transpose(a).to_dense(), a.to_dense().T)
    assert np.allclose(co.scale(a, -2.5).to_dense(), -2.5 * a.to_dense(), rtol=0, atol=1e-15)
