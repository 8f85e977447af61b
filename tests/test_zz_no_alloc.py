"""The allocation-free single-block compression (clr_block_compress_noalloc) against the
library's regular path (clr_mat_from_dense on a one-block matrix), through the C ABI.

The entry point exists for callers that may not allocate device memory (inside a stream
capture, on hosts with pre-planned device memory, inside a framework that owns the allocator);
its scratch is a fixed device array in the library.  Its results must match the allocating
path's, and two calls in a row must not disturb each other through the shared array.  This file
is collected last so that a failure here never hides another test's result."""
import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    return clr


def _blocks():
    w = wl.chain_overlap(n=768, n_clusters=6, lo=96, hi=160)
    off = np.concatenate([[0], np.cumsum(w.row_sizes)])
    blk = lambda i, j: w.a[off[i]:off[i + 1], off[j]:off[j + 1]]  # noqa: E731
    rng = np.random.default_rng(8)
    wide = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 200))   # m < n, rank 5
    return [("low rank (neighbours)", blk(2, 3)), ("dense (diagonal)", blk(1, 1)),
            ("zero after truncation (far)", blk(0, 5)), ("wide rank 5", wide)]


def _noalloc(lib, torch, a, eps):
    m, n = a.shape
    k = min(m, n)
    block = torch.from_numpy(np.ascontiguousarray(a.T)).cuda().T   # column-major view
    x = torch.full((m * k,), np.nan, dtype=torch.float64, device="cuda")
    w = torch.full((n * k,), np.nan, dtype=torch.float64, device="cuda")
    s = torch.zeros(k, dtype=torch.float64, device="cuda")
    st = torch.full((3,), -7, dtype=torch.int32, device="cuda")
    lib.block_compress_noalloc(block, eps, x, w, st, sigma_out=s)
    torch.cuda.synchronize()
    kind, rank, err = (int(v) for v in st.cpu())
    return kind, rank, err, x.cpu().numpy(), w.cpu().numpy(), s.cpu().numpy()


def _regular(ctx, a, eps):
    m, n = a.shape
    mat = ctx.from_dense(a, [m], [n], eps_lr=eps)
    kinds, ranks, _, pool = mat.get_blocks()
    kind, rank = int(kinds[0, 0]), int(ranks[0, 0])
    if kind == co.KIND_LR:
        x = pool[:m * rank].reshape((m, rank), order="F")
        wf = pool[m * rank:(m + n) * rank].reshape((n, rank), order="F")
        return kind, rank, x @ wf.T
    return kind, rank, mat.to_dense()


def test_noalloc_matches_regular_path_two_calls_in_a_row(lib):
    import torch
    eps = 1e-8
    ctx = lib.Context(0, precision="fp64", eps_lr=eps)
    cases = _blocks()
    for first, second in [(cases[0], cases[1]), (cases[2], cases[3]), (cases[3], cases[0])]:
        results = [_noalloc(lib, torch, a, eps) for _, a in (first, second)]
        for (name, a), (kind, rank, err, x, w, sig) in zip((first, second), results):
            m, n = a.shape
            rkind, rrank, rdense = _regular(ctx, a, eps)
            assert err == 0, name
            assert kind == rkind, name
            assert abs(rank - rrank) <= 1, name
            if kind == co.KIND_LR:
                rec = x[:m * rank].reshape((m, rank), order="F") @ \
                    w[:n * rank].reshape((n, rank), order="F").T
                assert np.linalg.norm(rec - rdense) <= 2 * eps + 1e-12 * np.linalg.norm(a), name
                assert np.linalg.norm(rec - a) <= eps * (1 + 1e-6), name
            if kind != co.KIND_ZERO:
                s_ref = np.linalg.svd(a, compute_uv=False)
                assert np.allclose(sig, s_ref, rtol=1e-10, atol=1e-12 * s_ref[0]), name


def test_noalloc_is_deterministic_and_rejects_oversize(lib):
    import torch
    a = _blocks()[0][1]
    r1 = _noalloc(lib, torch, a, 1e-8)
    r2 = _noalloc(lib, torch, a, 1e-8)
    assert r1[:3] == r2[:3]
    # the unwritten tails of the output buffers keep their NaN fill in both calls
    assert np.array_equal(r1[3], r2[3], equal_nan=True)
    assert np.array_equal(r1[4], r2[4], equal_nan=True)
    big = torch.zeros((4, 257), dtype=torch.float64, device="cuda").T   # 257 x 4, column-major
    out = torch.empty(257 * 4, dtype=torch.float64, device="cuda")
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.ClrError) as e:
        lib.block_compress_noalloc(big, 1e-8, out, out, st)
    assert e.value.status == lib.CLR_EINVAL
