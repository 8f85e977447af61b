"""The dense certificate of the pivoted-QR pre-reduction, checked on the CPU against exact
singular values: for A P = Q R (column-pivoted Householder QR, A p x q) and every leading
triangle R_K' with q/2 < K' <= q,

    sum_{i > q/2} sigma_i(A)^2  >=  (K' - q/2)^2 / ||R_K'^-1||_F^2

(interlacing of the first K' columns of Q^T A P, then the Cauchy-Schwarz inequality over the
K' - q/2 smallest singular values of R_K').  The GPU kernel stores a tile dense when the largest
of these bounds exceeds eps^2; the bound must never exceed the true tail, and it must certify
tiles whose tail is spread over many singular values below eps, which sigma_min(R_{q/2+1})
alone does not."""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")


def _tail_bound_sq(r, h):
    q = r.shape[0]
    ri = scipy_linalg.solve_triangular(r[:q, :q], np.eye(q))
    prefix = np.cumsum(np.sum(ri * ri, axis=0))     # ||R_K'^-1||_F^2 for K' = 1..q
    best = 0.0
    for kk in range(h + 1, q + 1):
        f = prefix[kk - 1]
        if not np.isfinite(f) or f <= 0:
            break
        best = max(best, (kk - h) ** 2 / f)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_tail_bound_never_exceeds_the_true_tail(seed):
    # geometric spectra of random decay through the eps region, random singular vectors
    rng = np.random.default_rng(seed)
    q = 96
    h = q // 2
    for trial in range(25):
        rate = rng.uniform(0.7, 0.95)
        s = np.exp(np.log(rate) * np.arange(q)) * rng.uniform(0.5, 5.0)
        u, _ = np.linalg.qr(rng.standard_normal((q + 16, q)))
        v, _ = np.linalg.qr(rng.standard_normal((q, q)))
        a = (u * s) @ v.T
        tail2 = float(np.sum(np.linalg.svd(a, compute_uv=False)[h:] ** 2))
        _, r, _ = scipy_linalg.qr(a, pivoting=True, mode="economic")
        b2 = _tail_bound_sq(r, h)
        assert b2 <= tail2 * (1 + 1e-8), (b2, tail2)
        # the sigma_min form is the first triangle's bound, never above the best one
        assert _tail_bound_sq(r[: h + 1, : h + 1], h) <= b2 * (1 + 1e-12)


def test_tail_bound_catches_a_flat_tail_below_eps():
    # 40 singular values at 0.4 eps beyond index q/2: sigma_{q/2+1} < eps, but the tail
    # sqrt(40) 0.4 eps > eps, so the tile is dense; the bound over the triangles certifies it
    rng = np.random.default_rng(11)
    q, eps = 96, 1e-8
    h = q // 2
    s = np.concatenate([np.geomspace(10.0, 1e-6, h), np.full(40, 0.4 * eps),
                        np.full(q - h - 40, 1e-14)])
    u, _ = np.linalg.qr(rng.standard_normal((q, q)))
    v, _ = np.linalg.qr(rng.standard_normal((q, q)))
    a = (u * s) @ v.T
    tail2 = float(np.sum(s[h:] ** 2))
    assert tail2 > eps ** 2
    _, r, _ = scipy_linalg.qr(a, pivoting=True, mode="economic")
    b2 = _tail_bound_sq(r, h)
    assert eps ** 2 < b2 <= tail2 * (1 + 1e-8)                 # certified dense
    assert _tail_bound_sq(r[: h + 1, : h + 1], h) < eps ** 2   # sigma_min alone: no


def _truncation_rank(s, eps):
    """Smallest r with sqrt(sum_{i >= r} s_i^2) <= eps (s descending)."""
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    hit = np.nonzero(np.append(tail, 0.0) <= eps)[0]
    return int(hit[0])


@pytest.mark.parametrize("m,n,lead,top", [(200, 200, 90, 0.3), (200, 200, 100, 0.5),
                                          (150, 230, 67, 0.3), (230, 150, 40, 2.0),
                                          (120, 120, 20, 0.05)])
def test_svd_of_r_truncation_error_at_any_qr_rank(m, n, lead, top):
    # The recompression of a densely accumulated tile: column-pivoted QR A P = Q R stopped at the
    # first k with ||R_22||_F <= eps/16, then the SVD of the k x q factor R truncated at the
    # budget sqrt(eps^2 - ||R_22||_F^2).  The two errors lie in orthogonal rows of Q^T A P, so
    # ||A - X W^T||_F <= eps whatever k is, also past 3q/5 (where the kernel used to take the
    # full SVD of A instead), and the rank is the exact SVD's or one more (the budget split).
    rng = np.random.default_rng(m + n + lead)
    eps = 1e-8
    q = min(m, n)
    u, _ = np.linalg.qr(rng.standard_normal((m, q)))
    v, _ = np.linalg.qr(rng.standard_normal((n, q)))
    rho = (2e-3) ** (1.0 / (q - lead - 1))
    s = np.concatenate([np.logspace(0, -2, lead), top * eps * rho ** np.arange(q - lead)])
    a = (u * s) @ v.T
    at = a if m >= n else a.T                         # p x q, p >= q
    qf, r, piv = scipy_linalg.qr(at, pivoting=True, mode="economic")
    trail = np.sqrt(np.cumsum((np.sum(r * r, axis=1))[::-1])[::-1])   # ||R[j:, :]||_F
    k = int(np.nonzero(np.append(trail, 0.0) <= eps / 16)[0][0])
    r22 = float(trail[k]) if k < q else 0.0
    ur, sr, vrt = np.linalg.svd(r[:k, :], full_matrices=False)
    budget = np.sqrt(eps ** 2 - r22 ** 2)
    rk = _truncation_rank(sr, budget)
    approx = (qf[:, :k] @ (ur[:, :rk] * sr[:rk]) @ vrt[:rk, :])[:, np.argsort(piv)]
    approx = approx if m >= n else approx.T
    assert np.linalg.norm(a - approx) <= eps * (1 + 1e-6)
    r_svd = _truncation_rank(np.linalg.svd(a, compute_uv=False), eps)
    assert r_svd <= rk <= r_svd + 1
    if (m, n, lead) in ((200, 200, 90), (150, 230, 67), (200, 200, 100)):
        assert k > (3 * q) // 5          # the cases the full SVD used to take
