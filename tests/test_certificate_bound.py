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
