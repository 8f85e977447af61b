"""Pins of the exact-slice (Ozaki-scheme) oracle against the scheme's definition and exact
arithmetic: digit ranges, reconstruction within 2^-48 of the row scale, the sliced product
against a brute-force evaluation in exact rational arithmetic, its error bound against the
exact product, exact results where the inputs need one digit, and the FP32 exactness
precondition of the GPU's segments."""
from fractions import Fraction

import numpy as np

from oracle import ozaki_oracle as oz


def _scaled(rng, m, n, spread=5.0):
    return rng.standard_normal((m, n)) * np.exp(rng.uniform(-spread, spread, (m, 1)))


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(1)
    a = _scaled(rng, 40, 60)
    a[3] = 0.0                       # a zero row
    a[5, 7] = 1e-300                 # a tiny entry beside normal ones
    d, e = oz.slices(a)
    assert len(d) == oz.SLICES
    assert np.abs(d[0]).max() <= 32
    for ds in d[1:]:
        assert ds.min() >= -32 and ds.max() <= 31
    # |a| < 2^e per row, and the digits reconstruct a within 2^-48 2^e
    nz = a != 0
    assert np.all(np.abs(a[nz]) < np.ldexp(1.0, np.broadcast_to(e[:, None], a.shape)[nz]))
    err = np.abs(oz.reconstruct(d, e) - a)
    assert np.all(err <= np.ldexp(1.0, e[:, None] - 48))
    assert not oz.reconstruct(d, e)[3].any()


def test_sliced_product_equals_exact_rational_evaluation():
    # brute force: the sliced product's definition evaluated with exact rationals
    rng = np.random.default_rng(2)
    a = _scaled(rng, 3, 5, 2.0)
    b = _scaled(rng, 4, 5, 2.0).T
    da, ea = oz.slices(a)
    db, eb = oz.slices(b.T)
    got = oz.sliced_product(a, b)
    for i in range(3):
        for j in range(4):
            tot = Fraction(0)
            for s in range(oz.SLICES):
                for t in range(oz.SLICES):
                    if s + t > oz.MAX_GROUP:
                        continue
                    w = Fraction(2) ** (int(ea[i]) + int(eb[j]) - 10 - 6 * (s + t))
                    tot += w * sum(int(da[s][i, k]) * int(db[t][j, k]) for k in range(5))
            assert abs(Fraction(got[i, j]) - tot) <= abs(tot) * Fraction(2) ** -50


def test_error_bound_against_exact_product():
    rng = np.random.default_rng(3)
    for m, k, n in ((7, 9, 5), (20, 64, 11)):
        a = _scaled(rng, m, k)
        b = _scaled(rng, n, k).T
        got = oz.sliced_product(a, b)
        bound = oz.error_bound(a, b)
        for i in range(m):
            for j in range(n):
                exact = sum(Fraction(a[i, q]) * Fraction(b[q, j]) for q in range(k))
                assert abs(Fraction(got[i, j]) - exact) <= Fraction(bound[i, j])


def test_one_digit_inputs_multiply_exactly():
    # entries with at most 5 significant bits at the row scale need only d_0: the sliced product
    # is then the exact product (no truncation, no dropped pair contributes)
    rng = np.random.default_rng(4)
    a = rng.integers(-31, 32, (12, 30)).astype(float) * 2.0 ** 7
    b = rng.integers(-31, 32, (30, 9)).astype(float) * 2.0 ** -3
    a[:, 0] = 31 * 2.0 ** 7          # every row reaches the top of its scale
    b[0, :] = -31 * 2.0 ** -3
    assert np.array_equal(oz.sliced_product(a, b), a @ b)


def test_segment_sums_fit_fp32():
    # the GPU sums a weight group over K segments of 1024 in FP32: with |digits| <= 32 the
    # worst case (all digits at the bound, all signs equal, the 8-pair group) stays below 2^24,
    # so every partial sum is an integer that FP32 represents exactly
    worst = oz.SLICES * 1024 * 32 * 32
    assert worst < 2 ** 24
    d = np.full((2, 1024), 32.0)
    assert float(np.max(oz.SLICES * (d @ d.T))) == worst
    assert np.float32(worst) == worst and np.float32(worst - 1) == worst - 1


def test_segmented_product_within_its_bound_and_sharper():
    # per-segment exponents: a row whose large entries sit in one K segment keeps its full
    # relative precision in the others.  A is large in segment 0 and B in segment 1, so no
    # term pairs two large entries: the segmented bound is far below the whole-row one, and
    # the segmented product meets it against the exact product (exact rationals)
    rng = np.random.default_rng(5)
    m, k, n, seg = 5, 12, 4, 4
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    a[:, :seg] *= 1e6
    b[seg:2 * seg, :] *= 1e6
    got = oz.sliced_product(a, b, seg=seg)
    bound = oz.error_bound(a, b, seg=seg)
    assert np.all(bound * 1e4 < oz.error_bound(a, b))
    for i in range(m):
        for j in range(n):
            exact = sum(Fraction(a[i, q]) * Fraction(b[q, j]) for q in range(k))
            assert abs(Fraction(got[i, j]) - exact) <= Fraction(bound[i, j])
    # one segment covering K is the unsegmented scheme
    assert np.array_equal(oz.sliced_product(a, b, seg=k), oz.sliced_product(a, b))
