"""Exact-slice (Ozaki-scheme) reference values for the FP64-accurate tensor-core products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The error-free transformation of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of
matrix multiplication by using fast routines of matrix multiplication and its applications",
Numer. Algorithms 59, 2012), with the parameters the library uses, written from the scheme's
definition:

* Each row i of A (and each column j of B, i.e. each row of B^T) gets the exponent
  e_i = max over its nonzero entries of the exponent x with |a| < 2^x, so |a_ik| / 2^e_i < 1.
* v = a 2^(47 - e_i), rounded to the nearest integer (halves away from zero in magnitude), is
  written in balanced base 64: v = sum_{s=0}^{7} d_s 64^(7 - s) with d_1..d_7 in [-32, 31] and
  d_0 in [-32, 32].  Then a / 2^e_i = sum_s d_s 2^(-5 - 6 s) + r with |r| <= 2^-48.
* C_ij = 2^(e_i + f_j - 10) sum_{g=0}^{7} 2^(-6 g) G_g with
  G_g = sum_{s + t = g} sum_k d_s(a_ik) d_t(b_kj): the 36 slice pairs of weight >= 2^-48.
  (Eight slices: the truncation and the dropped pairs then err by about 2^-48 relative to the
  rows' and columns' largest entries per term, which the low-rank sums of the Newton-Schulz
  iterates need at eps = 1e-8; seven would leave about 2^-42.)
* The library applies the scheme to each K segment of 1024 columns, with exponents taken over
  that segment only, and sums the segment products (sliced_product's seg argument): a row
  whose few large entries lie in one segment keeps its full relative precision elsewhere.

The digit products are integers of magnitude <= 2^10, so every G_g (and every partial sum of it)
is an integer far below 2^53: the FP64 matrix products of integer-valued digit matrices below
compute them exactly, and this module's value of the sliced product is exact up to the FP64
rounding of the final weighted sum over g.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

SLICES = 8
FRAC_BITS = 47          # v = round(a 2^(47 - e))
DIGIT_BASE = 64         # balanced digits: 6 bits each (the leading one 5 bits and a sign)
MAX_GROUP = SLICES - 1  # pairs with s + t <= 7 are kept


def row_exponents(a: np.ndarray) -> np.ndarray:
    """e_i = max over the nonzero entries of row i of the x with 2^(x-1) <= |a| < 2^x (numpy's
    frexp exponent); rows without nonzero entries get 0 (their digits are all zero)."""
    a = np.asarray(a, dtype=np.float64)
    _, x = np.frexp(a)
    x = np.where(a != 0.0, x.astype(np.int64), np.int64(-(1 << 40)))
    e = x.max(axis=1) if a.shape[1] else np.zeros(a.shape[0], dtype=np.int64)
    return np.where(e < -100000, 0, e).astype(np.int64)


def scaled_integers(a: np.ndarray, e: np.ndarray) -> np.ndarray:
    """v = round(|a| 2^(47 - e_i)) sign(a) per entry (nearest, halves up in magnitude), as int64.
    |v| <= 2^47 because |a| < 2^e_i."""
    a = np.asarray(a, dtype=np.float64)
    mant, x = np.frexp(np.abs(a))            # |a| = mant 2^x, 0.5 <= mant < 1
    x = x.astype(np.int64)
    # |a| 2^(47 - e) = mant 2^(x + 47 - e); mant has 53 bits: m53 = mant 2^53 is an integer
    m53 = np.ldexp(mant, 53).astype(np.int64)
    sh = (x + FRAC_BITS - e[:, None]) - 53     # v = m53 2^sh
    out = np.zeros(a.shape, dtype=np.int64)
    pos = sh >= 0
    out[pos] = np.left_shift(m53[pos], sh[pos])
    neg = (sh < 0) & (sh > -63)
    r = -sh[neg]
    out[neg] = np.right_shift(m53[neg] + np.left_shift(np.int64(1), r - 1), r)
    out[a == 0.0] = 0
    return np.where(a < 0.0, -out, out)


def balanced_digits(v: np.ndarray) -> List[np.ndarray]:
    """v = sum_{s=0}^{7} d_s 64^(7 - s): d_7 first from the bottom, each in [-32, 31], then the
    leading digit d_0 (the remaining quotient, |d_0| <= 32).  Returned as [d_0, ..., d_7]."""
    v = np.asarray(v, dtype=np.int64).copy()
    low = []
    for _ in range(SLICES - 1):
        d = ((v + 32) % DIGIT_BASE) - 32          # Python-style modulo: in [0, 64)
        low.append(d)
        v = (v - d) // DIGIT_BASE                 # exact
    return [v] + low[::-1]


def slices(a: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """Digit planes [d_0 .. d_7] of the rows of a and the row exponents."""
    e = row_exponents(a)
    return balanced_digits(scaled_integers(a, e)), e


def reconstruct(d: List[np.ndarray], e: np.ndarray) -> np.ndarray:
    """2^e_i sum_s d_s 2^(-5 - 6 s) (exact in FP64: at most 47 bits of fraction)."""
    acc = np.zeros(d[0].shape)
    for s, ds in enumerate(d):
        acc = acc + np.ldexp(ds.astype(np.float64), -5 - 6 * s)
    return np.ldexp(acc, e[:, None])


def group_sums(a: np.ndarray, b: np.ndarray):
    """G_g (g = 0..7) for C = A B, with the exponents of A's rows and B's columns."""
    da, ea = slices(a)
    db, eb = slices(np.asarray(b, dtype=np.float64).T)
    groups = []
    for g in range(MAX_GROUP + 1):
        acc = np.zeros((a.shape[0], b.shape[1]))
        for s in range(g + 1):
            t = g - s
            acc += da[s].astype(np.float64) @ db[t].astype(np.float64).T
        groups.append(acc)
    return groups, ea, eb


def _segments(k: int, seg):
    """Column ranges [k0, k1) of the K segments (one range when seg is None)."""
    if seg is None or seg >= k:
        return [(0, k)]
    return [(k0, min(k, k0 + seg)) for k0 in range(0, k, seg)]


def sliced_product(a: np.ndarray, b: np.ndarray, seg=None) -> np.ndarray:
    """The exact value (up to the FP64 rounding of the sums over g and over segments) of the
    sliced product.  With seg, the scheme runs on each K segment [k0, k0 + seg) separately --
    exponents e_i and f_j over that segment's entries only -- and the segment products are
    summed: sum over segments of 2^(e_i + f_j - 10) sum_g 2^(-6 g) G_g."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.zeros((a.shape[0], b.shape[1]))
    for k0, k1 in _segments(a.shape[1], seg):
        groups, ea, eb = group_sums(a[:, k0:k1], b[k0:k1, :])
        acc = np.zeros_like(groups[0])
        for g, gs in enumerate(groups):
            acc += np.ldexp(gs, -6 * g)
        out += np.ldexp(acc, (ea[:, None] + eb[None, :] - 10))
    return out


def error_bound(a: np.ndarray, b: np.ndarray, seg=None) -> np.ndarray:
    """Entrywise bound on |sliced product - A B|: per term of the sum over k, the truncation of
    both operands (2^-48 relative to 2^e_i and 2^f_j each, 2^-47 together with their product)
    and the dropped pairs s + t >= 8 (sum over g >= 8 of (15 - g) 2^(10 - 10 - 6 g)
    <= 7.2 2^-48), below 2^-44 2^(e_i + f_j): K 2^-44 2^(e_i + f_j), summed over the K
    segments with their own exponents when seg is given."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.zeros((a.shape[0], b.shape[1]))
    for k0, k1 in _segments(a.shape[1], seg):
        ea = row_exponents(a[:, k0:k1])
        eb = row_exponents(b[k0:k1, :].T)
        out += (k1 - k0) * np.ldexp(1.0, -44) * np.ldexp(1.0, ea[:, None] + eb[None, :])
    return out
