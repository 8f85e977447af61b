"""Exact-slice (Ozaki-scheme) reference values for the FP64-accurate tensor-core products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The error-free transformation of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of
matrix multiplication by using fast routines of matrix multiplication and its applications",
Numer. Algorithms 59, 2012), with the parameters the library uses, written from the scheme's
definition:

* Each row i of A (and each column j of B, i.e. each row of B^T) gets the exponent
  e_i = max over its nonzero entries of the exponent x with |a| < 2^x, so |a_ik| / 2^e_i < 1.
* v = a 2^(41 - e_i), rounded to the nearest integer (halves away from zero in magnitude), is
  written in balanced base 64: v = sum_{s=0}^{6} d_s 64^(6 - s) with d_1..d_6 in [-32, 31] and
  d_0 in [-32, 32].  Then a / 2^e_i = sum_s d_s 2^(-5 - 6 s) + r with |r| <= 2^-42.
* C_ij = 2^(e_i + f_j - 10) sum_{g=0}^{6} 2^(-6 g) G_g with
  G_g = sum_{s + t = g} sum_k d_s(a_ik) d_t(b_kj): the 28 slice pairs of weight >= 2^-42.

The digit products are integers of magnitude <= 2^10, so every G_g (and every partial sum of it)
is an integer far below 2^53: the FP64 matrix products of integer-valued digit matrices below
compute them exactly, and this module's value of the sliced product is exact up to the FP64
rounding of the final weighted sum over g.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

SLICES = 7
FRAC_BITS = 41          # v = round(a 2^(41 - e))
DIGIT_BASE = 64         # balanced digits: 6 bits each (the leading one 5 bits and a sign)
MAX_GROUP = SLICES - 1  # pairs with s + t <= 6 are kept


def row_exponents(a: np.ndarray) -> np.ndarray:
    """e_i = max over the nonzero entries of row i of the x with 2^(x-1) <= |a| < 2^x (numpy's
    frexp exponent); rows without nonzero entries get 0 (their digits are all zero)."""
    a = np.asarray(a, dtype=np.float64)
    _, x = np.frexp(a)
    x = np.where(a != 0.0, x.astype(np.int64), np.int64(-(1 << 40)))
    e = x.max(axis=1) if a.shape[1] else np.zeros(a.shape[0], dtype=np.int64)
    return np.where(e < -100000, 0, e).astype(np.int64)


def scaled_integers(a: np.ndarray, e: np.ndarray) -> np.ndarray:
    """v = round(|a| 2^(41 - e_i)) sign(a) per entry (nearest, halves up in magnitude), as int64.
    |v| <= 2^41 because |a| < 2^e_i."""
    a = np.asarray(a, dtype=np.float64)
    mant, x = np.frexp(np.abs(a))            # |a| = mant 2^x, 0.5 <= mant < 1
    x = x.astype(np.int64)
    # |a| 2^(41 - e) = mant 2^(x + 41 - e); mant has 53 bits: m53 = mant 2^53 is an integer
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
    """v = sum_{s=0}^{6} d_s 64^(6 - s): d_6 first from the bottom, each in [-32, 31], then the
    leading digit d_0 (the remaining quotient, |d_0| <= 32).  Returned as [d_0, ..., d_6]."""
    v = np.asarray(v, dtype=np.int64).copy()
    low = []
    for _ in range(SLICES - 1):
        d = ((v + 32) % DIGIT_BASE) - 32          # Python-style modulo: in [0, 64)
        low.append(d)
        v = (v - d) // DIGIT_BASE                 # exact
    return [v] + low[::-1]


def slices(a: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """Digit planes [d_0 .. d_6] of the rows of a and the row exponents."""
    e = row_exponents(a)
    return balanced_digits(scaled_integers(a, e)), e


def reconstruct(d: List[np.ndarray], e: np.ndarray) -> np.ndarray:
    """2^e_i sum_s d_s 2^(-5 - 6 s) (exact in FP64: at most 41 bits of fraction)."""
    acc = np.zeros(d[0].shape)
    for s, ds in enumerate(d):
        acc = acc + np.ldexp(ds.astype(np.float64), -5 - 6 * s)
    return np.ldexp(acc, e[:, None])


def group_sums(a: np.ndarray, b: np.ndarray):
    """G_g (g = 0..6) for C = A B, with the exponents of A's rows and B's columns."""
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


def sliced_product(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The exact value (up to the FP64 rounding of the sum over g) of the sliced product."""
    groups, ea, eb = group_sums(a, b)
    acc = np.zeros_like(groups[0])
    for g, gs in enumerate(groups):
        acc += np.ldexp(gs, -6 * g)
    return np.ldexp(acc, (ea[:, None] + eb[None, :] - 10))


def error_bound(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Entrywise bound on |sliced product - A B|: per term of the sum over k, the truncation of
    both operands (2^-42 relative to 2^e_i and 2^f_j each) and the dropped pairs s + t >= 7
    (sum over g >= 7 of (13 - g) 2^(10 - 10 - 6 g) <= 6.1 2^-42), i.e. K 2^-39 2^(e_i + f_j)."""
    ea = row_exponents(a)
    eb = row_exponents(np.asarray(b, dtype=np.float64).T)
    k = a.shape[1]
    return k * np.ldexp(1.0, -39) * np.ldexp(1.0, ea[:, None] + eb[None, :])
