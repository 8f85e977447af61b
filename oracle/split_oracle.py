"""Split-precision reference values (bfloat16 multi-term splits) for the tensor-core products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A FP64 value a is split into bf16 terms a = a_0 + a_1 + ... + a_{t-1} + residual, with
a_0 = bf16(a), a_1 = bf16(a - a_0), ... (every difference is exact in FP64).  A split product
sums selected term products A_p B_q; products of bf16 values are exact in FP64, so the FP64
sum here is the exact value of the split product up to FP64 rounding.  The GPU differs from it
only by its FP32 accumulation.

bf16 rounding is written from the format's definition (IEEE binary32 with the low 16 fraction
bits removed: 8 significant bits, exponent range of binary32), round to nearest, ties to even,
directly from FP64 (no intermediate rounding to FP32).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

BF16_SIG_BITS = 8          # significant bits including the implicit one
BF16_MIN_EXP = -126        # exponent of the smallest normal bf16 (same as binary32)

# Term pairs of the split products: BF16x3 uses 2 terms and drops a_1 b_1; BF16x6 uses 3
# terms and keeps every pair with p + q <= 2.
PAIRS = {
    "bf16x3": (2, ((0, 0), (0, 1), (1, 0))),
    "bf16x6": (3, ((0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0))),
}


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest bf16 value (ties to even), returned as FP64.

    For |x| in [2^e, 2^(e+1)) the bf16 spacing is 2^(e-7); below the smallest normal 2^-126
    the spacing stays 2^-133 (subnormals).  x / spacing is an exact power-of-two scaling, and
    numpy's rint rounds half to even."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = (x != 0.0) & np.isfinite(x)
    _, e = np.frexp(x[nz])                    # x = f * 2^e, 0.5 <= |f| < 1
    lead = np.maximum(e - 1, BF16_MIN_EXP)    # exponent of the leading bit (clamped)
    spacing_exp = lead - (BF16_SIG_BITS - 1)
    q = np.ldexp(x[nz], -spacing_exp)
    out[nz] = np.ldexp(np.rint(q), spacing_exp)
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out


def split_terms(x: np.ndarray, terms: int) -> List[np.ndarray]:
    """a_0 = bf16(a), a_i = bf16(a - a_0 - ... - a_{i-1}); each difference is exact in FP64."""
    rest = np.asarray(x, dtype=np.float64).copy()
    out = []
    for _ in range(terms):
        t = bf16_round(rest)
        out.append(t)
        rest = rest - t
    return out


def split_product(a: np.ndarray, b: np.ndarray, mode: str) -> np.ndarray:
    """Exact (FP64) value of the split product sum_{(p,q)} A_p B_q for ``mode`` in PAIRS."""
    terms, pairs = PAIRS[mode]
    sa, sb = split_terms(a, terms), split_terms(b, terms)
    out = np.zeros((a.shape[0], b.shape[1]))
    for p, q in pairs:
        out += sa[p] @ sb[q]
    return out


def abs_product(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """|A| |B| elementwise-absolute product: the scale of the rounding errors of A B."""
    return np.abs(a) @ np.abs(b)
