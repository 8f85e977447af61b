"""The bf16 term split of the staging kernels (csrc/split_bf16.cuh), compiled for the host,
against the oracle's split from the format's definition (oracle/split_oracle.py): bit-exact
terms for values spread over the whole FP64 range and for the rounding edge cases (ties at the
bf16 rounding point, carries into the exponent, exact bf16 values, zero lower terms,
the boundaries of the kernels' fast path, subnormals)."""
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

from oracle import split_oracle as so

HERE = Path(__file__).resolve().parent


def bf16_bits(t: np.ndarray) -> np.ndarray:
    """bf16 bit patterns of FP64 values that are exact bf16 numbers."""
    f = t.astype(np.float32)
    assert np.array_equal(f.astype(np.float64), t)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def cases(rng: np.random.Generator) -> np.ndarray:
    n = 200_000
    sig = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    e = rng.integers(-140, 127, n)            # a_0 stays below the bf16 overflow
    spread = np.ldexp(sig, e)                                # every exponent the split meets
    normal = rng.standard_normal(n)                          # the benchmark's distribution
    # bit-pattern edge cases around the a_0 rounding point (bit 45) and the lower terms
    base = rng.integers(0, 1 << 62, 20_000, dtype=np.int64).astype(np.uint64)
    keep_hi = base & np.uint64(~((1 << 45) - 1) & ((1 << 64) - 1))
    tie = keep_hi | np.uint64(1 << 44)                       # exact tie for a_0
    ones = base | np.uint64((1 << 52) - 1)                   # carry into the exponent
    exact = keep_hi                                          # a_0 exact, lower terms zero
    low_only = keep_hi | (base & np.uint64(0xFF))            # tiny residuals (a_1 exact)
    tie1 = keep_hi | np.uint64(1 << 30)                      # residual 2^30 ulp: ties below
    tie1b = keep_hi | np.uint64((1 << 30) + (1 << 22))
    near_up = keep_hi | np.uint64((1 << 45) - 256) | (base & np.uint64(0xFF))  # tiny, negative
    pats = np.concatenate([tie, ones, exact, low_only, tie1, tie1b, near_up])
    ex_b = (pats >> np.uint64(52)) & np.uint64(0x7FF)
    pats = pats[ex_b < np.uint64(1023 + 127)]                # finite, a_0 below the overflow
    edge = pats.view(np.float64)
    edge = np.concatenate([edge, -edge])
    # boundaries of the fast path (biased exponents 1023 - 74 and 1023 + 126) and beyond
    b = []
    for ex in (-76, -75, -74, -73, -126, -127, -133, -134, 125, 126):
        m = rng.uniform(1.0, 2.0, 2000)
        b.append(np.ldexp(m, ex))
        b.append(np.ldexp(np.nextafter(2.0, 0.0) * np.ones(10), ex))
    sub = rng.integers(1, 1 << 52, 5000, dtype=np.int64).view(np.float64)
    special = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, 2.2250738585072014e-308,
                        3.0e38, 3.0 * 2.0 ** -80])
    return np.concatenate([spread, normal, edge, *b, sub, -sub, special])


def test_split_matches_definition(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "split_main"
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", str(exe),
                    str(HERE / "native" / "split_rounding_main.cpp")], check=True)
    rng = np.random.default_rng(1509)
    x = cases(rng)
    x = np.concatenate([x, rng.permutation(x)])   # pairs within and across the case groups
    (tmp_path / "x.bin").write_bytes(x.astype(np.float64).tobytes())
    subprocess.run([str(exe), str(tmp_path / "x.bin"), str(tmp_path / "t.bin")], check=True)
    got = np.frombuffer((tmp_path / "t.bin").read_bytes(), dtype=np.uint16).reshape(-1, 10)
    want = [bf16_bits(t) for t in so.split_terms(x, 3)] + \
        [bf16_bits(t) for t in so.split_terms(x, 2)]
    for col in range(10):   # scalar split, then the paired split
        w = want[col % 5]
        bad = np.nonzero(got[:, col] != w)[0]
        assert bad.size == 0, (col, x[bad[:5]], got[bad[:5], col], w[bad[:5]])
