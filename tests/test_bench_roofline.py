"""Host arithmetic of the benchmark's batch rooflines (no GPU): the dense x dense flop count of a
product M M from block kinds against a brute-force triple loop, and the roofline fields built
from a batch run's profile, including the error path when an input is missing."""
import itertools
import sys

import numpy as np
import pytest


def test_dense_product_flops_brute_force():
    from paper_1509_00309_gb300 import clr
    from paper_1509_00309_gb300.diagnostics import dense_product_flops
    rng = np.random.default_rng(7)
    for n in (1, 3, 6):
        sizes = rng.integers(1, 40, n)
        kinds = rng.choice([clr.KIND_ZERO, clr.KIND_DENSE, clr.KIND_LR], size=(n, n))
        want = 0
        for i, k, j in itertools.product(range(n), repeat=3):
            if kinds[i, k] == clr.KIND_DENSE and kinds[k, j] == clr.KIND_DENSE:
                want += 2 * int(sizes[i]) * int(sizes[k]) * int(sizes[j])
        assert dense_product_flops(kinds, sizes) == want


def test_batch_roofline_fields(repo_root):
    sys.path.insert(0, repo_root)
    import bench
    inputs = {"ms_dense": 50.0, "ms_compress_qr": 2.0, "ms_compress_dense": 40.0,
              "svd_flops_fp64": 1.2e10, "svd_flops_fp32": 4.0e10, "svd_flops_fp64_qr": 2.0e9,
              "svd_flops_fp32_qr": 1.0e10, "dense_dd_flops": 4.0e10}
    r = bench.batch_roofline({"precision_mode": "fp64", "roofline_inputs": inputs}, 1.25)
    dn = r["recompression"]["compress_dense_kernel"]
    # 1e10 FP64 flops in 40 ms = 0.25 TFLOP/s of 1.25, plus 3e10 FP32 flops in 40 ms
    assert dn["achieved_fp64"] == pytest.approx(0.25)
    assert dn["frac"] == pytest.approx(0.2 + 0.75 / bench.FP32_TFLOPS_NOMINAL)
    d64 = r["dense_fp64"]
    assert d64["kernel"] == "dd_fp64_kernel" and d64["frac"] == pytest.approx(0.8 / 1.25)
    # an autotuned run mixes precisions in its dense phase: recompression only
    auto = bench.batch_roofline({"precision_mode": "auto", "roofline_inputs": inputs}, 1.25)
    assert set(auto) == {"recompression"}
    # missing inputs give an error field instead of failing the benchmark line
    assert "error" in bench.batch_roofline({"precision_mode": "fp64"}, 1.25)
    assert "error" in bench.batch_roofline(
        {"precision_mode": "fp64", "roofline_inputs": {"ms_dense": 1.0}}, 1.25)
