"""Pins of the split-precision reference (bf16 rounding from the format's definition)."""
import numpy as np
import pytest
import torch

from oracle import split_oracle as so


def test_bf16_round_hand_values():
    u = 2.0 ** -7  # bf16 spacing in [1, 2)
    vals = np.array([1.0, 1.0 + u / 2, 1.0 + 1.5 * u, 1.0 + 0.49 * u, -3.0, 0.0,
                     2.0 - u / 4, 2.0 ** -130 * 1.3])
    want = np.array([1.0, 1.0, 1.0 + 2 * u, 1.0, -3.0, 0.0, 2.0, 2.0 ** -133 * 10 * 1.0])
    got = so.bf16_round(vals)
    assert np.array_equal(got[:7], want[:7])
    # subnormal: 1.3 * 2^-130 = 10.4 * 2^-133 -> 10 * 2^-133
    assert got[7] == 10 * 2.0 ** -133


def test_bf16_round_matches_torch_on_binary32_inputs():
    # torch's float32 -> bfloat16 conversion rounds to nearest even; on inputs that are
    # binary32 values no double rounding can occur, so the two definitions must agree.
    rng = np.random.default_rng(0)
    x32 = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(so.bf16_round(x32.astype(np.float64)), ref)


@pytest.mark.parametrize("terms,bound", [(1, 2.0 ** -8), (2, 2.0 ** -16), (3, 2.0 ** -24)])
def test_split_terms_reconstruct(terms, bound):
    rng = np.random.default_rng(terms)
    x = rng.standard_normal(5000) * np.exp(rng.uniform(-5, 5, 5000))
    parts = so.split_terms(x, terms)
    for p in parts:
        assert np.array_equal(so.bf16_round(p), p)
    rest = np.abs(x - np.sum(parts, axis=0))
    assert np.all(rest <= bound * np.abs(x))


@pytest.mark.parametrize("mode,rel", [("bf16x3", 3 * 2.0 ** -16), ("bf16x6", 7 * 2.0 ** -24)])
def test_split_product_error_bound(mode, rel):
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((40, 300)), rng.standard_normal((300, 30))
    got = so.split_product(a, b, mode)
    err = np.abs(got - a @ b)
    assert np.all(err <= rel * so.abs_product(a, b))


def test_split_product_pair_sets_exactly():
    # a = 1 + 2^-9 + 2^-18 and b = 1 + 2^-10 + 2^-20 split (no ties) into the bf16 terms
    # (1, 2^-9, 2^-18) and (1, 2^-10, 2^-20), so every term pair contributes a distinct power of
    # two and the sum shows exactly which pairs a mode takes: bf16x3 the pairs (0,0), (0,1),
    # (1,0) of the 2-term split; bf16x6 also (0,2), (1,1), (2,0), leaving out 2^-28, 2^-29 and
    # 2^-38
    a = np.array([[1.0 + 2.0 ** -9 + 2.0 ** -18]])
    b = np.array([[1.0 + 2.0 ** -10 + 2.0 ** -20]])
    assert [float(t[0, 0]) for t in so.split_terms(a, 3)] == [1.0, 2.0 ** -9, 2.0 ** -18]
    assert [float(t[0, 0]) for t in so.split_terms(b, 3)] == [1.0, 2.0 ** -10, 2.0 ** -20]
    assert so.split_product(a, b, "bf16x3")[0, 0] == 1.0 + 2.0 ** -9 + 2.0 ** -10
    want6 = 1.0 + 2.0 ** -9 + 2.0 ** -10 + 2.0 ** -18 + 2.0 ** -19 + 2.0 ** -20
    assert so.split_product(a, b, "bf16x6")[0, 0] == want6
    assert (a @ b)[0, 0] - want6 == 2.0 ** -28 + 2.0 ** -29 + 2.0 ** -38
