"""Pins of the Coulomb-like input (the paper's second matrix V: no block sparsity, only block-rank
sparsity), checked against the definition erf(r)/r written out with math.erf, and of the block
structure the method relies on."""
import math

import numpy as np

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl


def test_coulomb_entries_follow_the_definition():
    w = wl.lattice_coulomb(shape=(2, 2, 2), points_per_site=4, min_points=8, max_points=16)
    pts = w.extra["points"]
    rng = np.random.default_rng(0)
    for i, j in rng.integers(0, w.n, size=(40, 2)):
        r = math.dist(pts[i], pts[j])
        want = (2.0 / math.sqrt(math.pi) if r == 0.0 else math.erf(r) / r) + \
            (2e-2 if i == j else 0.0)
        assert abs(w.a[i, j] - want) <= 1e-15 * abs(want)
    assert np.array_equal(w.a, w.a.T)
    assert np.allclose(np.diag(w.a), 2.0 / math.sqrt(math.pi) + 2e-2, rtol=0, atol=1e-15)


def test_coulomb_is_positive_definite_and_only_rank_sparse():
    w = wl.lattice_coulomb(shape=(4, 4, 2), min_points=32, max_points=96)
    lam = np.linalg.eigvalsh(w.a)
    # the erf(r)/r kernel is positive semi-definite; the shift bounds the spectrum below
    assert lam[0] >= 2e-2 * (1 - 1e-9)
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    k = s.kinds()
    assert (k != co.KIND_ZERO).all()                       # no block sparsity
    assert (np.diag(k) == co.KIND_DENSE).all()
    off = ~np.eye(len(w.row_sizes), dtype=bool)
    assert (k[off] == co.KIND_LR).mean() > 0.5             # far blocks low rank
