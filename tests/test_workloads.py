"""The synthetic inputs follow their stated recipes (they stand in for the paper's overlap and
Coulomb matrices of 190 waters, Section 5): seeds, cluster-size ranges, chain and lattice
geometry, kernel entries checked against their definitions written out with math.exp, and the
batched configuration's ranges."""
import math

import numpy as np

from paper_1509_00309_gb300 import workloads as wl


def test_uneven_cluster_sizes_sum_and_range():
    rng = np.random.default_rng(0)
    for n, k, lo, hi in [(2048, 16, 96, 160), (16384, 96, 128, 224), (1100, 6, 128, 224)]:
        s = wl.uneven_cluster_sizes(rng, n, k, lo, hi)
        assert len(s) == k and sum(s) == n
        # rescaled from U[lo, hi]: within the range scaled by n / sum, the last one adjusted
        scale = n / (k * (lo + hi) / 2)
        assert min(s[:-1]) >= math.floor(lo * scale * 0.8) and max(s[:-1]) <= hi * scale * 1.25


def test_chain_overlap_entries_follow_the_definition():
    w = wl.chain_overlap()
    assert w.n == 2048 and len(w.row_sizes) == 16 and w.eps_lr == 1e-8 and w.drop_norm == 1e-12
    r = w.extra["points"][:, 0]
    steps = np.diff(r)
    assert np.all(steps > 0.3 - 0.1 - 1e-12) and np.all(steps < 0.3 + 0.1 + 1e-12)
    rng = np.random.default_rng(1)
    for i, j in rng.integers(0, w.n, size=(50, 2)):
        want = math.exp(-(r[i] - r[j]) ** 2 / 2.0) + (1e-3 if i == j else 0.0)
        assert abs(w.a[i, j] - want) <= 1e-15 * max(1.0, abs(want))
    assert np.array_equal(w.a, w.a.T)


def test_dense_normal_is_seeded_and_standard_normal():
    w1 = wl.dense_normal(n=1024, n_clusters=6)
    w2 = wl.dense_normal(n=1024, n_clusters=6)
    assert np.array_equal(w1.a, w2.a) and np.array_equal(w1.b, w2.b)
    assert sum(w1.row_sizes) == 1024 and w1.eps_lr == 0.0
    for x in (w1.a, w1.b):
        assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert not np.array_equal(w1.a, w1.b)


def test_lattice_overlap_geometry_and_clusters():
    shape = (4, 4, 2)
    w = wl.lattice_overlap(shape=shape)
    assert w.n == 16 * 4 * 4 * 2
    assert min(w.row_sizes) >= 64 and max(w.row_sizes) <= 256
    assert all(s % 16 == 0 for s in w.row_sizes)          # whole sites of 16 points
    assert (w.eps_lr, w.drop_norm, w.eps_sp) == (1e-6, 1e-10, 1e-13)
    pts = w.extra["points"]
    rng = np.random.default_rng(2)
    for i, j in rng.integers(0, w.n, size=(50, 2)):
        d2 = float(np.sum((pts[i] - pts[j]) ** 2))
        want = math.exp(-d2 / 1.5) + (1e-2 if i == j else 0.0)
        assert abs(w.a[i, j] - want) <= 1e-15 * max(1.0, abs(want))
    # every point within the jitter of a lattice site of spacing 0.5
    site = np.rint(pts / 0.5)
    assert np.all(np.abs(pts - 0.5 * site) <= 0.1 + 1e-12)


def test_batched_chains_ranges():
    ws = wl.batched_chains(n_instances=6, n_scale=0.05)
    again = wl.batched_chains(n_instances=6, n_scale=0.05)
    assert [w.n for w in ws] == [w.n for w in again]         # seeded
    for w in ws:
        assert w.eps_lr in (1e-6, 1e-8) and w.drop_norm == 1e-12
        assert 0.2 <= w.extra["spacing"] <= 0.6
        assert sum(w.row_sizes) == w.n


def test_chain_clusters_stay_within_range():
    # clusters from U[48, 256]; a short remainder joins or splits with its neighbour, so no
    # cluster exceeds the library's 256 nor falls below 24 (unless the chain itself is shorter)
    rng = np.random.default_rng(3)
    for _ in range(2000):
        n = int(rng.integers(1024, 8193))
        s = wl.chain_clusters(rng, n, 48, 256)
        assert sum(s) == n
        assert max(s) <= 256 and min(s) >= 24
