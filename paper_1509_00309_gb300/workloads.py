"""Seeded synthetic inputs for the CLR product and the Newton–Schulz S^-1/2 iteration.

This module only draws random numbers and evaluates the kernel functions that DEFINE the
input matrices (Gaussian overlap-like and erf(r)/r Coulomb-like kernels on jittered point sets,
i.i.d. normal entries).
It holds none of the method's arithmetic (no compression, no product, no iteration), so the
CUDA path and the FP64 oracle can both take their inputs from here.

The paper's own inputs (overlap and Coulomb matrices of 190 water molecules in the cc-pVTZ-RI
basis, N = 26,790 with 141x141 blocks; Section 4.2) are not available; these synthetic matrices
stand in for them. They share the features the method relies on: physics-driven uneven
blocking, block sparsity from distance decay, and low-rank off-diagonal blocks from a smooth
kernel (Section 4.1).

Every generator takes an explicit seed and uses ``numpy.random.default_rng(seed)``; the
default seed of workload ``c`` is ``1509 + c``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 1509


def default_seed(config_index: int) -> int:
    return SEED_BASE + int(config_index)


# ----------------------------------------------------------------------------------------------
# Cluster (tile) sizes
# ----------------------------------------------------------------------------------------------

def uneven_cluster_sizes(rng: np.random.Generator, n_total: int, n_clusters: int,
                         lo: int, hi: int) -> List[int]:
    """Draw ``n_clusters`` sizes uniformly from [lo, hi], rescale them to sum to ``n_total``
    (rounding, then adjusting the last cluster).  Non-uniform blocking is the normal case in
    the paper (blocking follows the physics, Section 3.2)."""
    raw = rng.integers(lo, hi + 1, size=n_clusters).astype(np.float64)
    sizes = np.maximum(1, np.rint(raw * (n_total / raw.sum()))).astype(np.int64)
    sizes[-1] += n_total - int(sizes.sum())
    if sizes[-1] < 1:
        raise ValueError("cluster rescaling produced an empty last cluster")
    return [int(s) for s in sizes]


def chain_clusters(rng: np.random.Generator, n_total: int, lo: int, hi: int) -> List[int]:
    """Contiguous clusters of a 1D chain with sizes drawn from [lo, hi] until ``n_total``
    points are covered; the last cluster takes the remainder.  A remainder shorter than
    ``lo // 2`` joins its neighbour, and where the two together would exceed ``hi`` they are
    split into two halves instead, so every cluster stays within [lo // 2, hi]."""
    sizes: List[int] = []
    left = n_total
    while left > 0:
        s = int(rng.integers(lo, hi + 1))
        s = min(s, left)
        sizes.append(s)
        left -= s
    if len(sizes) > 1 and sizes[-1] < max(1, lo // 2):
        both = sizes[-2] + sizes[-1]
        sizes.pop()
        if both <= hi:
            sizes[-1] = both
        else:
            sizes[-1] = both // 2
            sizes.append(both - both // 2)
    return sizes


# ----------------------------------------------------------------------------------------------
# Point sets and kernel matrices
# ----------------------------------------------------------------------------------------------

def chain_points(rng: np.random.Generator, n: int, spacing: float, jitter: float) -> np.ndarray:
    """1D chain r_i = spacing * i + U(-jitter, jitter); returns shape (n, 1)."""
    r = spacing * np.arange(n, dtype=np.float64) + rng.uniform(-jitter, jitter, size=n)
    return r.reshape(n, 1)


def gaussian_kernel_matrix(points: np.ndarray, width: float, diag_shift: float,
                           rows: Optional[slice] = None, cols: Optional[slice] = None,
                           chunk: int = 2048) -> np.ndarray:
    """S_ij = exp(-|r_i - r_j|^2 / width) + diag_shift * delta_ij (an overlap-like matrix of
    s-type Gaussians).  Evaluated in row chunks to bound temporaries."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    rs = rows if rows is not None else slice(0, pts.shape[0])
    cs = cols if cols is not None else slice(0, pts.shape[0])
    pr, pc = pts[rs], pts[cs]
    out = np.empty((pr.shape[0], pc.shape[0]), dtype=np.float64)
    for a in range(0, pr.shape[0], chunk):
        b = min(a + chunk, pr.shape[0])
        d2 = np.zeros((b - a, pc.shape[0]), dtype=np.float64)
        for ax in range(pts.shape[1]):
            diff = pr[a:b, ax][:, None] - pc[None, :, ax]
            d2 += diff * diff
        np.exp(-d2 / width, out=out[a:b])
    if diag_shift != 0.0:
        r0, c0 = rs.start or 0, cs.start or 0
        lo, hi = max(r0, c0), min(r0 + pr.shape[0], c0 + pc.shape[0])
        for g in range(lo, hi):
            out[g - r0, g - c0] += diag_shift
    return out


def coulomb_kernel_matrix(points: np.ndarray, beta: float, diag_shift: float,
                          chunk: int = 2048) -> np.ndarray:
    """V_ij = erf(beta r_ij) / r_ij (2 beta / sqrt(pi) at r = 0) + diag_shift * delta_ij: the
    Coulomb interaction of unit Gaussian charges (a positive definite, slowly decaying kernel:
    no block is negligible, far blocks are low rank).  Evaluated in row chunks."""
    from scipy.special import erf
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    out = np.empty((n, n), dtype=np.float64)
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        d2 = np.zeros((b - a, n), dtype=np.float64)
        for ax in range(pts.shape[1]):
            diff = pts[a:b, ax][:, None] - pts[None, :, ax]
            d2 += diff * diff
        r = np.sqrt(d2)
        with np.errstate(divide="ignore", invalid="ignore"):
            v = erf(beta * r) / r
        v[r == 0.0] = 2.0 * beta / np.sqrt(np.pi)
        out[a:b] = v
    out[np.diag_indices(n)] += diag_shift
    return out


def lattice_points(rng: np.random.Generator, shape: Sequence[int], spacing: float,
                   points_per_site: int, jitter: float) -> np.ndarray:
    """Jittered 3D lattice: each site of an ``shape`` lattice with the given spacing carries
    ``points_per_site`` points, each independently jittered by U(-jitter, jitter) per axis
    (like several basis functions per atom).  Returns (n_sites * points_per_site, 3) ordered
    site-major."""
    nx, ny, nz = shape
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    sites = spacing * g.reshape(-1, 3).astype(np.float64)
    pts = np.repeat(sites, points_per_site, axis=0)
    pts += rng.uniform(-jitter, jitter, size=pts.shape)
    return pts


def bisection_site_groups(rng: np.random.Generator, sites: np.ndarray, min_sites: int,
                          max_sites: int, frac_lo: float = 0.35,
                          frac_hi: float = 0.65) -> List[np.ndarray]:
    """Recursive coordinate bisection of lattice sites into spatial groups of between
    ``min_sites`` and ``max_sites`` sites: a group larger than ``max_sites`` is sorted along its
    widest axis and cut at a random fraction U(frac_lo, frac_hi) of its length (clipped so both
    parts keep ``min_sites``), which gives uneven cluster sizes.  Returns index arrays in
    traversal order."""
    out: List[np.ndarray] = []

    def rec(idx: np.ndarray) -> None:
        if len(idx) <= max_sites:
            out.append(idx)
            return
        ext = sites[idx].max(0) - sites[idx].min(0)
        ax = int(np.argmax(ext))
        order = idx[np.argsort(sites[idx, ax], kind="stable")]
        cut = int(round(rng.uniform(frac_lo, frac_hi) * len(order)))
        cut = min(max(cut, min_sites), len(order) - min_sites)
        rec(order[:cut])
        rec(order[cut:])

    rec(np.arange(sites.shape[0]))
    if min(len(g) for g in out) < min_sites:
        raise ValueError("bisection produced a group below the minimum size")
    return out


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    row_sizes: List[int]
    col_sizes: List[int]
    a: np.ndarray                 # dense FP64 (n_rows x n_cols), C order
    b: Optional[np.ndarray]       # None when B is A
    eps_lr: float
    drop_norm: float
    eps_sp: float = 0.0
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(sum(self.row_sizes))


def chain_overlap(n: int = 2048, n_clusters: int = 16, lo: int = 96, hi: int = 160,
                  spacing: float = 0.3, jitter: float = 0.05, width: float = 2.0,
                  diag_shift: float = 1e-3, eps_lr: float = 1e-8, drop_norm: float = 1e-12,
                  seed: int = default_seed(0)) -> Workload:
    """1D-chain overlap-like matrix S_ij = exp(-(r_i-r_j)^2/2) + 1e-3 delta_ij with N = 2048
    points split into 16 contiguous clusters of uneven size (U[96,160] rescaled to the sum).
    The product is S*S recompressed at 1e-8."""
    rng = np.random.default_rng(seed)
    sizes = uneven_cluster_sizes(rng, n, n_clusters, lo, hi)
    pts = chain_points(rng, n, spacing, jitter)
    s = gaussian_kernel_matrix(pts, width, diag_shift)
    return Workload("chain_overlap_n%d" % n, sizes, sizes, s, None, eps_lr, drop_norm,
                    extra={"points": pts})


def dense_normal(n: int = 16384, n_clusters: int = 96, lo: int = 128, hi: int = 224,
                 seed: int = default_seed(1), independent_b: bool = True) -> Workload:
    """All-dense product: N x N matrices with i.i.d. N(0,1) FP64 entries, clustered into
    ``n_clusters`` uneven clusters (U[lo,hi] rescaled).  Every block is full rank, so the CLR
    product is ordinary dense matrix multiplication (Section 4.3's epsilon -> 0 limit)."""
    rng = np.random.default_rng(seed)
    sizes = uneven_cluster_sizes(rng, n, n_clusters, lo, hi)
    a = rng.standard_normal((n, n))
    b = rng.standard_normal((n, n)) if independent_b else None
    return Workload("dense_normal_n%d" % n, sizes, sizes, a, b, 0.0, 0.0)


def lattice_overlap(shape=(16, 16, 8), points_per_site: int = 16, spacing: float = 0.5,
                    jitter: float = 0.1, width: float = 1.5, diag_shift: float = 1e-2,
                    min_points: int = 64, max_points: int = 256, eps_lr: float = 1e-6,
                    drop_norm: float = 1e-10, eps_sp: float = 1e-13,
                    seed: int = default_seed(2)) -> Workload:
    """3D overlap-like matrix on a jittered lattice: S_ij = exp(-|r_i-r_j|^2/1.5) + 1e-2
    delta_ij.  Each lattice site carries 16 points (like basis functions per atom), so a
    16x16x8 lattice gives N = 32768.  Sites are grouped into spatial clusters of 64..256 points
    by recursive coordinate bisection; points are ordered cluster by cluster."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    pts = lattice_points(rng, shape, spacing, points_per_site, jitter)
    sites = pts.reshape(-1, points_per_site, 3).mean(axis=1)
    groups = bisection_site_groups(rng, sites, max(1, min_points // points_per_site),
                                   max(1, max_points // points_per_site))
    order = np.concatenate([np.concatenate([np.arange(g * points_per_site,
                                                      (g + 1) * points_per_site)
                                            for g in grp]) for grp in groups])
    pts = pts[order]
    sizes = [len(g) * points_per_site for g in groups]
    s = gaussian_kernel_matrix(pts, width, diag_shift)
    return Workload("lattice_overlap_n%d" % pts.shape[0], sizes, sizes, s, None, eps_lr,
                    drop_norm, eps_sp, extra={"points": pts})


def lattice_coulomb(shape=(8, 8, 4), points_per_site: int = 16, spacing: float = 0.5,
                    jitter: float = 0.1, beta: float = 1.0, diag_shift: float = 2e-2,
                    min_points: int = 64, max_points: int = 256, eps_lr: float = 1e-6,
                    drop_norm: float = 1e-10, eps_sp: float = 1e-13,
                    seed: int = default_seed(5)) -> Workload:
    """Coulomb-like matrix on the jittered 3D lattice of ``lattice_overlap`` (the paper's second
    matrix V, which has no block sparsity, only block-rank sparsity): V_ij = erf(r_ij)/r_ij +
    2e-2 delta_ij (condition number ~1e5 at 8x8x4 sites), clusters of 64..256 points by
    bisection, eps_lr 1e-6."""
    rng = np.random.default_rng(seed)
    pts = lattice_points(rng, shape, spacing, points_per_site, jitter)
    sites = pts.reshape(-1, points_per_site, 3).mean(axis=1)
    groups = bisection_site_groups(rng, sites, max(1, min_points // points_per_site),
                                   max(1, max_points // points_per_site))
    order = np.concatenate([np.concatenate([np.arange(g * points_per_site,
                                                      (g + 1) * points_per_site)
                                            for g in grp]) for grp in groups])
    pts = pts[order]
    sizes = [len(g) * points_per_site for g in groups]
    v = coulomb_kernel_matrix(pts, beta, diag_shift)
    return Workload("lattice_coulomb_n%d" % pts.shape[0], sizes, sizes, v, None, eps_lr,
                    drop_norm, eps_sp, extra={"points": pts})


def batched_chains(n_instances: int = 64, n_lo: int = 1024, n_hi: int = 8192,
                   spacing_lo: float = 0.2, spacing_hi: float = 0.6, c_lo: int = 48,
                   c_hi: int = 256, eps_choices=(1e-6, 1e-8), seed: int = default_seed(3),
                   n_scale: float = 1.0) -> List[Workload]:
    """Independent 1D-chain overlap products of uneven size for one batched launch:
    N ~ U[1024, 8192], chain spacing ~ U[0.2, 0.6], clusters ~ U[48, 256], eps from
    {1e-6, 1e-8}.  ``n_scale`` shrinks every N (for tests) without changing the recipe."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n = int(rng.integers(n_lo, n_hi + 1))
        n = max(c_lo, int(round(n * n_scale)))
        sp = float(rng.uniform(spacing_lo, spacing_hi))
        eps = float(eps_choices[int(rng.integers(0, len(eps_choices)))])
        sizes = chain_clusters(rng, n, c_lo, c_hi)
        pts = chain_points(rng, n, sp, 0.05)
        s = gaussian_kernel_matrix(pts, 2.0, 1e-3)
        out.append(Workload("batched_%d_n%d" % (i, n), sizes, sizes, s, None, eps, 1e-12,
                            extra={"spacing": sp}))
    return out


def symmetric_normal(rng_or_seed, n: int) -> np.ndarray:
    """W = (G + G^T)/2 with G ~ N(0,1): the weight matrix of loss = trace(W S^-1/2)."""
    rng = rng_or_seed if isinstance(rng_or_seed, np.random.Generator) else \
        np.random.default_rng(rng_or_seed)
    g = rng.standard_normal((n, n))
    return 0.5 * (g + g.T)


def adjoint_lattice(n_sites_shape=(8, 8, 8), seed: int = default_seed(4), **kw) -> Workload:
    """The lattice-overlap construction scaled down (8x8x8 sites x 16 points = 8192; a 4x4x2
    lattice gives 512) plus a symmetric normal W for loss = trace(W S^-1/2)."""
    kw.setdefault("eps_lr", 1e-8)
    wl = lattice_overlap(shape=n_sites_shape, seed=seed, **kw)
    wl.extra["w"] = symmetric_normal(np.random.default_rng(seed + 100), wl.n)
    return wl


def random_blocks_spec(rng: np.random.Generator, row_sizes: Sequence[int],
                       col_sizes: Sequence[int], p_zero: float = 0.3, p_dense: float = 0.3,
                       max_rank: Optional[int] = None) -> List[List[tuple]]:
    """Random block structure for edge-case tests: for each block (I,J) a tuple
    (kind, payload) where kind 0 = zero, 1 = dense (payload: m x n array), 2 = low rank
    (payload: (X m x r, W n x r)) with X, W ~ N(0,1) and r drawn from [1, min(m,n)//2]."""
    out = []
    for m in row_sizes:
        row = []
        for n in col_sizes:
            u = rng.uniform()
            h = min(m, n) // 2
            if u < p_zero or (u >= p_zero + p_dense and h < 1):
                row.append((0, None))
            elif u < p_zero + p_dense:
                row.append((1, rng.standard_normal((m, n))))
            else:
                top = h if max_rank is None else max(1, min(h, max_rank))
                r = int(rng.integers(1, top + 1))
                row.append((2, (rng.standard_normal((m, r)), rng.standard_normal((n, r)))))
        out.append(row)
    return out
