"""Test helpers: move CLR matrices between the oracle's representation and the library's
block-slot pool layout (include/clr.h).  Used only by tests."""
import numpy as np

from oracle import clr_oracle as co


def slot(row_off, col_off, n_cols, i, j):
    m = row_off[i + 1] - row_off[i]
    return int(row_off[i]) * n_cols + m * int(col_off[j])


def pack(c: co.CLR):
    """Oracle CLR -> (kinds, ranks, pool) in the library's layout."""
    nr, nc = len(c.row_sizes), len(c.col_sizes)
    n_rows, n_cols = c.shape
    kinds = np.zeros((nr, nc), np.int32)
    ranks = np.zeros((nr, nc), np.int32)
    pool = np.zeros(n_rows * n_cols, np.float64)
    for (i, j), b in c.blocks.items():
        m, n = c.row_sizes[i], c.col_sizes[j]
        s = slot(c.row_off, c.col_off, n_cols, i, j)
        kinds[i, j] = b.kind
        if b.kind == co.KIND_DENSE:
            pool[s:s + m * n] = b.d.ravel(order="F")
            ranks[i, j] = min(m, n)
        elif b.kind == co.KIND_LR:
            r = b.x.shape[1]
            ranks[i, j] = r
            pool[s:s + m * r] = b.x.ravel(order="F")
            pool[s + m * r:s + (m + n) * r] = b.w.ravel(order="F")
    return kinds, ranks, pool


def unpack(row_sizes, col_sizes, kinds, ranks, pool) -> co.CLR:
    """Library layout -> oracle CLR (for inspecting factors and singular values)."""
    c = co.CLR(row_sizes, col_sizes)
    n_cols = c.shape[1]
    for i in range(len(row_sizes)):
        for j in range(len(col_sizes)):
            m, n = c.row_sizes[i], c.col_sizes[j]
            s = slot(c.row_off, c.col_off, n_cols, i, j)
            k = int(kinds[i, j])
            if k == co.KIND_DENSE:
                c.set(i, j, co.Block(co.KIND_DENSE, d=pool[s:s + m * n].reshape((m, n), order="F")))
            elif k == co.KIND_LR:
                r = int(ranks[i, j])
                x = pool[s:s + m * r].reshape((m, r), order="F")
                w = pool[s + m * r:s + (m + n) * r].reshape((n, r), order="F")
                c.set(i, j, co.Block(co.KIND_LR, x=x, w=w))
    return c


def to_library(ctx, c: co.CLR):
    kinds, ranks, pool = pack(c)
    return ctx.from_blocks(c.row_sizes, c.col_sizes, kinds, ranks, pool)


def from_library(m) -> co.CLR:
    kinds, ranks, _, pool = m.get_blocks()
    return unpack(m.row_sizes, m.col_sizes, kinds, ranks, pool)
