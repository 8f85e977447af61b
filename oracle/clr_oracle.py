"""FP64 CPU oracle: CLR matrices, their product, and the Newton–Schulz S^-1/2 iteration.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the library never imports this file.

Everything here is the plain definition written out in FP64 with NumPy/LAPACK.  Where the
method reaches a result with a plain definition, the oracle computes that definition:

* Build (Section 4.1): each block M_IJ is kept as X W^T with the smallest rank r whose
  Frobenius error is <= eps_lr.  The paper builds X, W with a rank-revealing QR; the optimal
  rank is reached by the truncated SVD, which is what this oracle uses (reading: SVD, the
  minimal form of the same criterion).  Blocks whose rank exceeds half of full rank are stored
  dense (Section 4.1); blocks whose norm is below ``drop_norm`` are dropped.
* Product (Section 4.1): low-rank GEMM (Z = W_A^T X_B, then X_A Z or W_B Z^T, whichever gives
  the smaller rank), low-rank addition by concatenating factors (Eq. lr_addition), and
  recompression by QR of both factors, a decomposition of the small core M = R_X R_W^T and
  re-expansion.  Recompressing the concatenated sum with an SVD of M gives exactly the
  truncated SVD of the summed block, so the oracle forms the block sum of the reconstructed
  products in FP64 and truncates it with the rule of Build.  Block C_IJ is computed only if
  the screening estimate sum_K ||A_IK||_F ||B_KJ||_F exceeds eps_sp * area(C_IJ) (reading of
  the inequality printed in Section 4.1, whose direction is inverted).
* A C tile that receives at least one dense x dense contribution is accumulated and kept dense
  (reading; re-tested for low rank only with ``recompress_dense``).
* Newton–Schulz (Section 4.2): X_n = alpha Y_n Z_n, T_n = (15 I - 10 X_n + 3 X_n^2)/8,
  Z_{n+1} = Z_n T_n, Y_{n+1} = T_n Y_n, Z_0 = I, Y_0 = M; sqrt(alpha) Z -> M^{-1/2}.
* The gradient of L = trace(W S^{-1/2}) is the Daleckii–Krein divided-difference formula;
  the NS adjoint runs the NS recurrences backwards.

Pins: tests/test_oracle_*.py check these functions against closed forms, brute force on tiny
inputs, invariants and library routines (dense GEMM, eigh), never against the CUDA path.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

KIND_ZERO, KIND_DENSE, KIND_LR = 0, 1, 2
# Kinds of a tile product (A block kind x B block kind), in the order used by the triple list.
T_DD, T_DL, T_LD, T_LL = 0, 1, 2, 3
# Accumulation mode of a C tile.
MODE_ZERO, MODE_DENSE, MODE_LR = 0, 1, 2


@dataclasses.dataclass
class Block:
    kind: int
    d: Optional[np.ndarray] = None      # dense m x n
    x: Optional[np.ndarray] = None      # low rank: X (m x r)
    w: Optional[np.ndarray] = None      # low rank: W (n x r), block = X W^T

    @property
    def rank(self) -> int:
        if self.kind == KIND_LR:
            return int(self.x.shape[1])
        if self.kind == KIND_DENSE:
            return int(min(self.d.shape))
        return 0

    def dense(self, m: int, n: int) -> np.ndarray:
        if self.kind == KIND_DENSE:
            return self.d
        if self.kind == KIND_LR:
            return self.x @ self.w.T
        return np.zeros((m, n))


ZERO = Block(KIND_ZERO)


class CLR:
    """A CLR matrix: uneven row/column clusters, each block zero, dense or X W^T
    (Section 4.1; the representation is hierarchy-free)."""

    def __init__(self, row_sizes: Sequence[int], col_sizes: Sequence[int]):
        self.row_sizes = [int(s) for s in row_sizes]
        self.col_sizes = [int(s) for s in col_sizes]
        self.row_off = np.concatenate([[0], np.cumsum(self.row_sizes)]).astype(np.int64)
        self.col_off = np.concatenate([[0], np.cumsum(self.col_sizes)]).astype(np.int64)
        self.blocks: Dict[Tuple[int, int], Block] = {}

    @property
    def shape(self) -> Tuple[int, int]:
        return int(self.row_off[-1]), int(self.col_off[-1])

    def get(self, i: int, j: int) -> Block:
        return self.blocks.get((i, j), ZERO)

    def set(self, i: int, j: int, blk: Block) -> None:
        if blk.kind == KIND_ZERO:
            self.blocks.pop((i, j), None)
        else:
            self.blocks[(i, j)] = blk

    def kinds(self) -> np.ndarray:
        k = np.zeros((len(self.row_sizes), len(self.col_sizes)), dtype=np.int32)
        for (i, j), b in self.blocks.items():
            k[i, j] = b.kind
        return k

    def ranks(self) -> np.ndarray:
        r = np.zeros((len(self.row_sizes), len(self.col_sizes)), dtype=np.int32)
        for (i, j), b in self.blocks.items():
            r[i, j] = b.rank
        return r

    def block_dense(self, i: int, j: int) -> np.ndarray:
        return self.get(i, j).dense(self.row_sizes[i], self.col_sizes[j])

    def to_dense(self) -> np.ndarray:
        out = np.zeros(self.shape)
        for (i, j), b in self.blocks.items():
            out[self.row_off[i]:self.row_off[i + 1], self.col_off[j]:self.col_off[j + 1]] = \
                b.dense(self.row_sizes[i], self.col_sizes[j])
        return out


# ----------------------------------------------------------------------------------------------
# Block compression (Section 4.1)
# ----------------------------------------------------------------------------------------------

def dense_rank_limit(m: int, n: int) -> int:
    """Largest rank kept in low-rank form: a block whose rank is greater than half of full
    rank is stored dense (Section 4.1); 'greater than half' read as r > floor(min(m,n)/2)."""
    return min(m, n) // 2


def truncation_rank(s: np.ndarray, eps: float) -> int:
    """Smallest r with sqrt(sum_{i >= r} s_i^2) <= eps for singular values s sorted in
    descending order: the rank at which the Frobenius error of the truncated SVD first drops
    to eps (the error criterion of Section 4.1)."""
    s = np.asarray(s, dtype=np.float64)
    for r in range(len(s) + 1):
        if math.sqrt(float(np.sum(s[r:] ** 2))) <= eps:
            return r
    return len(s)


def compress_block(m_blk: np.ndarray, eps: float, drop_norm: float = 0.0) -> Block:
    """Compress one block: drop it if ||M||_F < drop_norm; otherwise truncate its SVD at
    Frobenius error eps and keep X = U_r S_r, W = V_r (singular values on the left factor),
    or keep it dense when r > floor(min(m,n)/2).  A rank-0 result is a zero block."""
    m, n = m_blk.shape
    if m == 0 or n == 0:
        return ZERO
    if float(np.linalg.norm(m_blk)) < drop_norm:
        return ZERO
    u, s, vt = np.linalg.svd(m_blk, full_matrices=False)
    r = truncation_rank(s, eps)
    if r == 0:
        return ZERO
    if r > dense_rank_limit(m, n):
        return Block(KIND_DENSE, d=np.array(m_blk, dtype=np.float64, copy=True))
    return Block(KIND_LR, x=u[:, :r] * s[:r], w=vt[:r].T.copy())


def compress_block_rrqr(m_blk: np.ndarray, eps: float, drop_norm: float = 0.0) -> Block:
    """Compress one block the way Section 4.1 builds X and W: a rank-revealing QR with column
    pivoting (Businger-Golub: at every step the remaining column of largest norm), M P = Q R,
    truncated at the smallest r whose trailing block has ||R_22||_F <= eps (the Frobenius error
    of X W^T, since Q is orthogonal); X = Q_r, W = P R_r^T.  Dense when r > floor(min(m,n)/2),
    zero when r = 0 or ||M||_F < drop_norm.  Written out step by step (no LAPACK pivoting), so
    the pivot order is the definition's."""
    m, n = m_blk.shape
    if m == 0 or n == 0:
        return ZERO
    if float(np.linalg.norm(m_blk)) < drop_norm:
        return ZERO
    a = np.array(m_blk, dtype=np.float64, copy=True)
    perm = np.arange(n)
    q = np.eye(m)
    k = min(m, n)
    r = k
    for j in range(k):
        tail = a[j:, j:]
        if math.sqrt(float(np.sum(tail * tail))) <= eps:
            r = j
            break
        norms = np.sum(a[j:, j:] ** 2, axis=0)
        c = j + int(np.argmax(norms))          # first maximum
        a[:, [j, c]] = a[:, [c, j]]
        perm[[j, c]] = perm[[c, j]]
        x = a[j:, j]
        alpha = -math.copysign(float(np.linalg.norm(x)), float(x[0]) if x[0] != 0 else 1.0)
        v = x.copy()
        v[0] -= alpha
        vn = float(v @ v)
        if vn > 0.0:
            h = np.eye(m - j) - 2.0 * np.outer(v, v) / vn
            a[j:, :] = h @ a[j:, :]
            q[:, j:] = q[:, j:] @ h
    if r == 0:
        return ZERO
    if r > dense_rank_limit(m, n):
        return Block(KIND_DENSE, d=np.array(m_blk, dtype=np.float64, copy=True))
    w = np.zeros((n, r))
    w[perm, :] = np.triu(a[:r, :]).T
    return Block(KIND_LR, x=q[:, :r].copy(), w=w)


def build(dense: np.ndarray, row_sizes: Sequence[int], col_sizes: Sequence[int], eps: float,
          drop_norm: float = 0.0, rrqr: bool = False) -> CLR:
    """CLR form of a dense matrix: every block compressed with ``compress_block`` (truncated
    SVD, the minimal rank) or, with ``rrqr``, ``compress_block_rrqr`` (the paper's
    rank-revealing QR)."""
    out = CLR(row_sizes, col_sizes)
    comp = compress_block_rrqr if rrqr else compress_block
    for i in range(len(out.row_sizes)):
        for j in range(len(out.col_sizes)):
            blk = dense[out.row_off[i]:out.row_off[i + 1], out.col_off[j]:out.col_off[j + 1]]
            out.set(i, j, comp(blk, eps, drop_norm))
    return out


def from_blocks(row_sizes, col_sizes, spec) -> CLR:
    """CLR from an explicit block list spec[i][j] = (kind, payload) (payload: dense array for
    kind 1, (X, W) for kind 2).  No compression is applied."""
    out = CLR(row_sizes, col_sizes)
    for i, row in enumerate(spec):
        for j, (kind, payload) in enumerate(row):
            if kind == KIND_DENSE:
                out.set(i, j, Block(KIND_DENSE, d=np.asarray(payload, dtype=np.float64)))
            elif kind == KIND_LR:
                x, w = payload
                out.set(i, j, Block(KIND_LR, x=np.asarray(x, np.float64),
                                    w=np.asarray(w, np.float64)))
    return out


def block_norm(b: Block) -> float:
    """Frobenius norm of a block (of its reconstruction for low-rank blocks)."""
    if b.kind == KIND_DENSE:
        return float(np.linalg.norm(b.d))
    if b.kind == KIND_LR:
        return float(np.linalg.norm(b.x @ b.w.T))
    return 0.0


def identity(sizes: Sequence[int]) -> CLR:
    out = CLR(sizes, sizes)
    for i, s in enumerate(out.row_sizes):
        out.set(i, i, Block(KIND_DENSE, d=np.eye(s)))
    return out


def scale(a: CLR, alpha: float) -> CLR:
    """alpha * A, exact: the dense block or the X factor is scaled."""
    out = CLR(a.row_sizes, a.col_sizes)
    for (i, j), b in a.blocks.items():
        if b.kind == KIND_DENSE:
            out.set(i, j, Block(KIND_DENSE, d=alpha * b.d))
        else:
            out.set(i, j, Block(KIND_LR, x=alpha * b.x, w=b.w.copy()))
    return out


def transpose(a: CLR) -> CLR:
    out = CLR(a.col_sizes, a.row_sizes)
    for (i, j), b in a.blocks.items():
        if b.kind == KIND_DENSE:
            out.set(j, i, Block(KIND_DENSE, d=b.d.T.copy()))
        else:
            out.set(j, i, Block(KIND_LR, x=b.w.copy(), w=b.x.copy()))
    return out


# ----------------------------------------------------------------------------------------------
# The product's work list (the tile triples) and the product itself
# ----------------------------------------------------------------------------------------------

def lr_output_rank(r_a: int, r_b: int) -> Tuple[int, int]:
    """Low-rank x low-rank (Section 4.1, Eq. 1): Z = W_A^T X_B is r_A x r_B; it is contracted
    with X_A (giving rank r_B) or with W_B (giving rank r_A), whichever minimises the output
    rank; on a tie, with X_A (the form the paper writes).  Returns (output rank, side) with
    side 0 = contract with X_A, 1 = contract with W_B."""
    if r_b <= r_a:
        return r_b, 0
    return r_a, 1


def triple_flops(kind: int, m: int, k: int, n: int, r_a: int, r_b: int) -> int:
    """Algorithmic flops of one tile product, counted in the form the method computes it."""
    if kind == T_DD:
        return 2 * m * k * n
    if kind == T_DL:
        return 2 * m * k * r_b
    if kind == T_LD:
        return 2 * k * n * r_a
    _, side = lr_output_rank(r_a, r_b)
    return 2 * k * r_a * r_b + (2 * m * r_a * r_b if side == 0 else 2 * n * r_a * r_b)


def triple_out_rank(kind: int, r_a: int, r_b: int) -> int:
    """Rank of the low-rank form of one tile product (0 for dense x dense)."""
    if kind == T_DD:
        return 0
    if kind == T_DL:
        return r_b
    if kind == T_LD:
        return r_a
    return lr_output_rank(r_a, r_b)[0]


@dataclasses.dataclass
class TripleList:
    triples: np.ndarray        # int64 (n, 4): I, J, K, kind; sorted by (I, J) then K
    flops: np.ndarray          # int64 (n,)
    tile_mode: np.ndarray      # int32 (n_I, n_J): MODE_ZERO / MODE_DENSE / MODE_LR
    tile_rank_sum: np.ndarray  # int64 (n_I, n_J): sum of low-rank output ranks per tile
    tile_count: np.ndarray     # int32 (n_I, n_J): triples per tile


def screen_pass(a: CLR, b: CLR, i: int, j: int, eps_sp: float) -> bool:
    """Screening of C_IJ (Section 4.1): the Frobenius-norm estimate of C_IJ is the
    triangle-inequality/submultiplicativity bound sum_K ||A_IK||_F ||B_KJ||_F, and the block
    is computed only if the estimate exceeds eps_sp * area(C_IJ).  With eps_sp = 0 every tile
    with a nonzero contribution passes."""
    if eps_sp <= 0.0:
        return True
    est = 0.0
    for kk in range(len(a.col_sizes)):
        ba, bb = a.get(i, kk), b.get(kk, j)
        if ba.kind != KIND_ZERO and bb.kind != KIND_ZERO:
            est += block_norm(ba) * block_norm(bb)
    return est > eps_sp * a.row_sizes[i] * b.col_sizes[j]


def triple_list(a: CLR, b: CLR, eps_sp: float = 0.0) -> TripleList:
    """All (I, J, K) with A_IK and B_KJ both nonzero in tiles that pass the screen, sorted by
    C tile then K, with their kinds and flops; per tile the accumulation mode (dense when any
    dense x dense contribution is present) and the summed rank of the low-rank products."""
    if a.col_sizes != b.row_sizes:
        raise ValueError("inner tilings differ")
    ni, nk, nj = len(a.row_sizes), len(a.col_sizes), len(b.col_sizes)
    rows, fl = [], []
    mode = np.zeros((ni, nj), np.int32)
    rsum = np.zeros((ni, nj), np.int64)
    cnt = np.zeros((ni, nj), np.int32)
    for i in range(ni):
        for j in range(nj):
            if not screen_pass(a, b, i, j, eps_sp):
                continue
            for kk in range(nk):
                ba, bb = a.get(i, kk), b.get(kk, j)
                if ba.kind == KIND_ZERO or bb.kind == KIND_ZERO:
                    continue
                kind = (0 if ba.kind == KIND_DENSE else 2) + (0 if bb.kind == KIND_DENSE else 1)
                m, k, n = a.row_sizes[i], a.col_sizes[kk], b.col_sizes[j]
                rows.append((i, j, kk, kind))
                fl.append(triple_flops(kind, m, k, n, ba.rank, bb.rank))
                cnt[i, j] += 1
                if kind == T_DD:
                    mode[i, j] = MODE_DENSE
                else:
                    rsum[i, j] += triple_out_rank(kind, ba.rank, bb.rank)
                    if mode[i, j] == MODE_ZERO:
                        mode[i, j] = MODE_LR
    tri = np.array(rows, dtype=np.int64).reshape(-1, 4)
    return TripleList(tri, np.array(fl, dtype=np.int64), mode, rsum, cnt)


def multiply(a: CLR, b: CLR, eps: float, eps_sp: float = 0.0,
             recompress_dense: bool = False) -> CLR:
    """C = A B in CLR form (definition of the screened, recompressed block product).

    For each C tile that passes the screen, the FP64 sum of the reconstructed tile products is
    formed; a tile with a dense x dense contribution stays dense (unless
    ``recompress_dense``), every other tile is truncated with ``compress_block`` at eps (no
    drop threshold)."""
    tl = triple_list(a, b, eps_sp)
    out = CLR(a.row_sizes, b.col_sizes)
    acc: Dict[Tuple[int, int], np.ndarray] = {}
    for i, j, kk, _ in tl.triples:
        i, j, kk = int(i), int(j), int(kk)
        prod = a.block_dense(i, kk) @ b.block_dense(kk, j)
        acc[(i, j)] = acc[(i, j)] + prod if (i, j) in acc else prod
    for (i, j), s in acc.items():
        if tl.tile_mode[i, j] == MODE_DENSE and not recompress_dense:
            out.set(i, j, Block(KIND_DENSE, d=s))
        else:
            out.set(i, j, compress_block(s, eps, 0.0))
    return out


def lincomb(a_coef: float, x: CLR, b_coef: float, y: CLR, diag: float, eps: float,
            recompress_dense: bool = False) -> CLR:
    """a X + b Y + diag I, block by block (low-rank addition, Eq. lr_addition, then
    recompression).  Rules: a block present in one operand only is scaled exactly; a block
    with a dense operand, or a diagonal block when diag != 0, is summed densely (and re-tested
    for low rank only with ``recompress_dense``); two low-rank blocks are concatenated and
    recompressed at eps."""
    if x.row_sizes != y.row_sizes or x.col_sizes != y.col_sizes:
        raise ValueError("tilings differ")
    out = CLR(x.row_sizes, x.col_sizes)
    for i in range(len(x.row_sizes)):
        for j in range(len(x.col_sizes)):
            bx, by = x.get(i, j), y.get(i, j)
            shift = diag if (i == j and diag != 0.0) else 0.0
            m, n = x.row_sizes[i], x.col_sizes[j]
            if bx.kind == KIND_ZERO and by.kind == KIND_ZERO and shift == 0.0:
                continue
            if shift == 0.0 and (bx.kind == KIND_ZERO or by.kind == KIND_ZERO):
                src, c = (by, b_coef) if bx.kind == KIND_ZERO else (bx, a_coef)
                if c == 0.0:
                    continue
                if src.kind == KIND_DENSE:
                    out.set(i, j, Block(KIND_DENSE, d=c * src.d))
                else:
                    out.set(i, j, Block(KIND_LR, x=c * src.x, w=src.w.copy()))
                continue
            s = a_coef * bx.dense(m, n) + b_coef * by.dense(m, n)
            if shift != 0.0:
                s = s + shift * np.eye(m, n)
            if (bx.kind == KIND_DENSE or by.kind == KIND_DENSE or shift != 0.0) and \
                    not recompress_dense:
                out.set(i, j, Block(KIND_DENSE, d=s))
            else:
                out.set(i, j, compress_block(s, eps, 0.0))
    return out


def matvec(a: CLR, v: np.ndarray) -> np.ndarray:
    return a.to_dense() @ v


# ----------------------------------------------------------------------------------------------
# Newton–Schulz S^-1/2 (Section 4.2)
# ----------------------------------------------------------------------------------------------

POWER_STEPS = 30
ALPHA_MARGIN = 1.01


def alpha_estimate(s_dense: np.ndarray, steps: int = POWER_STEPS) -> float:
    """alpha = 1 / (1.01 * lambda), lambda the Rayleigh quotient after ``steps`` power
    iterations from the normalised all-ones vector (reading of Section 4.2, which only asks
    for ||alpha M - I||_2 <= 1)."""
    n = s_dense.shape[0]
    v = np.full(n, 1.0 / math.sqrt(n))
    for _ in range(steps):
        w = s_dense @ v
        v = w / np.linalg.norm(w)
    lam = float(v @ (s_dense @ v))
    return 1.0 / (ALPHA_MARGIN * lam)


def ns_poly(x: np.ndarray) -> np.ndarray:
    """T = (15 I - 10 X + 3 X^2) / 8 (Section 4.2)."""
    n = x.shape[0]
    return (15.0 * np.eye(n) - 10.0 * x + 3.0 * (x @ x)) / 8.0


@dataclasses.dataclass
class NSResult:
    inv_sqrt: np.ndarray         # sqrt(alpha) Z (dense)
    alpha: float
    iters: int                   # number of Z updates applied
    proxy: List[float]           # ||X_n - I||_F / sqrt(N) per iteration
    converged: bool
    tape: List[Tuple[np.ndarray, np.ndarray]]  # (Y_n, Z_n) before each update


def ns_dense(s: np.ndarray, alpha: float, max_iter: int, tol: float = 0.0,
             keep_tape: bool = False) -> NSResult:
    """The Newton–Schulz recurrences of Section 4.2 in dense FP64.  Stops when
    ||X_n - I||_F / sqrt(N) <= tol (X_n is computed each iteration anyway), or after
    ``max_iter`` updates; with tol = 0 exactly ``max_iter`` updates are applied."""
    n = s.shape[0]
    eye = np.eye(n)
    y, z = s.copy(), eye.copy()
    proxy, tape = [], []
    it = 0
    converged = False
    while True:
        x = alpha * (y @ z)
        p = float(np.linalg.norm(x - eye) / math.sqrt(n))
        proxy.append(p)
        if tol > 0.0 and p <= tol:
            converged = True
            break
        if it >= max_iter:
            break
        t = (15.0 * eye - 10.0 * x + 3.0 * (x @ x)) / 8.0
        if keep_tape:
            tape.append((y.copy(), z.copy()))
        z, y = z @ t, t @ y
        it += 1
    return NSResult(math.sqrt(alpha) * z, alpha, it, proxy, converged or tol == 0.0, tape)


@dataclasses.dataclass
class NSClrResult:
    z: CLR                        # sqrt(alpha) Z in CLR form
    alpha: float
    iters: int
    proxy: List[float]
    converged: bool
    # intermediates of iteration `snapshot_iter` (1-based): X_k = alpha Y_{k-1} Z_{k-1}, T_k,
    # Y_k = T_k Y_{k-1}, Z_k = Z_{k-1} T_k (Z unscaled); empty when not requested or not reached
    snapshot: Dict[str, CLR] = dataclasses.field(default_factory=dict)


def ns_clr(s: CLR, alpha: float, eps: float, max_iter: int, tol: float = 0.0,
           eps_sp: float = 0.0, recompress_dense: bool = False,
           snapshot_iter: int = 0) -> NSClrResult:
    """Newton–Schulz with every product a CLR product truncated at eps and T formed by the
    CLR linear combination; X_n = alpha (Y_n Z_n) is truncated before it is scaled.  With
    snapshot_iter = k > 0 the X, T, Y, Z of the k-th iteration are returned as well (the
    intermediates whose block ranks Section 5 shows for the 5th iteration)."""
    n = s.shape[0]
    sizes = s.row_sizes
    y, z = s, identity(sizes)
    proxy: List[float] = []
    snap: Dict[str, CLR] = {}
    it = 0
    converged = False
    while True:
        x = scale(multiply(y, z, eps, eps_sp, recompress_dense), alpha)
        p = float(np.linalg.norm(x.to_dense() - np.eye(n)) / math.sqrt(n))
        proxy.append(p)
        if tol > 0.0 and p <= tol:
            converged = True
            break
        if it >= max_iter:
            break
        x2 = multiply(x, x, eps, eps_sp, recompress_dense)
        t = lincomb(-10.0 / 8.0, x, 3.0 / 8.0, x2, 15.0 / 8.0, eps, recompress_dense)
        z, y = (multiply(z, t, eps, eps_sp, recompress_dense),
                multiply(t, y, eps, eps_sp, recompress_dense))
        it += 1
        if it == snapshot_iter:
            snap = {"X": x, "T": t, "Y": y, "Z": z}
    return NSClrResult(scale(z, math.sqrt(alpha)), alpha, it, proxy, converged or tol == 0.0,
                       snap)


def rank_histogram(m: CLR, max_cluster: int = 256) -> np.ndarray:
    """Block-rank histogram (Section 5's distribution of block ranks): entry 0 counts zero
    blocks, entry r (1 <= r <= max_cluster/2) low-rank blocks of rank r, and the last entry
    dense blocks (full rank)."""
    h = np.zeros(max_cluster // 2 + 2, dtype=np.int64)
    k, r = m.kinds(), m.ranks()
    h[0] = int(np.sum(k == KIND_ZERO))
    h[-1] = int(np.sum(k == KIND_DENSE))
    lr = r[k == KIND_LR]
    np.add.at(h, lr, 1)
    return h


def residual(s_dense: np.ndarray, z_scaled: np.ndarray) -> float:
    """||Z' S Z' - I||_F / sqrt(N) with Z' = sqrt(alpha) Z, i.e. ||alpha Z S Z - I||_F/sqrt(N):
    the RMS error of the eigenvalues of Z' S Z' (reading: the norm is not stated)."""
    n = s_dense.shape[0]
    return float(np.linalg.norm(z_scaled @ s_dense @ z_scaled - np.eye(n)) / math.sqrt(n))


def inv_sqrt_eigh(s: np.ndarray) -> np.ndarray:
    """Closed form S^-1/2 = Q diag(lambda^-1/2) Q^T of a symmetric positive definite S."""
    lam, q = np.linalg.eigh(s)
    return (q * lam ** -0.5) @ q.T


# ----------------------------------------------------------------------------------------------
# Gradient of L = trace(W S^-1/2)
# ----------------------------------------------------------------------------------------------

def grad_trace_inv_sqrt(s: np.ndarray, w: np.ndarray, rel_gap: float = 1e-12) -> np.ndarray:
    """dL/dS for L = trace(W S^-1/2), S symmetric positive definite: with S = Q diag(l) Q^T
    and W~ = Q^T W^T Q, dL/dS = Q (W~ o G) Q^T where G_ij = (l_i^-1/2 - l_j^-1/2)/(l_i - l_j)
    and G_ii = -1/2 l_i^-3/2 (Daleckii–Krein); the derivative at the mean eigenvalue is used
    when |l_i - l_j| < rel_gap * max(l)."""
    lam, q = np.linalg.eigh(s)
    f = lam ** -0.5
    li, lj = lam[:, None], lam[None, :]
    diff = li - lj
    near = np.abs(diff) < rel_gap * float(np.max(np.abs(lam)))
    safe = np.where(near, 1.0, diff)
    gam = np.where(near, -0.5 * (0.5 * (li + lj)) ** -1.5, (f[:, None] - f[None, :]) / safe)
    wt = q.T @ w.T @ q
    return q @ (wt * gam) @ q.T


def ns_adjoint_dense(s: np.ndarray, w: np.ndarray, alpha: float, n_iter: int) -> np.ndarray:
    """dL/dS for L = trace(W sqrt(alpha) Z_n) after exactly ``n_iter`` Newton–Schulz updates,
    by running the recurrences of Section 4.2 backwards with alpha held constant:
      Z_{n+1} = Z_n T_n      -> Zb_n  = Zb_{n+1} T_n^T,        Tb_n  = Z_n^T Zb_{n+1}
      Y_{n+1} = T_n Y_n      -> Yb_n  = T_n^T Yb_{n+1},        Tb_n += Yb_{n+1} Y_n^T
      T_n = (15I-10X+3X^2)/8 -> Xb_n  = (-10 Tb_n + 3 (Tb_n X_n^T + X_n^T Tb_n)) / 8
      X_n = alpha Y_n Z_n    -> Yb_n += alpha Xb_n Z_n^T,      Zb_n += alpha Y_n^T Xb_n
    with Zb_final = sqrt(alpha) W^T, Yb_final = 0 and dL/dS = Yb_0 (Y_0 = S)."""
    res = ns_dense(s, alpha, n_iter, 0.0, keep_tape=True)
    zb = math.sqrt(alpha) * w.T
    yb = np.zeros_like(s)
    n = s.shape[0]
    eye = np.eye(n)
    for y_n, z_n in reversed(res.tape):
        x = alpha * (y_n @ z_n)
        t = (15.0 * eye - 10.0 * x + 3.0 * (x @ x)) / 8.0
        tb = z_n.T @ zb + yb @ y_n.T
        zb_n = zb @ t.T
        yb_n = t.T @ yb
        xb = (-10.0 * tb + 3.0 * (tb @ x.T + x.T @ tb)) / 8.0
        yb_n = yb_n + alpha * (xb @ z_n.T)
        zb_n = zb_n + alpha * (y_n.T @ xb)
        zb, yb = zb_n, yb_n
    return yb


# ----------------------------------------------------------------------------------------------
# Error measures used by the parity tests
# ----------------------------------------------------------------------------------------------

def product_tolerance(a_dense: np.ndarray, b_dense: np.ndarray, eps: float) -> float:
    """Product tolerance 10 * eps * ||A||_F ||B||_F (absolute Frobenius)."""
    return 10.0 * eps * float(np.linalg.norm(a_dense)) * float(np.linalg.norm(b_dense))


def frob_err(x: np.ndarray, y: np.ndarray) -> float:
    return float(np.linalg.norm(x - y))
