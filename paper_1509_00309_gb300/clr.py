"""Python binding of the CLR C ABI (include/clr.h): argument marshalling only.

Every computation runs in ``libclr_gb300.so``'s CUDA kernels; this module only converts
arguments (torch tensors / numpy arrays to pointers, option structs, status codes to
exceptions).  If the library has not been built, or no sm_103a GPU is present, calls fail
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

CLR_OK, CLR_EINVAL, CLR_ENOMEM, CLR_ENOCONV, CLR_ETIMEOUT, CLR_ECUDA, CLR_ENOTSUP = \
    0, -1, -2, -3, -4, -5, -6
KIND_ZERO, KIND_DENSE, KIND_LR = 0, 1, 2
PREC = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "auto": 3, "ozaki": 4}
PREC_NAME = {v: k for k, v in PREC.items()}
MAX_CLUSTER = 256
NS_MAX_HISTORY = 256


class ClrOpts(C.Structure):
    _fields_ = [("eps_lr", C.c_double), ("eps_sp", C.c_double), ("precision", C.c_int),
                ("recompress_dense", C.c_int), ("ns_max_iter", C.c_int),
                ("ns_tol", C.c_double), ("ns_alpha", C.c_double),
                ("ns_power_steps", C.c_int), ("ns_fp64_tail", C.c_int),
                ("ns_ladder_switch", C.c_double), ("jacobi_max_sweeps", C.c_int),
                ("ns_snapshot_iter", C.c_int), ("build_rrqr", C.c_int),
                ("wait_timeout_us", C.c_int), ("svd_no_prereduce", C.c_int),
                ("reserved", C.c_int * 4)]


class ClrInfo(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("n_row_clusters", C.c_int32),
                ("n_col_clusters", C.c_int32), ("n_blocks", C.c_int64 * 3),
                ("max_rank", C.c_int32), ("sum_rank", C.c_int64),
                ("stored_doubles", C.c_int64), ("frob_norm", C.c_double),
                ("rank_hist", C.c_int32 * (MAX_CLUSTER // 2 + 2))]


class ClrProductStats(C.Structure):
    _fields_ = [("n_triples", C.c_int64 * 4), ("flops", C.c_int64), ("n_tiles", C.c_int64 * 3),
                ("max_rank_sum", C.c_int64), ("precision", C.c_int32),
                ("n_tiles_tensor", C.c_int32)]


class ClrNsStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("alpha", C.c_double),
                ("residual", C.c_double), ("proxy", C.c_double * NS_MAX_HISTORY),
                ("precision_used", C.c_int32 * NS_MAX_HISTORY), ("ms_total", C.c_double),
                ("proxy_met", C.c_int32), ("residual_met", C.c_int32),
                ("ms_residual", C.c_double)]


class ClrProfile(C.Structure):
    _fields_ = [("products", C.c_int64), ("launches", C.c_int64),
                ("dense_launches", C.c_int64), ("dense_tensor_flops", C.c_double),
                ("ms_plan", C.c_double), ("ms_stage", C.c_double), ("ms_dense", C.c_double),
                ("ms_lowrank", C.c_double), ("ms_compress", C.c_double),
                ("ms_finalize", C.c_double), ("svd_blocks", C.c_int64),
                ("svd_sweeps_fp32", C.c_int64), ("svd_sweeps_fp64", C.c_int64),
                ("svd_early_dense", C.c_int64), ("svd_flops_fp64", C.c_double),
                ("svd_flops_fp32", C.c_double), ("svd_prereduced", C.c_int64),
                ("ms_compress_qr", C.c_double), ("ms_compress_dense", C.c_double),
                ("svd_flops_fp64_qr", C.c_double), ("svd_flops_fp32_qr", C.c_double),
                ("svd_path_cycles", C.c_double * 4), ("svd_path_blocks", C.c_int64 * 4),
                ("svd_full_cycles", C.c_double * 7), ("svd_full_blocks", C.c_int64),
                ("svd_full_dense", C.c_int64), ("svd_pre_cycles", C.c_double * 7),
                ("svd_pre_blocks", C.c_int64)]


_VP = C.c_void_p
_SIGNATURES = {
    "clr_strerror": (C.c_char_p, [C.c_int]),
    "clr_last_error": (C.c_char_p, [_VP]),
    "clr_opts_default": (None, [C.POINTER(ClrOpts)]),
    "clr_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(ClrOpts)]),
    "clr_destroy": (C.c_int, [_VP]),
    "clr_set_opts": (C.c_int, [_VP, C.POINTER(ClrOpts)]),
    "clr_get_opts": (C.c_int, [_VP, C.POINTER(ClrOpts)]),
    "clr_mat_create": (C.c_int, [_VP, C.c_int, _VP, C.c_int, _VP, C.POINTER(_VP)]),
    "clr_mat_from_dense": (C.c_int, [_VP, _VP, C.c_int64, C.c_int, C.c_int, _VP, C.c_int, _VP,
                                     C.c_double, C.c_double, _VP, C.POINTER(_VP)]),
    "clr_mat_from_blocks": (C.c_int, [_VP, C.c_int, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP,
                                      C.POINTER(_VP)]),
    "clr_mat_to_dense": (C.c_int, [_VP, _VP, _VP, C.c_int64, C.c_int, _VP]),
    "clr_mat_get_blocks": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "clr_mat_info": (C.c_int, [_VP, _VP, C.POINTER(ClrInfo), _VP]),
    "clr_mat_shape": (C.c_int, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "clr_mat_copy": (C.c_int, [_VP, _VP, _VP, _VP]),
    "clr_mat_transpose": (C.c_int, [_VP, _VP, C.POINTER(_VP), _VP]),
    "clr_mat_free": (C.c_int, [_VP, _VP]),
    "clr_multiply": (C.c_int, [_VP, _VP, _VP, C.POINTER(_VP), _VP]),
    "clr_multiply_into": (C.c_int, [_VP, _VP, _VP, _VP, C.c_double,
                                    C.POINTER(ClrProductStats), _VP]),
    "clr_multiply_batched": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, _VP]),
    "clr_multiply_backward": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(_VP), C.POINTER(_VP),
                                        _VP]),
    "clr_lincomb": (C.c_int, [_VP, C.c_double, _VP, C.c_double, _VP, C.c_double, _VP, _VP]),
    "clr_sqrt_inv": (C.c_int, [_VP, _VP, C.POINTER(_VP), C.POINTER(ClrNsStats),
                               C.POINTER(_VP), _VP]),
    "clr_ns_residual": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_double), _VP]),
    "clr_check": (C.c_int, [_VP, _VP]),
    "clr_sqrt_inv_backward": (C.c_int, [_VP, _VP, _VP, C.POINTER(_VP), _VP]),
    "clr_tape_free": (C.c_int, [_VP, _VP]),
    "clr_ns_snapshot": (C.c_int, [_VP, C.c_int, C.POINTER(_VP)]),
    "clr_matvec": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "clr_block_compress_noalloc": (C.c_int, [C.c_int, _VP, C.c_int64, C.c_int, C.c_int,
                                             C.c_double, C.c_int, _VP, _VP, _VP, _VP, _VP]),
    "clr_batch_create": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.c_int, _VP,
                                   C.POINTER(_VP)]),
    "clr_batch_run": (C.c_int, [_VP, _VP, _VP]),
    "clr_batch_output": (C.c_int, [_VP, C.c_int, C.POINTER(_VP)]),
    "clr_batch_tuning": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    "clr_batch_free": (C.c_int, [_VP, _VP]),
    "clr_autotune_save": (C.c_int, [_VP, C.c_char_p]),
    "clr_autotune_load": (C.c_int, [_VP, C.c_char_p]),
    "clr_autotune_entries": (C.c_int, [_VP]),
    "clr_mem_trim": (C.c_int, [_VP]),
    "clr_mem_cached": (C.c_int64, []),
    "clr_profile_enable": (C.c_int, [_VP, C.c_int]),
    "clr_profile_read": (C.c_int, [_VP, C.POINTER(ClrProfile)]),
    "clr_probe_fp64_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "clr_split_bf16": (C.c_int, [_VP, C.c_int64, C.c_int, _VP, _VP]),
    "clr_multiply_host_stream": (C.c_int, [_VP, _VP, C.c_int64, _VP, C.c_int64, _VP, C.c_int64,
                                           C.c_int, _VP, C.c_int, _VP, C.c_int, _VP, C.c_int,
                                           _VP]),
}

_LIB: Optional[C.CDLL] = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libclr_gb300.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libclr_gb300.so is not built (run "
                               "paper_1509_00309_gb300.build.build()); there is no fallback")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols() -> List[str]:
    return sorted(_SIGNATURES)


class ClrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (load().clr_strerror(status).decode(), status, msg))
        self.status = status


def _i32(seq: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int32))


def _ptr(a) -> int:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Matrix:
    """A CLR matrix handle owned by this object (freed on close/garbage collection)."""

    def __init__(self, ctx: "Context", handle: int, row_sizes, col_sizes):
        self.ctx = ctx
        self.handle = handle
        self.row_sizes = [int(s) for s in row_sizes]
        self.col_sizes = [int(s) for s in col_sizes]

    @property
    def shape(self) -> Tuple[int, int]:
        return sum(self.row_sizes), sum(self.col_sizes)

    def close(self):
        if self.handle:
            load().clr_mat_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def to_dense(self, out=None, stream=None):
        """Reconstruct: into a torch CUDA float64 tensor ``out`` (device path), or to a new
        numpy array when ``out`` is None (host path, synchronises)."""
        n, m = self.shape
        if out is None:
            host = np.empty((n, m), dtype=np.float64)
            self.ctx._check(load().clr_mat_to_dense(self.ctx.handle, self.handle, _ptr(host), m,
                                                    1, _stream(stream)))
            return host
        on_host = isinstance(out, np.ndarray) or not out.is_cuda
        ld = out.shape[1] if isinstance(out, np.ndarray) else out.stride(0)
        self.ctx._check(load().clr_mat_to_dense(self.ctx.handle, self.handle, _ptr(out), ld,
                                                int(on_host), _stream(stream)))
        return out

    def get_blocks(self, pool: bool = True, stream=None):
        nb = len(self.row_sizes) * len(self.col_sizes)
        kinds = np.empty(nb, np.int32)
        ranks = np.empty(nb, np.int32)
        norms = np.empty(nb, np.float64)
        p = np.empty(self.shape[0] * self.shape[1], np.float64) if pool else None
        self.ctx._check(load().clr_mat_get_blocks(self.ctx.handle, self.handle, _ptr(kinds),
                                                  _ptr(ranks), _ptr(norms), _ptr(p),
                                                  _stream(stream)))
        shp = (len(self.row_sizes), len(self.col_sizes))
        return kinds.reshape(shp), ranks.reshape(shp), norms.reshape(shp), p

    def info(self, stream=None) -> Dict:
        inf = ClrInfo()
        self.ctx._check(load().clr_mat_info(self.ctx.handle, self.handle, C.byref(inf),
                                            _stream(stream)))
        return {"n_rows": inf.n_rows, "n_cols": inf.n_cols,
                "n_blocks": list(inf.n_blocks), "max_rank": inf.max_rank,
                "sum_rank": inf.sum_rank, "stored_doubles": inf.stored_doubles,
                "frob_norm": inf.frob_norm, "rank_hist": list(inf.rank_hist)}


class Context:
    """A library context bound to one CUDA device."""

    def __init__(self, device: int = 0, **opts):
        lib = load()
        o = ClrOpts()
        lib.clr_opts_default(C.byref(o))
        for k, v in opts.items():
            if k == "precision" and isinstance(v, str):
                v = PREC[v]
            setattr(o, k, v)
        h = C.c_void_p()
        st = lib.clr_create(C.byref(h), int(device), C.byref(o))
        if st != CLR_OK:
            raise ClrError(st, "clr_create failed: no usable sm_103a device %d" % device)
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            load().clr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != CLR_OK:
            raise ClrError(st, load().clr_last_error(self.handle).decode())

    # options -----------------------------------------------------------------------------
    def get_opts(self) -> ClrOpts:
        o = ClrOpts()
        self._check(load().clr_get_opts(self.handle, C.byref(o)))
        return o

    def set_opts(self, **kw):
        o = self.get_opts()
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PREC[v]
            setattr(o, k, v)
        self._check(load().clr_set_opts(self.handle, C.byref(o)))

    def check(self, stream=None):
        """Synchronise and raise any error a kernel reported since the last synchronising
        call (clr_check)."""
        self._check(load().clr_check(self.handle, _stream(stream)))

    def mem_trim(self):
        self._check(load().clr_mem_trim(self.handle))

    # observability -----------------------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._check(load().clr_profile_enable(self.handle, int(on)))

    def profile_read(self) -> Dict:
        p = ClrProfile()
        self._check(load().clr_profile_read(self.handle, C.byref(p)))
        out = {f: getattr(p, f) for f, _ in ClrProfile._fields_}
        for f in ("svd_path_cycles", "svd_path_blocks", "svd_full_cycles", "svd_pre_cycles"):
            out[f] = list(out[f])
        return out

    # matrices ------------------------------------------------------------------------------
    def zeros(self, row_sizes, col_sizes=None) -> Matrix:
        col_sizes = row_sizes if col_sizes is None else col_sizes
        rs, cs = _i32(row_sizes), _i32(col_sizes)
        h = C.c_void_p()
        self._check(load().clr_mat_create(self.handle, len(rs), _ptr(rs), len(cs), _ptr(cs),
                                          C.byref(h)))
        return Matrix(self, h.value, rs, cs)

    def from_dense(self, a, row_sizes, col_sizes=None, eps_lr: float = 0.0,
                   drop_norm: float = 0.0, stream=None) -> Matrix:
        """``a``: row-major float64 torch CUDA tensor (device path), or a numpy array / torch
        CPU tensor (host path; pinned memory makes the upload fast)."""
        col_sizes = row_sizes if col_sizes is None else col_sizes
        rs, cs = _i32(row_sizes), _i32(col_sizes)
        on_host = isinstance(a, np.ndarray) or (hasattr(a, "is_cuda") and not a.is_cuda)
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float64)
            lda = a.shape[1]
        elif on_host:
            if a.dtype != __import__("torch").float64 or a.stride(1) != 1:
                raise ValueError("host tensor input must be row-major float64")
            lda = a.stride(0)
        else:
            if a.dtype != __import__("torch").float64 or not a.is_cuda or a.stride(1) != 1:
                raise ValueError("device input must be a row-major float64 CUDA tensor")
            lda = a.stride(0)
        h = C.c_void_p()
        self._check(load().clr_mat_from_dense(self.handle, _ptr(a), lda, int(on_host), len(rs),
                                              _ptr(rs), len(cs), _ptr(cs), float(eps_lr),
                                              float(drop_norm), _stream(stream), C.byref(h)))
        return Matrix(self, h.value, rs, cs)

    def from_blocks(self, row_sizes, col_sizes, kinds, ranks, pool, stream=None) -> Matrix:
        rs, cs = _i32(row_sizes), _i32(col_sizes)
        k, r = _i32(np.ravel(kinds)), _i32(np.ravel(ranks))
        p = np.ascontiguousarray(pool, dtype=np.float64)
        h = C.c_void_p()
        self._check(load().clr_mat_from_blocks(self.handle, len(rs), _ptr(rs), len(cs), _ptr(cs),
                                               _ptr(k), _ptr(r), _ptr(p), _stream(stream),
                                               C.byref(h)))
        return Matrix(self, h.value, rs, cs)

    def copy(self, src: Matrix, dst: Matrix, stream=None):
        self._check(load().clr_mat_copy(self.handle, src.handle, dst.handle, _stream(stream)))

    def transpose(self, src: Matrix, stream=None) -> Matrix:
        h = C.c_void_p()
        self._check(load().clr_mat_transpose(self.handle, src.handle, C.byref(h),
                                             _stream(stream)))
        return Matrix(self, h.value, src.col_sizes, src.row_sizes)

    # arithmetic ------------------------------------------------------------------------------
    def multiply(self, a: Matrix, b: Matrix, stream=None) -> Matrix:
        h = C.c_void_p()
        self._check(load().clr_multiply(self.handle, a.handle, b.handle, C.byref(h),
                                        _stream(stream)))
        return Matrix(self, h.value, a.row_sizes, b.col_sizes)

    def multiply_into(self, a: Matrix, b: Matrix, c: Matrix, alpha: float = 1.0,
                      stats: bool = False, stream=None) -> Optional[Dict]:
        s = ClrProductStats() if stats else None
        self._check(load().clr_multiply_into(self.handle, a.handle, b.handle, c.handle,
                                             float(alpha), C.byref(s) if stats else None,
                                             _stream(stream)))
        if not stats:
            return None
        return {"n_triples": list(s.n_triples), "flops": s.flops, "n_tiles": list(s.n_tiles),
                "max_rank_sum": s.max_rank_sum, "precision": PREC_NAME[s.precision],
                "n_tiles_tensor": s.n_tiles_tensor}

    def multiply_backward(self, a: Matrix, b: Matrix, cbar: Matrix, need_a: bool = True,
                          need_b: bool = True, stream=None):
        """Adjoint of C = A B: (cbar B^T, A^T cbar) as CLR matrices (clr_multiply_backward);
        an adjoint not asked for is None."""
        ha, hb = C.c_void_p(), C.c_void_p()
        self._check(load().clr_multiply_backward(self.handle, a.handle, b.handle, cbar.handle,
                                                 C.byref(ha) if need_a else None,
                                                 C.byref(hb) if need_b else None,
                                                 _stream(stream)))
        abar = Matrix(self, ha.value, a.row_sizes, a.col_sizes) if need_a else None
        bbar = Matrix(self, hb.value, b.row_sizes, b.col_sizes) if need_b else None
        return abar, bbar

    def multiply_host_stream(self, a, b, c, row_sizes, inner_sizes=None, col_sizes=None,
                             n_chunks: int = 4, stream=None):
        """C = A B for page-locked host torch tensors (row-major float64), streamed: A in two
        row chunks, B and C in n_chunks column chunks, so that host-device copies in both
        directions overlap the tile products (clr_multiply_host_stream)."""
        inner_sizes = row_sizes if inner_sizes is None else inner_sizes
        col_sizes = inner_sizes if col_sizes is None else col_sizes
        rs, ks, cs = _i32(row_sizes), _i32(inner_sizes), _i32(col_sizes)
        self._check(load().clr_multiply_host_stream(
            self.handle, _ptr(a), a.stride(0), _ptr(b), b.stride(0), _ptr(c), c.stride(0),
            len(rs), _ptr(rs), len(ks), _ptr(ks), len(cs), _ptr(cs), int(n_chunks),
            _stream(stream)))
        return c

    def multiply_batched(self, a: Sequence[Matrix], b: Sequence[Matrix],
                         stream=None) -> List[Matrix]:
        n = len(a)
        ah = (C.c_void_p * n)(*[m.handle for m in a])
        bh = (C.c_void_p * n)(*[m.handle for m in b])
        ch = (C.c_void_p * n)()
        self._check(load().clr_multiply_batched(self.handle, n, ah, bh, ch, _stream(stream)))
        return [Matrix(self, ch[i], a[i].row_sizes, b[i].col_sizes) for i in range(n)]

    def batch(self, a: Sequence[Matrix], b: Sequence[Matrix], eps=None, tune: bool = True,
              stream=None) -> "Batch":
        n = len(a)
        ah = (C.c_void_p * n)(*[m.handle for m in a])
        bh = (C.c_void_p * n)(*[m.handle for m in b])
        ep = None if eps is None else np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        h = C.c_void_p()
        self._check(load().clr_batch_create(self.handle, n, ah, bh, _ptr(ep), int(tune),
                                            _stream(stream), C.byref(h)))
        return Batch(self, h.value, list(a), list(b))

    def autotune_save(self, path: str):
        self._check(load().clr_autotune_save(self.handle, path.encode()))

    def autotune_load(self, path: str):
        self._check(load().clr_autotune_load(self.handle, path.encode()))

    def autotune_entries(self) -> int:
        return load().clr_autotune_entries(self.handle)

    def lincomb(self, a: float, x: Matrix, b: float, y: Matrix, diag: float = 0.0,
                out: Optional[Matrix] = None, stream=None) -> Matrix:
        out = out if out is not None else self.zeros(x.row_sizes, x.col_sizes)
        self._check(load().clr_lincomb(self.handle, float(a), x.handle, float(b), y.handle,
                                       float(diag), out.handle, _stream(stream)))
        return out

    def matvec(self, a: Matrix, x, y, stream=None):
        self._check(load().clr_matvec(self.handle, a.handle, _ptr(x), _ptr(y), _stream(stream)))

    def sqrt_inv(self, s: Matrix, keep_tape: bool = False, stream=None,
                 allow_noconv: bool = False):
        """Z ~ S^-1/2 by Newton–Schulz.  Returns (Z, stats dict, tape handle or None)."""
        z = C.c_void_p()
        st = ClrNsStats()
        tape = C.c_void_p()
        status = load().clr_sqrt_inv(self.handle, s.handle, C.byref(z), C.byref(st),
                                     C.byref(tape) if keep_tape else None, _stream(stream))
        if status != CLR_OK and not (allow_noconv and status == CLR_ENOCONV and z.value):
            self._check(status)
        n = st.iters + 1
        stats = {"iters": st.iters, "converged": bool(st.converged), "alpha": st.alpha,
                 "residual": st.residual, "proxy": list(st.proxy[:n]),
                 "precision_used": [PREC_NAME[p] for p in st.precision_used[:n]],
                 "ms_total": st.ms_total, "proxy_met": bool(st.proxy_met),
                 "residual_met": bool(st.residual_met), "ms_residual": st.ms_residual,
                 "status": status}
        return Matrix(self, z.value, s.row_sizes, s.col_sizes), stats, \
            (Tape(self, tape.value) if keep_tape else None)

    def ns_snapshot(self, which: str, like: Matrix) -> Matrix:
        """The X, T, Y or Z of the NS iteration named by the option ns_snapshot_iter, from
        the last sqrt_inv on this context (ownership passes to the returned Matrix)."""
        h = C.c_void_p()
        self._check(load().clr_ns_snapshot(self.handle, "XTYZ".index(which), C.byref(h)))
        return Matrix(self, h.value, like.row_sizes, like.col_sizes)

    def ns_residual(self, s: Matrix, z: Matrix, stream=None) -> float:
        out = C.c_double()
        self._check(load().clr_ns_residual(self.handle, s.handle, z.handle, C.byref(out),
                                           _stream(stream)))
        return out.value

    def sqrt_inv_backward(self, tape: "Tape", zbar: Matrix, stream=None) -> Matrix:
        h = C.c_void_p()
        self._check(load().clr_sqrt_inv_backward(self.handle, tape.handle, zbar.handle,
                                                 C.byref(h), _stream(stream)))
        return Matrix(self, h.value, zbar.row_sizes, zbar.col_sizes)


def probe_fp64_rate(device: int = 0) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s (clr_probe_fp64_rate)."""
    out = C.c_double()
    st = load().clr_probe_fp64_rate(int(device), C.byref(out))
    if st != CLR_OK:
        raise ClrError(st, "clr_probe_fp64_rate failed")
    return out.value


def split_bf16(x, terms: int, out=None, stream=None):
    """bf16 term split of a contiguous CUDA float64 tensor x (clr_split_bf16): returns a
    (terms, x.numel()) int16 tensor of bf16 bit patterns (term t of element i at [t, i])."""
    import torch
    if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ClrError(CLR_EINVAL, "x must be a contiguous CUDA float64 tensor")
    n = x.numel()
    if out is None:
        out = torch.empty((terms, n), dtype=torch.int16, device=x.device)
    st = load().clr_split_bf16(_ptr(x), n, int(terms), _ptr(out), _stream(stream))
    if st != CLR_OK:
        raise ClrError(st, "clr_split_bf16 failed")
    return out


def block_compress_noalloc(block, eps: float, x_out, w_out, status, sigma_out=None,
                           max_sweeps: int = 40, stream=None) -> None:
    """Truncated SVD of one dense block (a column-major view: a CUDA float64 tensor whose
    transpose is contiguous, or any tensor with stride(0) == 1) into caller-owned device
    buffers, without any device allocation (see clr_block_compress_noalloc in clr.h)."""
    import torch
    m, n = block.shape
    if not block.is_cuda or block.dtype != torch.float64:
        raise ValueError("block must be a CUDA float64 tensor")
    if block.stride(0) != 1:
        raise ValueError("block must be column-major (stride(0) == 1)")
    ld = block.stride(1) if n > 1 else m
    k = min(m, n)
    # the kernel writes m*k, n*k and k doubles and 3 int32: refuse buffers it would overrun
    for name, t, need, dt in (("x_out", x_out, m * k, torch.float64),
                              ("w_out", w_out, n * k, torch.float64),
                              ("sigma_out", sigma_out, k, torch.float64),
                              ("status", status, 3, torch.int32)):
        if t is None and name == "sigma_out":
            continue
        if t is None or not t.is_cuda or t.device != block.device or t.dtype != dt or \
                not t.is_contiguous() or t.numel() < need:
            raise ValueError("%s must be a contiguous %s tensor on %s with at least %d "
                             "elements" % (name, dt, block.device, need))
    st = load().clr_block_compress_noalloc(block.device.index or 0, _ptr(block), ld, m, n,
                                           float(eps), int(max_sweeps), _ptr(x_out),
                                           _ptr(w_out), _ptr(sigma_out), _ptr(status),
                                           _stream(stream))
    if st != CLR_OK:
        raise ClrError(st, "clr_block_compress_noalloc failed")


class Batch:
    """Products captured into one CUDA graph (clr_batch_*); outputs are owned by the batch."""

    def __init__(self, ctx: Context, handle: int, a, b):
        self.ctx = ctx
        self.handle = handle
        self._inputs = (a, b)   # inputs must outlive the batch
        self.n = len(a)

    def run(self, stream=None):
        self.ctx._check(load().clr_batch_run(self.ctx.handle, self.handle, _stream(stream)))

    def output(self, i: int) -> Matrix:
        h = C.c_void_p()
        self.ctx._check(load().clr_batch_output(self.handle, i, C.byref(h)))
        a, b = self._inputs
        m = Matrix(self.ctx, h.value, a[i].row_sizes, b[i].col_sizes)
        m.close = lambda: None    # borrowed: freed with the batch
        return m

    def tuning(self, i: int):
        p, c, br = C.c_int(), C.c_int(), C.c_int()
        self.ctx._check(load().clr_batch_tuning(self.handle, i, C.byref(p), C.byref(c),
                                                C.byref(br)))
        return {"precision": PREC_NAME[p.value], "ctas_per_sm": c.value, "branch": br.value}

    def close(self):
        if self.handle:
            load().clr_batch_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tape:
    def __init__(self, ctx: Context, handle: int):
        self.ctx = ctx
        self.handle = handle

    def close(self):
        if self.handle:
            load().clr_tape_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
