// Layout conversions between a row-major dense matrix and the block-slot pool, through
// 32 x 32 shared-memory tiles so that both sides are accessed coalesced.  In the pool, the
// block-row panel of block-row R is an m_R x n_cols column-major matrix, so element (r, c)
// of a dense block lives at row_off[R] * n_cols + (r - row_off[R]) + c * m_R.
#include "clr_internal.h"

namespace clr {

__device__ __forceinline__ int64_t panel_index(const MatView& M, int R, int64_t r, int64_t c,
                                               int mR) {
  return (int64_t)M.row_off[R] * M.n_cols + (r - M.row_off[R]) + c * mR;
}

// pool <- row-major src for every block (used when every kept block is dense).
__global__ void __launch_bounds__(256) rowmajor_to_pool_kernel(MatView M, const int* row_idx,
                                                               const double* src, int64_t lds) {
  __shared__ double tile[32][33];
  const int64_t tiles_r = (M.n_rows + 31) / 32;
  const int64_t r0 = (int64_t)(blockIdx.x % tiles_r) * 32;
  const int64_t c0 = (int64_t)(blockIdx.x / tiles_r) * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int rr = ty; rr < 32; rr += 8) {  // coalesced along columns
    const int64_t r = r0 + rr, c = c0 + tx;
    tile[rr][tx] = (r < M.n_rows && c < M.n_cols) ? src[r * lds + c] : 0.0;
  }
  __syncthreads();
  const int64_t r = r0 + tx;
  if (r >= M.n_rows) return;
  const int R = row_idx[r];
  const int mR = M.row_off[R + 1] - M.row_off[R];
  for (int cc = ty; cc < 32; cc += 8) {  // coalesced along rows of a block-row panel
    const int64_t c = c0 + cc;
    if (c < M.n_cols) M.pool[panel_index(M, R, r, c, mR)] = tile[tx][cc];
  }
}

void launch_rowmajor_to_pool(const MatView& M, const int* row_idx, const double* src,
                             int64_t lds, cudaStream_t st) {
  const int64_t n = ((M.n_rows + 31) / 32) * ((M.n_cols + 31) / 32);
  rowmajor_to_pool_kernel<<<(unsigned)n, 256, 0, st>>>(M, row_idx, src, lds);
}

// After rowmajor_to_pool and block norms: keep every block dense unless its norm is below
// drop_norm (or zero); non-finite norms raise the error flag.
__global__ void dense_kinds_kernel(MatView M, double drop_norm, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M.nr * M.nc) return;
  const int I = t / M.nc, J = t % M.nc;
  const int m = M.row_off[I + 1] - M.row_off[I];
  const int n = M.col_off[J + 1] - M.col_off[J];
  const double nrm = M.norm[t];
  if (!isfinite(nrm)) atomicCAS(err, 0, 3);  // an earlier error keeps precedence
  if (!(nrm >= drop_norm) || nrm == 0.0) {
    M.kind[t] = CLR_KIND_ZERO;
    M.rank[t] = 0;
    M.norm[t] = 0.0;
  } else {
    M.kind[t] = CLR_KIND_DENSE;
    M.rank[t] = m < n ? m : n;
  }
}

void launch_dense_kinds(const MatView& M, double drop_norm, int* err, cudaStream_t st) {
  const int n = M.nr * M.nc;
  dense_kinds_kernel<<<(n + 127) / 128, 128, 0, st>>>(M, drop_norm, err);
}

// row-major out <- reconstruction of every block.
__global__ void __launch_bounds__(256) pool_to_rowmajor_kernel(MatView M, const int* row_idx,
                                                               const int* col_idx, double* out,
                                                               int64_t ldo) {
  __shared__ double tile[32][33];
  const int64_t tiles_r = (M.n_rows + 31) / 32;
  const int64_t r0 = (int64_t)(blockIdx.x % tiles_r) * 32;
  const int64_t c0 = (int64_t)(blockIdx.x / tiles_r) * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int64_t r = r0 + tx;
  if (r < M.n_rows) {
    const int R = row_idx[r];
    const int mR = M.row_off[R + 1] - M.row_off[R];
    const int64_t rloc = r - M.row_off[R];
    for (int cc = ty; cc < 32; cc += 8) {
      const int64_t c = c0 + cc;
      double v = 0.0;
      if (c < M.n_cols) {
        const int Cc = col_idx[c];
        const int b = R * M.nc + Cc;
        const int kind = M.kind[b];
        if (kind == CLR_KIND_DENSE) {
          v = M.pool[panel_index(M, R, r, c, mR)];
        } else if (kind == CLR_KIND_LR) {
          const int n = M.col_off[Cc + 1] - M.col_off[Cc];
          const int rk = M.rank[b];
          const double* X = M.pool + slot_of(M, R, Cc, mR);
          const double* W = X + (int64_t)mR * rk;
          const int64_t cloc = c - M.col_off[Cc];
          for (int q = 0; q < rk; ++q) v = fma(X[rloc + (int64_t)q * mR], W[cloc + (int64_t)q * n], v);
        }
      }
      tile[tx][cc] = v;
    }
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t rw = r0 + rr, c = c0 + tx;
    if (rw < M.n_rows && c < M.n_cols) out[rw * ldo + c] = tile[rr][tx];
  }
}

void launch_pool_to_rowmajor(const MatView& M, const int* row_idx, const int* col_idx,
                             double* out, int64_t ldo, cudaStream_t st) {
  const int64_t n = ((M.n_rows + 31) / 32) * ((M.n_cols + 31) / 32);
  pool_to_rowmajor_kernel<<<(unsigned)n, 256, 0, st>>>(M, row_idx, col_idx, out, ldo);
}

}  // namespace clr
