// Split-precision staging: the dense blocks of an operand are written as bf16 term panels for
// the tensor-core products (the FP64 value a is split as a = a_0 + a_1 (+ a_2) + residual with
// a_0 = bf16(a), a_1 = bf16(a - a_0), a_2 = bf16(a - a_0 - a_1); every difference is exact in
// FP64).  The dense pass writes dense blocks and zeros elsewhere; a second pass writes each
// low-rank block as its reconstruction X W^T, so a dense GEMM over the panels computes the whole
// sum sum_K A_IK B_KJ of the C tiles it serves (route DENSE or DACC_G), while low-rank C tiles
// (route QR) keep the factorised products of Section 4.1.
//
// Panel layout (K-major for the MMA): for A, panel[t][i][k] = A(i, k), rows_pad x cols_pad;
// for B, panel[t][j][k] = B(k, j).  Padding is zero.
#include <cuda_bf16.h>

#include "clr_internal.h"
#include "split_bf16.cuh"

namespace clr {

using split::split_bf16;
using split::split_bf16_pair;

// A panel: one CTA converts a 32 (rows) x 128 (k) tile.  The source block-row panels are
// column-major (consecutive rows contiguous), the panel is row-major (consecutive k
// contiguous), so the tile goes through shared memory; each thread then packs 4 consecutive
// k of one row into one 8-byte store per term.
constexpr int kTk = 128;

template <int TERMS>
__global__ void __launch_bounds__(256) split_stage_a_kernel(MatView M, const int* row_idx,
                                                            const int* col_idx,
                                                            unsigned short* panels,
                                                            int64_t rows_pad, int64_t cols_pad) {
  __shared__ double tile[32][kTk + 1];
  __shared__ int s_col[kTk];  // column cluster of each of the tile's k (-1 past the end)
  const int64_t tiles_r = rows_pad / 32;
  const int64_t r0 = (int64_t)(blockIdx.x % tiles_r) * 32;
  const int64_t k0 = (int64_t)(blockIdx.x / tiles_r) * kTk;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  const int64_t r = r0 + tx;
  int R = 0, mR = 1;
  int64_t rbase = 0;
  const bool rin = r < M.n_rows;
  if (rin) {
    R = row_idx[r];
    mR = M.row_off[R + 1] - M.row_off[R];
    rbase = (int64_t)M.row_off[R] * M.n_cols + (r - M.row_off[R]);
  }
  const int* kind_row = M.kind + (int64_t)R * M.nc;
  if (threadIdx.x < kTk) s_col[threadIdx.x] = k0 + threadIdx.x < M.n_cols ? col_idx[k0 + threadIdx.x] : -1;
  __syncthreads();
  // all 16 loads of the thread are issued before the first is used
  double v[kTk / 8];
#pragma unroll
  for (int i = 0; i < kTk / 8; ++i) {
    const int cc = ty + 8 * i;
    const int C = s_col[cc];
    v[i] = rin && C >= 0 && kind_row[C] == CLR_KIND_DENSE ? M.pool[rbase + (k0 + cc) * mR] : 0.0;
  }
#pragma unroll
  for (int i = 0; i < kTk / 8; ++i) tile[tx][ty + 8 * i] = v[i];
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = r0 + rr;
    const int64_t k = k0 + 4 * tx;
    unsigned long long packed[TERMS];
#pragma unroll
    for (int t = 0; t < TERMS; ++t) packed[t] = 0;
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      unsigned b[TERMS];
      split_bf16_pair<TERMS>(tile[rr][4 * tx + q], tile[rr][4 * tx + q + 1], b);
#pragma unroll
      for (int t = 0; t < TERMS; ++t) packed[t] |= (unsigned long long)b[t] << (16 * q);
    }
#pragma unroll
    for (int t = 0; t < TERMS; ++t)
      *reinterpret_cast<unsigned long long*>(panels + t * plane + i * cols_pad + k) = packed[t];
  }
}

// B panel: panel[j][k] = B(k, j).  Consecutive k are contiguous in both the source block-row
// panels and the panel, so no transpose: each thread converts 4 consecutive k of one column.
template <int TERMS>
__global__ void __launch_bounds__(256) split_stage_b_kernel(MatView M, const int* row_idx,
                                                            const int* col_idx,
                                                            unsigned short* panels,
                                                            int64_t rows_pad, int64_t cols_pad) {
  // grid: x = panel row j (a column of B), y = 1024-wide chunk of k; 4 consecutive k per thread
  const int64_t j = blockIdx.x;
  const int64_t k = ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * 4;
  if (k >= cols_pad) return;
  // the 4 values first (zeros outside dense blocks), then one split path for all of them: a
  // second split path for groups that straddle a block boundary made every group slower
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < M.n_cols && k < M.n_rows) {
    const int Cc = col_idx[j];
    const int R0 = row_idx[k];
    const int end0 = M.row_off[R0 + 1];
    if (k + 3 < end0) {
      // the 4 elements lie in one block: one kind lookup, contiguous source
      if (M.kind[R0 * M.nc + Cc] == CLR_KIND_DENSE) {
        const int mR = end0 - M.row_off[R0];
        const double* src = M.pool + (int64_t)M.row_off[R0] * M.n_cols + (k - M.row_off[R0]) + j * mR;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = src[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = k + q;
        if (kk < M.n_rows) {
          const int R = row_idx[kk];
          if (M.kind[R * M.nc + Cc] == CLR_KIND_DENSE) {
            const int mR = M.row_off[R + 1] - M.row_off[R];
            v[q] = M.pool[(int64_t)M.row_off[R] * M.n_cols + (kk - M.row_off[R]) + j * mR];
          }
        }
      }
    }
  }
  unsigned long long packed[TERMS];
#pragma unroll
  for (int t = 0; t < TERMS; ++t) packed[t] = 0;
#pragma unroll
  for (int q = 0; q < 4; q += 2) {
    unsigned b[TERMS];
    split_bf16_pair<TERMS>(v[q], v[q + 1], b);
#pragma unroll
    for (int t = 0; t < TERMS; ++t) packed[t] |= (unsigned long long)b[t] << (16 * q);
  }
  const int64_t plane = rows_pad * cols_pad;
#pragma unroll
  for (int t = 0; t < TERMS; ++t)
    *reinterpret_cast<unsigned long long*>(panels + t * plane + j * cols_pad + k) = packed[t];
}

// Low-rank blocks into the panels: one CTA per block of M (blocks of another kind return at
// once), entry (i, j) = sum_t X(i, t) W(j, t) in FP64, then split as the dense pass does.
// a_mode: panel[t][row][k] = A(row, k); else panel[t][col][k] = B(k, col).
template <int TERMS>
__global__ void __launch_bounds__(256) split_stage_lr_kernel(MatView M, unsigned short* panels,
                                                             int64_t rows_pad, int64_t cols_pad,
                                                             int a_mode) {
  const int b = blockIdx.x;
  if (M.kind[b] != CLR_KIND_LR) return;
  const int R = b / M.nc, Cc = b % M.nc;
  const int mR = M.row_off[R + 1] - M.row_off[R];
  const int nC = M.col_off[Cc + 1] - M.col_off[Cc];
  const int r = M.rank[b];
  const double* x = M.pool + (int64_t)M.row_off[R] * M.n_cols + (int64_t)mR * M.col_off[Cc];
  const double* w = x + (int64_t)mR * r;
  const int64_t plane = rows_pad * cols_pad;
  for (int e = threadIdx.x; e < mR * nC; e += blockDim.x) {
    const int i = a_mode ? e / nC : e % mR;  // consecutive threads along the panel's k
    const int j = a_mode ? e % nC : e / mR;
    double v = 0.0;
    for (int q = 0; q < r; ++q) v = fma(x[i + (int64_t)q * mR], w[j + (int64_t)q * nC], v);
    unsigned short t[TERMS];
    split_bf16<TERMS>(v, t);
    const int64_t row = M.row_off[R] + i, col = M.col_off[Cc] + j;
    const int64_t off = a_mode ? row * cols_pad + col : col * cols_pad + row;
#pragma unroll
    for (int k = 0; k < TERMS; ++k) panels[k * plane + off] = t[k];
  }
}

void launch_split_stage(const MatView& M, const int* row_idx, const int* col_idx, void* panels,
                        int terms, int64_t rows_pad, int64_t cols_pad, int a_mode,
                        cudaStream_t st) {
  unsigned short* pn = (unsigned short*)panels;
  if (a_mode) {
    const unsigned n = (unsigned)((rows_pad / 32) * (cols_pad / kTk));
    if (terms == 2)
      split_stage_a_kernel<2><<<n, 256, 0, st>>>(M, row_idx, col_idx, pn, rows_pad, cols_pad);
    else
      split_stage_a_kernel<3><<<n, 256, 0, st>>>(M, row_idx, col_idx, pn, rows_pad, cols_pad);
  } else {
    const dim3 n((unsigned)rows_pad, (unsigned)((cols_pad / 4 + 255) / 256));
    if (terms == 2)
      split_stage_b_kernel<2><<<n, 256, 0, st>>>(M, row_idx, col_idx, pn, rows_pad, cols_pad);
    else
      split_stage_b_kernel<3><<<n, 256, 0, st>>>(M, row_idx, col_idx, pn, rows_pad, cols_pad);
  }
  const unsigned nb = (unsigned)(M.nr * M.nc);
  if (terms == 2)
    split_stage_lr_kernel<2><<<nb, 256, 0, st>>>(M, pn, rows_pad, cols_pad, a_mode);
  else
    split_stage_lr_kernel<3><<<nb, 256, 0, st>>>(M, pn, rows_pad, cols_pad, a_mode);
}

// The split of a plain array: one thread per pair of values (the staging kernels' paired
// split), the last value of an odd count alone.
template <int TERMS>
__global__ void split_values_kernel(const double* x, int64_t n, unsigned short* out) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i >= n) return;
  if (i + 1 < n) {
    unsigned b[TERMS];
    split_bf16_pair<TERMS>(x[i], x[i + 1], b);
#pragma unroll
    for (int t = 0; t < TERMS; ++t) {
      out[t * n + i] = (unsigned short)(b[t] & 0xFFFFu);
      out[t * n + i + 1] = (unsigned short)(b[t] >> 16);
    }
  } else {
    unsigned short b[TERMS];
    split_bf16<TERMS>(x[i], b);
#pragma unroll
    for (int t = 0; t < TERMS; ++t) out[t * n + i] = b[t];
  }
}

}  // namespace clr

extern "C" int clr_split_bf16(const double* x, int64_t n, int terms, uint16_t* out,
                              void* stream) {
  if (n < 0 || (terms != 2 && terms != 3) || (n > 0 && (!x || !out))) return CLR_EINVAL;
  if (n == 0) return CLR_OK;
  const int64_t pairs = (n + 1) / 2;
  if ((pairs + 255) / 256 > 0x7fffffff) return CLR_EINVAL;  // beyond one launch's grid
  const unsigned blocks = (unsigned)((pairs + 255) / 256);
  cudaStream_t st = (cudaStream_t)stream;
  if (terms == 2)
    clr::split_values_kernel<2><<<blocks, 256, 0, st>>>(x, n, (unsigned short*)out);
  else
    clr::split_values_kernel<3><<<blocks, 256, 0, st>>>(x, n, (unsigned short*)out);
  return cudaGetLastError() == cudaSuccess ? CLR_OK : CLR_ECUDA;
}
