// Split-precision staging: the dense blocks of an operand are written as bf16 term panels for
// the tensor-core products (the FP64 value a is split as a = a_0 + a_1 (+ a_2) + residual with
// a_0 = bf16(a), a_1 = bf16(a - a_0), a_2 = bf16(a - a_0 - a_1); every difference is exact in
// FP64).  Non-dense blocks are written as zeros, so a dense GEMM over the panels computes
// exactly the dense x dense part of the CLR product.
//
// Panel layout (K-major for the MMA): for A, panel[t][i][k] = A(i, k), rows_pad x cols_pad;
// for B, panel[t][j][k] = B(k, j).  Padding is zero.
#include <cuda_bf16.h>

#include "clr_internal.h"

namespace clr {

// Round a double to the nearest bf16 (ties to even), from the format's definition: 8
// significant bits, exponent range of binary32, subnormal spacing 2^-133.
__device__ __forceinline__ unsigned short bf16_bits_rn(double x) {
  if (x == 0.0 || !isfinite(x)) {
    const float f = (float)x;
    return (unsigned short)(__float_as_uint(f) >> 16);
  }
  int e = ilogb(x);
  if (e < -126) e = -126;
  const double r = rint(scalbn(x, 7 - e));
  const float f = (float)scalbn(r, e - 7);
  return (unsigned short)(__float_as_uint(f) >> 16);
}

__device__ __forceinline__ double bf16_bits_to_double(unsigned short b) {
  return (double)__uint_as_float(((unsigned)b) << 16);
}

__device__ __forceinline__ int cluster_of(const int* off, int n, int x) {
  int lo = 0, hi = n - 1;  // off[lo] <= x < off[hi+1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One CTA stages a 32 (matrix rows) x 32 (matrix cols) tile.
__global__ void __launch_bounds__(256) split_stage_kernel(MatView M, unsigned short* panels,
                                                          int terms, int64_t rows_pad,
                                                          int64_t cols_pad, int a_mode) {
  __shared__ double tile[32][33];
  // tile origin in matrix coordinates (r = matrix row, c = matrix col)
  const int64_t prow_tiles = a_mode ? rows_pad / 32 : cols_pad / 32;  // along matrix rows
  const int64_t r0 = (a_mode ? blockIdx.x % prow_tiles : blockIdx.x % prow_tiles) * 32;
  const int64_t c0 = (int64_t)(blockIdx.x / prow_tiles) * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  // load: consecutive threads take consecutive matrix rows (column-major source)
  for (int cc = ty; cc < 32; cc += 8) {
    const int64_t r = r0 + tx, c = c0 + cc;
    double v = 0.0;
    if (r < M.n_rows && c < M.n_cols) {
      const int R = cluster_of(M.row_off, M.nr, (int)r);
      const int Cc = cluster_of(M.col_off, M.nc, (int)c);
      if (M.kind[R * M.nc + Cc] == CLR_KIND_DENSE) {
        const int mR = M.row_off[R + 1] - M.row_off[R];
        v = M.pool[(int64_t)M.row_off[R] * M.n_cols + (r - M.row_off[R]) + c * mR];
      }
    }
    tile[tx][cc] = v;
  }
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  if (a_mode) {
    // panel[i][k] = A(i,k): consecutive threads write consecutive k
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t i = r0 + rr, k = c0 + tx;
      if (i >= rows_pad || k >= cols_pad) continue;
      double rest = tile[rr][tx];
      for (int t = 0; t < terms; ++t) {
        const unsigned short b = bf16_bits_rn(rest);
        panels[t * plane + i * cols_pad + k] = b;
        rest -= bf16_bits_to_double(b);
      }
    }
  } else {
    // panel[j][k] = B(k,j): rows of the panel are matrix columns; consecutive threads write
    // consecutive k (matrix rows)
    for (int cc = ty; cc < 32; cc += 8) {
      const int64_t j = c0 + cc, k = r0 + tx;
      if (j >= rows_pad || k >= cols_pad) continue;
      double rest = tile[tx][cc];
      for (int t = 0; t < terms; ++t) {
        const unsigned short b = bf16_bits_rn(rest);
        panels[t * plane + j * cols_pad + k] = b;
        rest -= bf16_bits_to_double(b);
      }
    }
  }
}

void launch_split_stage(const MatView& M, void* panels, int terms, int64_t rows_pad,
                        int64_t cols_pad, int a_mode, cudaStream_t st) {
  // tiles cover the padded panel: A: rows_pad x cols_pad over (matrix rows, matrix cols);
  // B: panel rows are matrix columns (rows_pad) and panel cols are matrix rows (cols_pad).
  const int64_t along_rows = (a_mode ? rows_pad : cols_pad) / 32;
  const int64_t along_cols = (a_mode ? cols_pad : rows_pad) / 32;
  const int64_t n = along_rows * along_cols;
  split_stage_kernel<<<(unsigned)n, 256, 0, st>>>(M, (unsigned short*)panels, terms, rows_pad,
                                                   cols_pad, a_mode);
}

__global__ void cluster_index_kernel(const int* off, int n_clusters, int* index_of) {
  for (int I = blockIdx.x; I < n_clusters; I += gridDim.x)
    for (int i = off[I] + threadIdx.x; i < off[I + 1]; i += blockDim.x) index_of[i] = I;
}

void launch_cluster_index(const int* off, int n_clusters, int* index_of, int64_t n,
                          cudaStream_t st) {
  (void)n;
  cluster_index_kernel<<<n_clusters, 256, 0, st>>>(off, n_clusters, index_of);
}

}  // namespace clr
