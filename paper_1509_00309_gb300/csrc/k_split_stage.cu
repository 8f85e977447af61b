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

namespace clr {

// Round the value R * 2^s (R a signed integer, |R| < 2^62) to the nearest bf16, ties to
// even, from the format's definition: 8 significant bits, exponent range of binary32, below
// the smallest normal 2^-126 a fixed spacing of 2^-133.  Returns the bf16 bits and, in *Rr,
// the rounded value in units of 2^s (exact), so the caller can form the residual R - Rr.
// Integer operations only: FP64 arithmetic runs at a small fraction of the integer rate.
__device__ __forceinline__ unsigned short round_bf16(long long R, int s, long long* Rr) {
  if (R == 0) {
    *Rr = 0;
    return 0;
  }
  const unsigned short sign = R < 0 ? 0x8000 : 0;
  const unsigned long long mag = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
  const int msb = 63 - __clzll(mag);
  int shift = msb - 7;
  const int sub = -133 - s;
  if (shift < sub) shift = sub;
  unsigned long long q;
  if (shift <= 0) {
    q = mag;  // at most 8 significant bits: exact
    shift = 0;
  } else if (shift > 62) {
    q = 0;
  } else {
    const unsigned long long rem = mag & ((1ull << shift) - 1);
    const unsigned long long half = 1ull << (shift - 1);
    q = mag >> shift;
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  if (q == 0) {
    *Rr = 0;
    return sign;
  }
  const long long rr = (long long)(q << shift);
  *Rr = R < 0 ? -rr : rr;
  const int vexp = s + shift;
  const int qb = 63 - __clzll(q);  // <= 8
  const int E = qb + vexp;         // exponent of the leading bit
  if (E < -126) return sign | (unsigned short)(q << (vexp + 133));  // subnormal
  const unsigned mant = qb >= 7 ? (unsigned)(q >> (qb - 7)) & 0x7Fu
                                : (unsigned)(q << (7 - qb)) & 0x7Fu;
  return sign | (unsigned short)((E + 127) << 7) | (unsigned short)mant;
}

// The same rounding for |R| < 2^46 with 32-bit operations: when R does not fit in 32 bits its 14
// low bits are folded into a sticky bit (round to odd); the rounding position is then at least
// 11 bits above that bit, so round-to-nearest-even is unchanged.
__device__ __forceinline__ unsigned short round_bf16_32(long long R, int s, long long* Rr) {
  if (R == 0) {
    *Rr = 0;
    return 0;
  }
  const unsigned short sign = R < 0 ? 0x8000 : 0;
  const unsigned long long m = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
  int extra = 0;
  unsigned m32;
  if (m >> 32) {
    m32 = (unsigned)(m >> 14) | ((m & 0x3FFFull) ? 1u : 0u);
    extra = 14;
  } else {
    m32 = (unsigned)m;
  }
  const int s2 = s + extra;
  const int msb = 31 - __clz(m32);
  int shift = msb - 7;
  const int sub = -133 - s2;
  if (shift < sub) shift = sub;
  unsigned q;
  if (shift <= 0) {
    q = m32;
    shift = 0;
  } else if (shift >= 32) {
    q = (shift == 32 && m32 > 0x80000000u) ? 1u : 0u;
  } else {
    const unsigned rem = m32 & ((1u << shift) - 1u);
    const unsigned half = 1u << (shift - 1);
    q = m32 >> shift;
    if (rem > half || (rem == half && (q & 1u))) ++q;
  }
  if (q == 0) {
    *Rr = 0;
    return sign;
  }
  const long long rr = (long long)((unsigned long long)q << (shift + extra));
  *Rr = R < 0 ? -rr : rr;
  const int vexp = s2 + shift;
  const int qb = 31 - __clz(q);  // <= 8
  const int E = qb + vexp;
  if (E < -126) return sign | (unsigned short)(q << (vexp + 133));
  const unsigned mant = qb >= 7 ? (q >> (qb - 7)) & 0x7Fu : (q << (7 - qb)) & 0x7Fu;
  return sign | (unsigned short)((E + 127) << 7) | (unsigned short)mant;
}

// a = a_0 + a_1 (+ a_2) + residual: successive round-to-nearest bf16 terms of a finite double.
// Fast path (exponent of a in [-110, 126], so a_0 is a normal bf16): a_0 by adding the
// rounding bias to the FP64 bit pattern and clearing the 45 low bits (carries into the exponent
// are exact), the residual a - a_0 as an integer multiple of a's ulp; the lower terms, and the
// whole split outside that range, by the generic integer rounding above.
template <int TERMS>
__device__ __forceinline__ void split_bf16(double x, unsigned short (&out)[TERMS]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E >= 1023 - 110 && E <= 1023 + 126) {
    const unsigned long long u0 = (u + 0xFFFFFFFFFFFull + ((u >> 45) & 1ull)) & ~0x1FFFFFFFFFFFull;
    const unsigned hi0 = (unsigned)(u0 >> 32);
    const unsigned E0 = (hi0 >> 20) & 0x7FFu;
    out[0] = (unsigned short)(((hi0 >> 16) & 0x8000u) | ((E0 - 896u) << 7) | ((hi0 >> 13) & 0x7Fu));
    if (TERMS == 1) return;
    const long long M = (long long)((u & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const long long M0 = (long long)((u0 & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (E0 - E);
    long long R = (u >> 63) ? M0 - M : M - M0;
    const int s = E - 1075;
#pragma unroll
    for (int t = 1; t < TERMS; ++t) {
      long long rr;
      out[t] = round_bf16_32(R, s, &rr);  // |R| < 2^45 after a_0
      R -= rr;
    }
    return;
  }
  const long long bits = (long long)u;
  const long long frac = bits & ((1ll << 52) - 1);
  const long long M = E == 0 ? frac : (frac | (1ll << 52));
  const int s = E == 0 ? -1074 : E - 1075;
  long long R = bits < 0 ? -M : M;
#pragma unroll
  for (int t = 0; t < TERMS; ++t) {
    long long rr;
    out[t] = round_bf16(R, s, &rr);
    R -= rr;
  }
}

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
  for (int cc = ty; cc < kTk; cc += 8) {
    const int64_t c = k0 + cc;
    double v = 0.0;
    if (rin && c < M.n_cols && kind_row[col_idx[c]] == CLR_KIND_DENSE) v = M.pool[rbase + c * mR];
    tile[tx][cc] = v;
  }
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = r0 + rr;
    const int64_t k = k0 + 4 * tx;
    unsigned long long packed[TERMS];
#pragma unroll
    for (int t = 0; t < TERMS; ++t) packed[t] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned short b[TERMS];
      split_bf16<TERMS>(tile[rr][4 * tx + q], b);
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
  const int64_t per_row = cols_pad / 4;                 // 4-wide groups along k
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= rows_pad * per_row) return;
  const int64_t j = g / per_row;
  const int64_t k = (g % per_row) * 4;
  unsigned long long packed[TERMS];
#pragma unroll
  for (int t = 0; t < TERMS; ++t) packed[t] = 0;
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
        for (int q = 0; q < 4; ++q) {
          unsigned short b[TERMS];
          split_bf16<TERMS>(src[q], b);
#pragma unroll
          for (int t = 0; t < TERMS; ++t) packed[t] |= (unsigned long long)b[t] << (16 * q);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = k + q;
        double v = 0.0;
        if (kk < M.n_rows) {
          const int R = row_idx[kk];
          if (M.kind[R * M.nc + Cc] == CLR_KIND_DENSE) {
            const int mR = M.row_off[R + 1] - M.row_off[R];
            v = M.pool[(int64_t)M.row_off[R] * M.n_cols + (kk - M.row_off[R]) + j * mR];
          }
        }
        unsigned short b[TERMS];
        split_bf16<TERMS>(v, b);
#pragma unroll
        for (int t = 0; t < TERMS; ++t) packed[t] |= (unsigned long long)b[t] << (16 * q);
      }
    }
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
    const unsigned n = (unsigned)((rows_pad * (cols_pad / 4) + 255) / 256);
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

}  // namespace clr
