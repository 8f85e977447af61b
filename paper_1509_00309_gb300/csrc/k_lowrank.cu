// K2/K3/K4 -- low-rank tile products and their accumulation into C tiles (FP64).
//
// Section 4.1: products are kept in low-rank form whenever an operand is low rank.
//   dense x LR  (DL):  A_IK (X_B W_B^T)          -> (A_IK X_B) W_B^T        rank r_B
//   LR x dense  (LD):  (X_A W_A^T) B_KJ          -> X_A (B_KJ^T W_A)^T      rank r_A
//   LR x LR     (LL):  Z = W_A^T X_B (r_A x r_B), then X_A Z with W_B (rank r_B) or X_A with
//                      W_B Z^T (rank r_A), whichever output rank is smaller (Eq. 1; tie: X_A Z)
// Low-rank sums are concatenations of factors (Eq. lr_addition).  One CTA owns one C tile and
// walks its products in k order:
//   ROUTE_QR     the factor pairs are written side by side into the tile's concatenation
//                workspace (X_cat m x R, W_cat n x R) for recompression by K5;
//   ROUTE_DENSE  the tile already holds the dense x dense sum; every low-rank product is
//                added as X_t W_t^T;
//   ROUTE_DACC   the concatenated rank exceeds floor(min(m,n)/2), so the sum is accumulated
//                densely (from zero) and K5 takes a dense truncated SVD.
// With a tensor-core GEMM (split precision or exact slices: dense_by_gemm) the GEMM sums all
// contributions of DENSE and DACC_G tiles; this kernel builds the ROUTE_QR concatenations and the
// FP64 DACC sums.
#include "clr_internal.h"

namespace clr {

// out(i,j) (= or +=) sum_l a(i,l) b(l,j) for a P x Q output with arbitrary element strides
// (register-tiled, clr_internal.h).
__device__ __forceinline__ void cta_gemm(int P, int Q, int L, const double* a, int64_t a_r,
                                         int64_t a_c, const double* b, int64_t b_r, int64_t b_c,
                                         double* out, int64_t ldo, bool accumulate) {
  cta_gemm_tiled<256>(P, Q, L, a, a_r, a_c, b, b_r, b_c, out, ldo, accumulate);
}

__device__ void cta_copy_cols(int rows, int cols, const double* src, int64_t lds, double* dst,
                              int64_t ldd) {
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int i = e % rows, j = e / rows;
    dst[i + (int64_t)j * ldd] = src[i + (int64_t)j * lds];
  }
}

constexpr int64_t kZElems = (int64_t)(CLR_MAX_CLUSTER / 2) * (CLR_MAX_CLUSTER / 2);

__global__ void __launch_bounds__(256) lr_products_kernel(MatView A, MatView B, MatView C,
                                                          Plan p, double* ws, double* scratch,
                                                          int64_t scratch_per_cta,
                                                          int dense_by_gemm) {
  __shared__ int sh_next;
  double* scrZ = scratch + (int64_t)blockIdx.x * scratch_per_cta;
  double* scrF = scrZ + kZElems;
  const int n_lr = p.counters->n_lr;
  int* sched = &p.counters->sched[0];
  for (int li = next_item(sched, &sh_next); li < n_lr; li = next_item(sched, &sh_next)) {
    const int t = p.l_lr[li];
    const int I = t / p.nJ, J = t % p.nJ;
    const int m = C.row_off[I + 1] - C.row_off[I];
    const int n = C.col_off[J + 1] - C.col_off[J];
    const int route = p.t_route[t];
    // with a tensor-core GEMM the dense tiles and the DACC_G tiles already hold every
    // contribution (low-rank operand blocks staged as X W^T)
    if ((dense_by_gemm && route == ROUTE_DENSE) || route == ROUTE_DACC_G) continue;
    const int R = p.t_rsum[t];
    const int64_t sC = slot_of(C, I, J, m);
    double* D = C.pool + sC;
    double* Xcat = ws + 2 * sC;
    double* Wcat = Xcat + (int64_t)m * R;
    const bool concat = route == ROUTE_QR;
    if (route == ROUTE_DACC) {
      for (int e = threadIdx.x; e < m * n; e += blockDim.x) D[e] = 0.0;
      __syncthreads();
    }
    const int start = p.t_start[t], count = p.t_count[t];
    for (int q = 0; q < count; ++q) {
      const Triple tr = p.triples[start + q];
      if (tr.kind == T_DD) continue;
      const int K = tr.k;
      const int k = A.col_off[K + 1] - A.col_off[K];
      const int ra = A.rank[I * A.nc + K], rb = B.rank[K * B.nc + J];
      const double* Ab = A.pool + slot_of(A, I, K, m);
      const double* Bb = B.pool + slot_of(B, K, J, k);
      const double* Xt;  // m x rt, ld m
      const double* Wt;  // n x rt, ld n
      int rt;
      if (tr.kind == T_DL) {
        // X_t = A_IK X_B, W_t = W_B
        const double* XB = Bb;
        const double* WB = Bb + (int64_t)k * rb;
        rt = rb;
        double* dst = concat ? Xcat + (int64_t)m * tr.col : scrF;
        cta_gemm(m, rb, k, Ab, 1, m, XB, 1, k, dst, m, false);
        Xt = dst;
        Wt = WB;
        if (concat) cta_copy_cols(n, rb, WB, n, Wcat + (int64_t)n * tr.col, n);
      } else if (tr.kind == T_LD) {
        // X_t = X_A, W_t = B_KJ^T W_A
        const double* XA = Ab;
        const double* WA = Ab + (int64_t)m * ra;
        rt = ra;
        double* dst = concat ? Wcat + (int64_t)n * tr.col : scrF;
        cta_gemm(n, ra, k, Bb, k, 1, WA, 1, k, dst, n, false);
        Xt = XA;
        Wt = dst;
        if (concat) cta_copy_cols(m, ra, XA, m, Xcat + (int64_t)m * tr.col, m);
      } else {
        const double* XA = Ab;
        const double* WA = Ab + (int64_t)m * ra;
        const double* XB = Bb;
        const double* WB = Bb + (int64_t)k * rb;
        // Z = W_A^T X_B  (ra x rb, column-major)
        cta_gemm(ra, rb, k, WA, k, 1, XB, 1, k, scrZ, ra, false);
        __syncthreads();
        if (rb <= ra) {
          rt = rb;  // X_t = X_A Z, W_t = W_B
          double* dst = concat ? Xcat + (int64_t)m * tr.col : scrF;
          cta_gemm(m, rb, ra, XA, 1, m, scrZ, 1, ra, dst, m, false);
          Xt = dst;
          Wt = WB;
          if (concat) cta_copy_cols(n, rb, WB, n, Wcat + (int64_t)n * tr.col, n);
        } else {
          rt = ra;  // X_t = X_A, W_t = W_B Z^T
          double* dst = concat ? Wcat + (int64_t)n * tr.col : scrF;
          cta_gemm(n, ra, rb, WB, 1, n, scrZ, ra, 1, dst, n, false);
          Xt = XA;
          Wt = dst;
          if (concat) cta_copy_cols(m, ra, XA, m, Xcat + (int64_t)m * tr.col, m);
        }
      }
      __syncthreads();
      if (!concat) {
        // D += X_t W_t^T
        cta_gemm(m, n, rt, Xt, 1, m, Wt, n, 1, D, m, true);
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

void launch_lr_products(const MatView& A, const MatView& B, const MatView& C, const Plan& p,
                        double* ws, double* scratch, int64_t scratch_per_cta, int dense_by_gemm,
                        int grid, cudaStream_t st) {
  lr_products_kernel<<<grid, 256, 0, st>>>(A, B, C, p, ws, scratch, scratch_per_cta,
                                           dense_by_gemm);
}

}  // namespace clr
