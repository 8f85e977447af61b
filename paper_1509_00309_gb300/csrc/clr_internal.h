// Internal declarations of the CLR library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "clr.h"

namespace clr {

// ---------------------------------------------------------------------------------------------
// Device view of a CLR matrix.  Block (I,J) owns the fixed pool slot
//   slot(I,J) = row_off[I] * n_cols + m_I * col_off[J]
// (the block-row panel of block-row I is an m_I x n_cols column-major matrix, and block
// (I,J) is its columns col_off[J] .. col_off[J+1]-1).  Dense blocks are column-major m x n;
// low-rank blocks store X (m x r) then W (n x r), both column-major.
// ---------------------------------------------------------------------------------------------
struct MatView {
  int nr, nc;            // clusters
  int64_t n_rows, n_cols;
  const int* row_off;    // nr + 1 (device)
  const int* col_off;    // nc + 1 (device)
  int* kind;             // nr * nc
  int* rank;             // nr * nc
  double* norm;          // nr * nc, Frobenius norm of each block
  double* pool;          // n_rows * n_cols
  // nr * nc: SM kilocycles of the block's last dense recompression into this matrix (0: none
  // yet), the scheduling cost of the next one (recompression lists in decreasing cost)
  unsigned int* cost = nullptr;
};

__host__ __device__ inline int64_t slot_of(const MatView& m, int I, int J, int mI) {
  return (int64_t)m.row_off[I] * m.n_cols + (int64_t)mI * m.col_off[J];
}

// Triple kinds and tile routes.
enum { T_DD = 0, T_DL = 1, T_LD = 2, T_LL = 3 };
// MODE_* mirror the accumulation modes of the method: none, dense (a dense x dense product is
// present), low rank.  ROUTE_* refine MODE_LR by how the GPU accumulates:
//   ROUTE_QR   : concatenated rank R <= floor(min(m,n)/2): concatenate factors, QR both,
//                SVD of the R x R core.
//   ROUTE_DACC : larger R: accumulate the sum densely (FP64), then a dense truncated SVD.
//   ROUTE_DACC_G: as ROUTE_DACC, the dense sum formed by the split-precision tensor-core GEMM;
//                only where the split error bound u sum_K ||A_IK|| ||B_KJ|| is below eps/16, so
//                the rank found by the SVD is that of the FP64 sum.
enum { ROUTE_ZERO = 0, ROUTE_DENSE = 1, ROUTE_QR = 2, ROUTE_DACC = 3, ROUTE_DACC_G = 4 };

// Dynamic distribution of a tile list over a persistent grid: the CTA's next item index from
// a launch-wide counter (zeroed before the launch), so that CTAs that drew cheap tiles take
// more of them (tile costs vary with the cube of the cluster size).
__device__ __forceinline__ int next_item(int* counter, int* sh_slot) {
  __syncthreads();
  if (threadIdx.x == 0) *sh_slot = atomicAdd(counter, 1);
  __syncthreads();
  return *sh_slot;
}

// out(i,j) (= or +=) sum_l a(i,l) b(l,j) for a P x Q output with arbitrary element strides, by a
// CTA of NT threads.  FP64 runs at ~2 FMAs per clock per SM on this part, and a single
// accumulator per thread leaves the pipe waiting on each FMA's latency and its two loads: the
// output is cut into 4 x 2 micro-tiles (4 consecutive rows, 2 consecutive columns; the ragged
// last ones clamped), taken by the threads in turn, so a thread runs 8 independent chains whose 6
// loads per step feed 8 FMAs, and skinny outputs (a few dozen columns: the rank of a low-rank
// factor) waste no lanes.  No synchronisation inside: the caller orders dependent calls.
template <int NT>
__device__ __forceinline__ void cta_gemm_tiled(int P, int Q, int L, const double* a,
                                               int64_t a_r, int64_t a_c, const double* b,
                                               int64_t b_r, int64_t b_c, double* out,
                                               int64_t ldo, bool accumulate) {
  const int mp = (P + 3) / 4, mq = (Q + 1) / 2;
  for (int t = threadIdx.x; t < mp * mq; t += NT) {
    const int i0 = (t % mp) * 4, j0 = (t / mp) * 2;
    const double* ap[4];
    const double* bp[2];
#pragma unroll
    for (int x = 0; x < 4; ++x) ap[x] = a + (int64_t)(i0 + x < P ? i0 + x : i0) * a_r;
#pragma unroll
    for (int y = 0; y < 2; ++y) bp[y] = b + (int64_t)(j0 + y < Q ? j0 + y : j0) * b_c;
    double acc[4][2];
#pragma unroll
    for (int x = 0; x < 4; ++x) acc[x][0] = acc[x][1] = 0.0;
    for (int l = 0; l < L; ++l) {
      double av[4], bv[2];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        av[x] = *ap[x];
        ap[x] += a_c;
      }
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        bv[y] = *bp[y];
        bp[y] += b_r;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y)
        if (i0 + x < P && j0 + y < Q) {
          double* o = out + (i0 + x) + (int64_t)(j0 + y) * ldo;
          *o = accumulate ? *o + acc[x][y] : acc[x][y];
        }
  }
}

struct Triple {
  int tile;   // C block index I * nJ + J
  int k;      // inner cluster K
  int kind;   // T_*
  int col;    // QR route: first column of this product's factors in the tile concatenation
};

// Counters written by the planning kernels (device, zeroed before each plan).
struct PlanCounters {
  unsigned long long n_triples;
  unsigned long long by_kind[4];
  unsigned long long flops;
  unsigned long long by_mode[3];
  unsigned long long max_rsum;
  unsigned long long n_gemm_dacc;  // tiles routed ROUTE_DACC_G
  int n_dense, n_lr, n_qr, n_dacc, n_dcomp;
  int sched[4];   // work counters of the tile-list kernels (next_item), zeroed with the plan
  // error flag raised by kernels (1: a bounded wait gave up, 2: triple list overflow, 3:
  // non-finite data).  Sticky: a plan clears only the fields before it, and the host reads and
  // clears it at its next synchronisation.
  int err;
};
// Bytes of PlanCounters a new plan clears (everything but the sticky error flag).
constexpr size_t kPlanCountersClear = offsetof(PlanCounters, err);

struct Plan {
  int nI, nJ, nK;
  int* t_count;   // nI*nJ
  int* t_start;   // nI*nJ
  int* t_route;   // nI*nJ
  int* t_rsum;    // nI*nJ
  int* l_dense;   // tiles with ROUTE_DENSE
  int* l_lr;      // tiles with at least one low-rank product (any route)
  int* l_qr;      // ROUTE_QR
  int* l_dcomp;   // tiles needing a dense truncated SVD (ROUTE_DACC, or ROUTE_DENSE when
                  // dense tiles are recompressed)
  int* l_qr_s;    // l_qr and l_dcomp reordered by decreasing recompression cost (plan_scan)
  int* l_dcomp_s;
  int* l_dense_s;  // l_dense reordered by decreasing cost m n (number of products)
  const int* row_off;  // C's cluster offsets (device), for those costs
  const int* col_off;
  const unsigned int* c_cost;  // C's measured recompression costs (MatView::cost), or null
  Triple* triples;
  int64_t max_triples;
  PlanCounters* counters;
};

// ---------------------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All are asynchronous on `st`.
// ---------------------------------------------------------------------------------------------
// k_plan.cu
// Exact slices: the routing of densely accumulated low-rank sums to the tensor-core GEMM
// (plan_count_kernel); sa/sb: per cluster and K segment, sum over its rows (columns) of 4^e.
struct OzDaccRule {
  const double* sa = nullptr;   // nI x n_seg
  const double* sb = nullptr;   // nJ x n_seg
  int n_seg = 0;
  double bound2 = 0.0;
};
void launch_plan(const MatView& A, const MatView& B, const Plan& p, double eps_sp,
                 int recompress_dense, double gemm_dacc_bound, const OzDaccRule& oz,
                 cudaStream_t st);
void launch_plan_scan(const Plan& p, int recompress_dense, cudaStream_t st);
// k_dense64.cu
// uses p.counters->sched[3]
void launch_dd_fp64(const MatView& A, const MatView& B, const MatView& C, const Plan& p,
                    int grid, cudaStream_t st);
void launch_set_route_kinds(const MatView& C, const Plan& p, cudaStream_t st);
void launch_dense_tile_norms(const MatView& C, const Plan& p, cudaStream_t st);
// norm = sqrt(norm) of the route-DENSE tiles (their sums of squares came from the GEMM epilogue)
void launch_sqrt_dense_norms(const MatView& C, const Plan& p, cudaStream_t st);
// k_layout.cu
void launch_rowmajor_to_pool(const MatView& M, const int* row_idx, const double* src,
                             int64_t lds, cudaStream_t st);
void launch_dense_kinds(const MatView& M, double drop_norm, int* err, cudaStream_t st);
void launch_pool_to_rowmajor(const MatView& M, const int* row_idx, const int* col_idx,
                             double* out, int64_t ldo, cudaStream_t st);
// k_lowrank.cu
// dense_by_gemm: DENSE and DACC tiles were fully summed by the split GEMM (skip them).
void launch_lr_products(const MatView& A, const MatView& B, const MatView& C, const Plan& p,
                        double* ws, double* scratch, int64_t scratch_per_cta, int dense_by_gemm,
                        int grid, cudaStream_t st);  // uses p.counters->sched[0]
// k_svd.cu
// jstats (may be null): device counters {svd blocks, FP32 sweeps, FP64 sweeps, early dense}
// svd_scratch: grid x kSvdScratchPerCta doubles (FP32 working copies and an FP64 q x q factor
// of the mixed-precision SVD, then the pivoted-QR path's R and the right factor of its SVD).
constexpr int64_t kSvdScratchPerCta = (int64_t)4 * CLR_MAX_CLUSTER * CLR_MAX_CLUSTER;
// sched: a zeroed work counter (dynamic tile distribution).
void launch_compress_qr(const MatView& C, const int* list, const int* count, const int* rsum,
                        double* ws, double* svd_scratch, double eps, int max_sweeps, int grid,
                        int* err, int* sched,
                        unsigned long long* jstats, cudaStream_t st);
// Dense truncated SVD of blocks listed in `list` (count on device).  The source of block b is
// either the matrix's own slot (src == nullptr) or a row-major dense matrix src with leading
// dimension lds.  drop_norm: blocks with norm below it become zero.  dense_only: skip the
// SVD (eps = 0 rule) and store every non-dropped block dense.
// order (list == nullptr only, may be null): the order in which all blocks are visited.
// rrqr: truncate by rank-revealing QR instead of the SVD.
// prereduce: reduce every block by a column-pivoted QR (stopped at eps/16) before the SVD of
// its k x q factor R, unless the QR's triangles certify it dense; without it every block takes
// the full SVD.
// jstats (7 counters): SVD blocks, FP32 sweeps, FP64 sweeps, early dense exits, FP64 flops,
// FP32 flops, pre-reduced blocks.
void launch_compress_dense(const MatView& C, const int* list, const int* count,
                           const int* order, const double* src, int64_t lds, double* ws,
                           double* svd_scratch, double eps, double drop_norm,
                           int dense_only, int rrqr, int prereduce, int max_sweeps, int grid,
                           int* err, int* sched, unsigned long long* jstats, cudaStream_t st);
void launch_block_norms(const MatView& M, cudaStream_t st);
void launch_block_norms_dense(const MatView& M, cudaStream_t st);
void launch_scale_blocks(const MatView& M, double alpha, cudaStream_t st);
// k_ns.cu
void launch_lincomb_plan(double a, const MatView& X, double b, const MatView& Y, double diag,
                         const MatView& O, const Plan& p, double* ws, int recompress_dense,
                         cudaStream_t st);
void launch_identity_distance(const MatView& X, double* out_sq, cudaStream_t st);
void launch_matvec(const MatView& M, const double* x, double* y, cudaStream_t st);
void launch_transpose(const MatView& S, const MatView& T, cudaStream_t st);
// k_split_gemm.cu
struct SplitGemmArgs {
  const MatView* A;
  const MatView* B;
  const MatView* C;
  const Plan* p;
  int terms;          // 2 (bf16x3) or 3 (bf16x6)
  void* a_panels;     // terms x M_pad x K_pad bf16
  void* b_panels;     // terms x N_pad x K_pad bf16
  int64_t M_pad, N_pad, K_pad;
  const int* row_tile_of;  // n_rows: C block-row of each row
  const int* col_tile_of;  // n_cols
  unsigned char* tile_active;  // (M_pad/128) * (N_pad/256) flags
  int n_sm;
  int* err;
  unsigned long long wait_ns = 2000000000ull;  // give-up limit of the pipeline's waits
  void* encode_fn;    // cuTensorMapEncodeTiled
  // fused norms (may be null): the epilogue adds the squares of the values it writes into
  // route-DENSE C tiles to norm_sq[I * nJ + J] (zeroed before; needs row clusters >= 32 rows
  // and column clusters >= 16 columns)
  double* norm_sq = nullptr;
};
int split_gemm_dd(const SplitGemmArgs& a, cudaStream_t st, std::string* why);
// k_ozaki.cu: FP64-accurate dense x dense products on the tensor cores (exact slices)
constexpr int kOzakiSlices = 8;
constexpr int kOzakiSegK = 1024;   // K segment: exact FP32 group sums, exponents per segment
constexpr int kOzakiTileN = 32;    // the GEMM's output tiles are 128 x kOzakiTileN
constexpr int kOzakiPassK = 2048;  // K per GEMM launch (later launches add into C)
struct OzakiGemmArgs {
  const MatView* C;
  const Plan* p;
  void* a_panels;     // kOzakiSlices x M_pad x K_pad bf16 digits
  void* b_panels;     // kOzakiSlices x N_pad x K_pad
  const int* ea;      // n_seg x M_pad row exponents of A per K segment
  const int* eb;      // n_seg x N_pad column exponents (rows of the B panel) per K segment
  int64_t M_pad, N_pad, K_pad;   // multiples of 128, kOzakiTileN, 128
  const int* row_tile_of;
  const int* col_tile_of;
  unsigned char* tile_active;  // (M_pad/128) * (N_pad/kOzakiTileN) flags
  int* active_list;            // 1 + that many ints: the active tiles' count and ids
  int n_sm;
  int* err;
  unsigned long long wait_ns = 2000000000ull;
  void* encode_fn;
};
int ozaki_gemm_dd(const OzakiGemmArgs& a, cudaStream_t st, std::string* why);
// exps: n_seg x rows_pad ints (n_seg = K segments of kOzakiSegK), written (the row exponents
// per segment); panels: kOzakiSlices planes
// recon: scratch of M.n_rows x M.n_cols doubles (the low-rank blocks' reconstructions)
void launch_ozaki_stage(const MatView& M, const int* row_idx, const int* col_idx, void* panels,
                        int* exps, double* recon, int64_t rows_pad, int64_t cols_pad,
                        int a_mode, cudaStream_t st);
// out[c * n_seg + s] = sum over rows i in [off[c], off[c + 1]) of 4^exps[s * rows_pad + i]
void launch_ozaki_scale_sums(const int* exps, int64_t rows_pad, const int* off, int n_cl,
                             int n_seg, double* out, cudaStream_t st);
void launch_split_stage(const MatView& M, const int* row_idx, const int* col_idx, void* panels,
                        int terms, int64_t rows_pad, int64_t cols_pad, int a_mode,
                        cudaStream_t st);

}  // namespace clr
