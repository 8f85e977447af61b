/*
 * clr.h -- C ABI of a GB300 (sm_103a) library for products of Clustered Low-Rank (CLR,
 * block-rank-sparse) matrices and the Newton–Schulz iteration for S^-1/2.
 *
 * Method: Calvin, Lewis & Valeev, "Scalable Task-Based Algorithm for Multiplication of
 * Block-Rank-Sparse Matrices", IA^3 2015.  Section 4.1 defines the CLR representation and its
 * block arithmetic; Section 4.2 the Newton–Schulz iteration.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status: CLR_OK (0) or a negative CLR_E* code.  No C++
 *    exception crosses this boundary.  clr_strerror() names a code; clr_last_error() gives
 *    the context's last detailed message.
 *  - Errors found on the device (a bounded device-side wait that gave up, non-finite data met
 *    by recompression, an overflowing triple list) raise a sticky flag in the context's
 *    workspaces.  Asynchronous calls cannot report it; the next call that synchronises (NS
 *    iterations, clr_multiply_into with stats, clr_check, clr_multiply_host_stream,
 *    clr_multiply_batched, clr_multiply_backward, clr_batch_create, clr_mat_from_dense)
 *    returns it as CLR_ETIMEOUT
 *    or CLR_EINVAL and clears it.  The outputs of the failed work are then unspecified.
 *  - A CLR matrix (clr_mat_t) is an opaque, library-owned handle living on the context's
 *    device.  Handles returned through an out-pointer are new and owned by the caller, who
 *    releases them with clr_mat_free().  Input matrices are never modified.
 *  - Block layout (used by clr_mat_from_blocks / clr_mat_get_blocks): a matrix with row
 *    clusters of sizes m_0..m_{nr-1} and column clusters n_0..n_{nc-1} owns a pool of
 *    n_rows * n_cols doubles.  Block (I,J) owns the fixed slot starting at
 *    row_off[I] * n_cols + m_I * col_off[J] (row_off / col_off: exclusive prefix sums of
 *    the cluster sizes).  A dense block stores its m x n values column-major (element (i,j)
 *    at i + j*m).  A low-rank block of rank r stores X (m x r, column-major) followed by W
 *    (n x r, column-major); the block equals X W^T.  Low-rank blocks have
 *    1 <= r <= floor(min(m,n)/2) (blocks of larger rank are stored dense, Section 4.1), so
 *    (m + n) r <= m n and every block fits its slot.  Block (I,J) has index I*nc + J.
 *  - Cluster sizes must be in [1, CLR_MAX_CLUSTER].
 *  - Device work is issued on the caller's stream (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream).  Calls that must read device results on the host
 *    (sizes, statistics, convergence tests) synchronise that stream; each such call says so.
 *  - There is no CPU fallback: without a usable sm_103a device, clr_create fails with
 *    CLR_ECUDA.
 */
#ifndef CLR_H_
#define CLR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define CLR_OK        0
#define CLR_EINVAL   -1   /* bad argument: tiling mismatch, size out of range, NaN input ... */
#define CLR_ENOMEM   -2   /* device allocation failed */
#define CLR_ENOCONV  -3   /* Newton–Schulz did not reach ns_tol within ns_max_iter */
#define CLR_ETIMEOUT -4   /* a bounded device-side wait gave up (error flag set by a kernel) */
#define CLR_ECUDA    -5   /* CUDA runtime/driver error (see clr_last_error) */
#define CLR_ENOTSUP  -6   /* operation not supported for these arguments */

/* ---- block kinds (Section 4.1: each block is zero, dense, or low-rank X W^T) ------------- */
#define CLR_KIND_ZERO  0
#define CLR_KIND_DENSE 1
#define CLR_KIND_LR    2

/* ---- arithmetic of dense x dense tile products ------------------------------------------ */
#define CLR_PREC_FP64   0  /* FP64 on CUDA cores */
#define CLR_PREC_BF16X3 1  /* 2-term bf16 split, 3 tensor-core products, FP32 accumulation */
#define CLR_PREC_BF16X6 2  /* 3-term bf16 split, 6 tensor-core products, FP32 accumulation */
#define CLR_PREC_AUTO   3  /* cheapest of bf16x3, bf16x6, the exact slices below and FP64 whose
                              a-priori error model meets eps_lr (the batch autotuner times each
                              candidate and keeps the fastest) */
#define CLR_PREC_OZAKI  4  /* FP64-accurate tile products on the tensor cores: in each K
                              segment of 1024, rows of A and columns of B scaled by powers of
                              two and cut into 8 fixed-point slices of 6 bits (bf16 digits), the
                              36 slice pairs of weight >= 2^-48 summed exactly in FP32, segments
                              summed in FP64 (Ozaki, Ogita, Oishi, Rump 2012); error at most
                              sum over segments of K_seg 2^-44 max|a_i.| max|b_.j| (maxima over
                              the segment) per entry.  Low-rank operand blocks enter as their
                              reconstructions, so the GEMM forms the whole sum of the dense C
                              tiles and of densely accumulated low-rank sums whose expected
                              sliced error is within eps_lr / 64; other low-rank sums stay FP64 */

#define CLR_MAX_CLUSTER 256

typedef struct clr_ctx_s* clr_ctx_t;
typedef struct clr_mat_s* clr_mat_t;
typedef struct clr_tape_s* clr_tape_t;
typedef struct clr_batch_s* clr_batch_t;

/* Options of a context.  Fill with clr_opts_default() and override fields. */
typedef struct clr_opts {
  double eps_lr;         /* truncation threshold: Frobenius error per block (Section 4.1) */
  double eps_sp;         /* screening threshold: C_IJ computed only if its norm estimate
                            exceeds eps_sp * area(C_IJ) (Section 4.1); 0 disables */
  int precision;         /* CLR_PREC_* for dense x dense tile products */
  int recompress_dense;  /* 1: dense-accumulated C tiles are re-tested for low rank */
  int ns_max_iter;       /* Newton–Schulz: maximum number of Z updates */
  double ns_tol;         /* stated error of NS: the loop stops when ||X_n - I||_F / sqrt(N)
                            <= ns_tol, and succeeds when the returned Z has
                            ||alpha Z S Z - I||_F / sqrt(N) <= ns_tol; 0 runs exactly
                            ns_max_iter updates */
  double ns_alpha;       /* NS scale alpha; 0 = 1 / (1.01 * power-iteration estimate) */
  int ns_power_steps;    /* power iterations for the alpha estimate (default 30) */
  int ns_fp64_tail;      /* precision ladder: switch tile products to FP64 once
                            ||X_n - I||_F / sqrt(N) <= ns_ladder_switch */
  double ns_ladder_switch;
  int jacobi_max_sweeps; /* one-sided Jacobi sweep limit (default 40) */
  int ns_snapshot_iter;  /* k > 0: clr_sqrt_inv keeps copies of X_k, Y_k, Z_k, T_k of its k-th
                            iteration (Section 5's rank distribution of 5th-iteration
                            intermediates), read back with clr_ns_snapshot; 0 = off */
  int build_rrqr;        /* 1: clr_mat_from_dense builds low-rank blocks by rank-revealing QR
                            (greedy column pivoting, truncated at ||R_22||_F <= eps_lr; the
                            paper's construction, Section 4.1) instead of the truncated SVD
                            (the minimal rank for the same error) */
  int wait_timeout_us;   /* limit of every bounded device-side wait of the tensor-core
                            pipeline, in microseconds (0: 2 s).  A wait that runs out stops
                            the kernel cleanly and raises CLR_ETIMEOUT at the next
                            synchronising call */
  int svd_no_prereduce;  /* 1: dense truncated SVDs (recompression of densely accumulated
                            tiles, clr_mat_from_dense) always run the one-sided Jacobi on the
                            whole block; 0 (default): a column-pivoted QR stopped at eps/16
                            first reduces blocks of low numerical rank to a k x q factor */
  int reserved[4];
} clr_opts;

/* Summary of a CLR matrix (clr_mat_info). */
typedef struct clr_info {
  int64_t n_rows, n_cols;
  int32_t n_row_clusters, n_col_clusters;
  int64_t n_blocks[3];      /* by kind: zero, dense, low rank */
  int32_t max_rank;         /* over low-rank blocks */
  int64_t sum_rank;         /* over low-rank blocks */
  int64_t stored_doubles;   /* doubles actually used by dense values and factors */
  double frob_norm;         /* sqrt(sum of squared block norms) */
  int32_t rank_hist[CLR_MAX_CLUSTER / 2 + 2]; /* low-rank blocks by rank; [0] counts zero
                                                 blocks, the last bin counts dense blocks */
} clr_info;

/* Work statistics of one product (clr_multiply_into with a non-NULL stats pointer). */
typedef struct clr_product_stats {
  int64_t n_triples[4];     /* tile products by kind: DD, DL, LD, LL */
  int64_t flops;            /* algorithmic flops of the tile products */
  int64_t n_tiles[3];       /* C tiles accumulated as: none, dense, low rank */
  int64_t max_rank_sum;     /* largest concatenated rank of a low-rank C tile */
  int32_t precision;        /* precision used for dense x dense products */
  int32_t n_tiles_tensor;   /* C tiles summed entirely by the tensor-core GEMM (split precision:
                               tiles with a dense x dense product, and densely accumulated
                               low-rank sums within the split error bound) */
} clr_product_stats;

/* Newton–Schulz statistics (clr_sqrt_inv). */
#define CLR_NS_MAX_HISTORY 256
typedef struct clr_ns_stats {
  int32_t iters;            /* Z updates applied */
  int32_t converged;        /* the stated error was met: residual <= ns_tol (ns_tol > 0), or
                               ns_tol == 0 (a fixed number of iterations) */
  double alpha;
  double residual;          /* ||alpha Z S Z - I||_F / sqrt(N) of the returned Z */
  double proxy[CLR_NS_MAX_HISTORY]; /* ||X_n - I||_F / sqrt(N), n = 0..iters */
  int32_t precision_used[CLR_NS_MAX_HISTORY];
  double ms_total;          /* device time of the iteration loop (CUDA events) */
  int32_t proxy_met;        /* the loop's stopping test ||X_n - I||_F / sqrt(N) <= ns_tol held */
  int32_t residual_met;     /* residual <= ns_tol */
  double ms_residual;       /* device time of the final residual (two CLR products) */
} clr_ns_stats;

/* ---- errors and options ------------------------------------------------------------------ */
const char* clr_strerror(int status);
const char* clr_last_error(clr_ctx_t ctx);
void clr_opts_default(clr_opts* opts);

/* ---- context ------------------------------------------------------------------------------
 * clr_create: binds a context to CUDA device `device` (made current on the calling thread),
 * checks that it is an sm_103 part, and loads the TMA encoder from the driver.  Fails with
 * CLR_ECUDA when no such device exists.  clr_destroy frees the context's workspaces; it does
 * not free matrices.
 * Workspaces are allocated on first use, grow to the largest product seen and stay until
 * clr_destroy.  For C = A B they take about 16 bytes per element of C's dense footprint (tile
 * accumulation and SVD workspace), 2 MiB per CTA of the low-rank and recompression kernels
 * (2 CTAs per SM unless the autotuner picks another count), and with a tensor-core precision
 * the operands' panels: 4 (bf16x3), 6 (bf16x6) or 16 (exact slices, plus FP64 images of the
 * low-rank operand blocks) bytes per element of A and of B.  Newton-Schulz keeps a second set
 * for its concurrent products; each batch owns one set per graph branch. */
int clr_create(clr_ctx_t* ctx, int device, const clr_opts* opts);
int clr_destroy(clr_ctx_t ctx);
int clr_set_opts(clr_ctx_t ctx, const clr_opts* opts);
int clr_get_opts(clr_ctx_t ctx, clr_opts* opts);

/* ---- matrices -----------------------------------------------------------------------------
 * clr_mat_create: an all-zero matrix with the given clusters (capacity for any content).
 * clr_mat_from_dense: CLR form of a dense row-major n_rows x n_cols FP64 matrix `a` (leading
 *   dimension lda >= n_cols; `a_on_host` 1 for host memory, 0 for device memory).  Each block
 *   is dropped when ||block||_F < drop_norm, else truncated by its SVD at Frobenius error
 *   eps_lr (Section 4.1 builds X, W by rank-revealing QR; the SVD gives the minimal rank of
 *   the same criterion), else stored dense when the rank exceeds floor(min(m,n)/2).  With
 *   eps_lr == 0 every block that is not dropped is stored dense.
 * clr_mat_from_blocks: copies kinds[nr*nc], ranks[nr*nc] and a host pool of n_rows*n_cols
 *   doubles in the block layout above; no compression is applied.
 * clr_mat_to_dense: reconstructs the matrix into row-major `out` (leading dimension ldo).
 * clr_mat_get_blocks: copies kinds, ranks, block Frobenius norms and the pool to the host
 *   (any pointer may be NULL).  Synchronises `stream`.
 * clr_mat_info: summary statistics; synchronises `stream`. */
int clr_mat_create(clr_ctx_t ctx, int n_rt, const int32_t* row_sizes, int n_ct,
                   const int32_t* col_sizes, clr_mat_t* out);
int clr_mat_from_dense(clr_ctx_t ctx, const double* a, int64_t lda, int a_on_host, int n_rt,
                       const int32_t* row_sizes, int n_ct, const int32_t* col_sizes,
                       double eps_lr, double drop_norm, void* stream, clr_mat_t* out);
int clr_mat_from_blocks(clr_ctx_t ctx, int n_rt, const int32_t* row_sizes, int n_ct,
                        const int32_t* col_sizes, const int32_t* kinds, const int32_t* ranks,
                        const double* pool_host, void* stream, clr_mat_t* out);
int clr_mat_to_dense(clr_ctx_t ctx, clr_mat_t m, double* out, int64_t ldo, int out_on_host,
                     void* stream);
int clr_mat_get_blocks(clr_ctx_t ctx, clr_mat_t m, int32_t* kinds, int32_t* ranks,
                       double* norms, double* pool_host, void* stream);
int clr_mat_info(clr_ctx_t ctx, clr_mat_t m, clr_info* info, void* stream);
int clr_mat_shape(clr_mat_t m, int64_t* n_rows, int64_t* n_cols, int* n_rt, int* n_ct);
int clr_mat_copy(clr_ctx_t ctx, clr_mat_t src, clr_mat_t dst, void* stream);
int clr_mat_transpose(clr_ctx_t ctx, clr_mat_t src, clr_mat_t* out, void* stream);
/* clr_mat_free returns the storage to the caching allocator below, whose buffers are handed to
 * later allocations without stream ordering: the device work that reads or writes `m` must have
 * completed (synchronise its stream first). */
int clr_mat_free(clr_ctx_t ctx, clr_mat_t m);
/* Matrix storage comes from a process-wide caching allocator: freed buffers are kept (up to
 * 64 GiB) and reused by later matrices of the same size.  clr_mem_trim returns the context
 * device's cached buffers to CUDA; clr_mem_cached reports the bytes currently cached. */
int clr_mem_trim(clr_ctx_t ctx);
int64_t clr_mem_cached(void);

/* ---- the CLR product (Section 4.1) --------------------------------------------------------
 * C = alpha * (A B): every C tile receives the tile products A_IK B_KJ with both blocks
 * nonzero (dense x dense, dense x low-rank, low-rank x dense, low-rank x low-rank with
 * Z = W_A^T X_B contracted on the side of smaller output rank), screened with eps_sp; tiles
 * with a dense x dense product are accumulated dense, the others by concatenating factors
 * and recompressing (QR of both factors, SVD of the small core, truncation at eps_lr).  The
 * truncation happens before the scaling by alpha.  A's column clusters must equal B's row
 * clusters (else CLR_EINVAL).
 * clr_multiply: allocates C.  clr_multiply_into: C must have A's row clusters and B's column
 *   clusters and must not be A or B; no host synchronisation unless `stats` is non-NULL.
 * clr_multiply_batched: n independent products in one CUDA graph launch (see clr_batch_*;
 *   tuned when the precision is CLR_PREC_AUTO); the outputs are new handles for the caller. */
int clr_multiply(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t* c, void* stream);
int clr_multiply_into(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, double alpha,
                      clr_product_stats* stats, void* stream);
int clr_multiply_batched(clr_ctx_t ctx, int n, const clr_mat_t* a, const clr_mat_t* b,
                         clr_mat_t* c, void* stream);
/* clr_multiply_backward: the adjoint of C = A B (Section 4.1's block product run backwards,
 * with truncation treated as the identity): given cbar = dL/dC (A's row clusters, B's column
 * clusters), returns abar = cbar B^T (A's clusters) and bbar = A^T cbar (B's clusters), each a
 * CLR product of the transposed operand recompressed at eps_lr in the context's precision.
 * Either output pointer may be NULL (that adjoint is skipped), not both.  The outputs are new
 * handles.  Synchronises `stream` (the transposed operands are freed after the products). */
int clr_multiply_backward(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t cbar,
                          clr_mat_t* abar, clr_mat_t* bbar, void* stream);

/* Dense product of host matrices through the CLR product, streamed: C = A B with A (m x k),
 * B (k x n) and C (m x n) row-major in page-locked host memory (leading dimensions lda, ldb,
 * ldc >= the column counts), tiled by the cluster sizes rs (rows of A and C), ks (columns of A,
 * rows of B) and cs (columns of B and C).  A moves in two row chunks and B in n_chunks column
 * chunks (whole clusters each), copied on one stream in the order the products need them
 * (A_0, B_0, A_1, B_1, B_2, ...) through two alternating device staging buffers and laid out
 * into matrices on another, so the copies run back to back; the product of row chunk i and
 * column chunk j starts as soon as both are laid out, on one of two streams with their own
 * workspaces (one per row chunk, so that chunk's bf16 panels are staged once), and its tile of
 * C goes back to the host at once from two download streams that do not hold up the products:
 * the copy engines' transfers in both directions overlap the products.  Every
 * block is kept dense (the eps = 0 build); the products use the context's precision.
 * Synchronises `stream` before returning.  CLR_EINVAL when a buffer is not page-locked or
 * holds non-finite values. */
int clr_multiply_host_stream(clr_ctx_t ctx, const double* a, int64_t lda, const double* b,
                             int64_t ldb, double* c, int64_t ldc, int n_rt, const int32_t* rs,
                             int n_kt, const int32_t* ks, int n_ct, const int32_t* cs,
                             int n_chunks, void* stream);

/* ---- batched products in one CUDA graph, and the autotuner ------------------------------
 * clr_batch_create: n independent products C_i = A_i B_i (uneven sizes, clusters and ranks),
 *   product i truncated at eps[i] (eps NULL: the context's eps_lr).  Allocates the outputs, picks each product's launch configuration (with tune_on: the
 *   autotuner measures every allowed precision -- the configured one, or under CLR_PREC_AUTO
 *   each mode whose error model meets eps_lr -- times 1, 2 or 4 CTAs per SM for the low-rank
 *   and recompression kernels, once per shape key, and keeps the fastest), runs each product
 *   once to size its workspaces, and captures all of them into one CUDA graph whose products
 *   run on up to 4 parallel branches with their own workspaces (longest-first assignment).
 *   Synchronises `stream`.  The inputs must stay alive and unchanged while the batch exists.
 * clr_batch_run: one graph launch computing every product on `stream` (replayable).
 * clr_batch_free: waits for the batch's last launch (an event recorded by clr_batch_run), then
 *   frees its outputs and workspaces.
 * clr_batch_output: the i-th output (owned by the batch until clr_batch_free).
 * clr_batch_tuning: the chosen precision, CTAs per SM and branch of product i.
 * clr_autotune_save / clr_autotune_load: the autotuner's cache as a text file (one line per
 *   shape key: key precision ctas_per_sm ms); clr_autotune_entries: cache size. */
int clr_batch_create(clr_ctx_t ctx, int n, const clr_mat_t* a, const clr_mat_t* b,
                     const double* eps, int tune_on, void* stream, clr_batch_t* out);
int clr_batch_run(clr_ctx_t ctx, clr_batch_t batch, void* stream);
int clr_batch_output(clr_batch_t batch, int i, clr_mat_t* c);
int clr_batch_tuning(clr_batch_t batch, int i, int* precision, int* ctas_per_sm, int* branch);
int clr_batch_free(clr_ctx_t ctx, clr_batch_t batch);
int clr_autotune_save(clr_ctx_t ctx, const char* path);
int clr_autotune_load(clr_ctx_t ctx, const char* path);
int clr_autotune_entries(clr_ctx_t ctx);

/* ---- CLR linear combination (low-rank addition, Section 4.1, Eq. lr_addition) ------------
 * out = a X + b Y + diag I.  A block present in one operand only is scaled exactly; a block
 * with a dense operand, or a diagonal block when diag != 0, is summed densely; two low-rank
 * blocks are concatenated and recompressed at eps_lr.  `out` must be preallocated with X's
 * clusters and must not alias X or Y. */
int clr_lincomb(clr_ctx_t ctx, double a, clr_mat_t x, double b, clr_mat_t y, double diag,
                clr_mat_t out, void* stream);

/* ---- Newton–Schulz S^-1/2 (Section 4.2) ---------------------------------------------------
 * X_n = alpha Y_n Z_n, T_n = (15 I - 10 X_n + 3 X_n^2)/8, Z_{n+1} = Z_n T_n,
 * Y_{n+1} = T_n Y_n, Z_0 = I, Y_0 = S; returns Z = sqrt(alpha) Z_n.  Every product is a CLR
 * product at the context's eps_lr / eps_sp; T is formed by clr_lincomb.  Synchronises
 * `stream` once per iteration to read the loop's stopping scalar ||X_n - I||_F / sqrt(N).
 * With ns_tol > 0 the loop stops once that proxy is <= ns_tol, and the stated error is then
 * checked on the returned Z: the residual ||alpha Z S Z - I||_F / sqrt(N) (two more CLR
 * products).  Returns CLR_ENOCONV (with *z still set) unless that residual is <= ns_tol: the
 * proxy can meet the tolerance while truncation at eps_lr holds the residual above it.  With
 * `tape` non-NULL the iterates (Y_n, Z_n) are kept for clr_sqrt_inv_backward (checkpointed
 * every iteration); the tape owns copies of everything it needs, so S may be freed before the
 * backward call. */
int clr_sqrt_inv(clr_ctx_t ctx, clr_mat_t s, clr_mat_t* z, clr_ns_stats* stats,
                 clr_tape_t* tape, void* stream);
/* clr_check: synchronises `stream` and returns (and clears) any error a kernel raised since the
 * last synchronising call. */
int clr_check(clr_ctx_t ctx, void* stream);
/* ||alpha Z S Z - I||_F / sqrt(N) for z = sqrt(alpha) Z: two CLR products in FP64, or by exact
 * slices when the context's precision is CLR_PREC_OZAKI (FP64-accurate: at most
 * K 2^-39 2^(e_i + f_j) per entry), whose densely accumulated tiles are summed without the
 * low-rank re-test; synchronises. */
int clr_ns_residual(clr_ctx_t ctx, clr_mat_t s, clr_mat_t z, double* out, void* stream);
/* Adjoint of clr_sqrt_inv for L = trace(W^T-weighted) losses: given zbar = dL/dZ (Z the
 * returned sqrt(alpha) Z_n), returns sbar = dL/dS by running the NS recurrences backwards
 * over the tape with alpha held constant; truncation is treated as the identity and every
 * adjoint product is a CLR product at eps_lr. */
int clr_sqrt_inv_backward(clr_ctx_t ctx, clr_tape_t tape, clr_mat_t zbar, clr_mat_t* sbar,
                          void* stream);
int clr_tape_free(clr_ctx_t ctx, clr_tape_t tape);
/* Intermediates of the k-th NS iteration (k = opts.ns_snapshot_iter, 1-based) of the last
 * clr_sqrt_inv on this context: which = 0: X_k = alpha Y_{k-1} Z_{k-1}, 1: T_k, 2: Y_k = T_k
 * Y_{k-1}, 3: Z_k = Z_{k-1} T_k (Z unscaled, before the final sqrt(alpha)).  Ownership passes
 * to the caller (free with clr_mat_free); CLR_EINVAL when no such snapshot is held (snapshot
 * off, the iteration not reached, or already taken).  Use clr_mat_info's rank histogram on it. */
int clr_ns_snapshot(clr_ctx_t ctx, int which, clr_mat_t* out);

/* ---- observability ------------------------------------------------------------------------
 * With profiling on, every product records CUDA events on its stream at its phase boundaries
 * and counts the kernels it launches; clr_sqrt_inv then runs its two independent products one
 * after the other (not on two streams), so that each interval times its own kernels.  clr_profile_read synchronises the device, converts the
 * events to per-phase device times (ms, summed over products) and returns the totals;
 * clr_profile_enable(ctx, 1) resets them. */
typedef struct clr_profile {
  int64_t products;            /* products recorded */
  int64_t launches;            /* kernels launched by those products */
  int64_t dense_launches;      /* launches of the dense x dense kernel */
  double dense_tensor_flops;   /* tensor-core flops issued by the split dense kernel */
  double ms_plan;              /* triple list: screen, count, scan, fill */
  double ms_stage;             /* split-precision staging of operand panels */
  double ms_dense;             /* dense x dense tile products */
  double ms_lowrank;           /* low-rank tile products and accumulation */
  double ms_compress;          /* recompression (QR + SVD): the two kernels below */
  double ms_finalize;          /* norms and scaling */
  int64_t svd_blocks;          /* truncated SVDs (one-sided Jacobi) run by recompression */
  int64_t svd_sweeps_fp32;     /* FP32 sweeps, summed over those SVDs */
  int64_t svd_sweeps_fp64;     /* FP64 sweeps, summed */
  int64_t svd_early_dense;     /* SVDs stopped after the FP32 phase (certified dense) */
  double svd_flops_fp64;       /* algorithmic FP64 flops of recompression: QR 2(m+n)R^2, core
                                  products, orthonormalisations 2q^3, projections 2pq^2, Jacobi
                                  4pq^2 per FP64 sweep, factor recovery / re-expansion */
  double svd_flops_fp32;       /* algorithmic FP32 flops: Jacobi 4pq^2 per FP32 sweep */
  int64_t svd_prereduced;      /* dense blocks truncated through the pivoted-QR pre-reduction */
  double ms_compress_qr;       /* the QR route's recompression (compress_qr_kernel) */
  double ms_compress_dense;    /* dense truncated SVDs (compress_dense_kernel) */
  double svd_flops_fp64_qr;    /* the part of svd_flops_fp64 done by the QR route */
  double svd_flops_fp32_qr;    /* the part of svd_flops_fp32 done by the QR route */
  double svd_path_cycles[4];   /* SM cycles in compress_dense_kernel summed over blocks, by
                                  path: pivoted QR and the SVD of its factor R stored low rank;
                                  certified dense by the QR's triangles (no SVD); the full SVD
                                  of the block (pre-reduction off); pivoted QR and the SVD of R
                                  stored dense */
  int64_t svd_path_blocks[4];  /* blocks by path */
  double svd_full_cycles[7];   /* SM cycles summed over the full-SVD blocks of
                                  compress_dense_kernel, by stage: the pivoted QR attempt, FP32
                                  sweeps on A, FP64 orthonormalisation and A V, FP32 sweeps on G,
                                  FP64 orthonormalisation and G V2, FP64 sweeps, truncation and
                                  the stores of the result */
  int64_t svd_full_blocks;     /* full-SVD blocks that ran every stage (not certified dense
                                  after the first FP32 stage) */
  int64_t svd_full_dense;      /* of those, blocks whose truncation rank exceeded half the
                                  smaller side (stored dense) */
  double svd_pre_cycles[7];    /* the same for the blocks that took the SVD of R after the
                                  pivoted-QR pre-reduction (stored low rank or dense): the QR,
                                  the five stages of the mixed SVD of R^T, truncation, recovery
                                  and stores */
  int64_t svd_pre_blocks;
} clr_profile;
int clr_profile_enable(clr_ctx_t ctx, int on);
int clr_profile_read(clr_ctx_t ctx, clr_profile* out);
/* FP64 FMA throughput of `device` measured by a short kernel of independent FMA chains on every
 * SM (the roofline of the FP64 arithmetic in recompression): *tflops = 2 x FMAs / second.
 * Synchronises the device. */
int clr_probe_fp64_rate(int device, double* tflops);
/* The bf16 term split of the split-precision products (the dense operands of a split product
 * are staged this way): x = a_0 + ... + a_{terms-1} + residual with a_0 = bf16(x) and
 * a_t = bf16(x - a_0 - ... - a_{t-1}), each rounding to nearest-even from the exact FP64
 * difference.  x: n doubles on the device (finite); out: terms x n bf16 bit patterns on the
 * device, term-major (out[t * n + i]).  terms: 2 (bf16x3) or 3 (bf16x6).  Runs on `stream`
 * (a cudaStream_t, may be null), asynchronous.  Device pointers are the caller's.  CLR_EINVAL
 * for n < 0, other term counts, null pointers with n > 0, or n > 2^40 - 512 (one launch covers
 * at most 2^31 - 1 blocks of 256 value pairs); CLR_ECUDA when the launch fails. */
int clr_split_bf16(const double* x, int64_t n, int terms, uint16_t* out, void* stream);

/* ---- allocation-free single-block compression ---------------------------------------------
 * clr_block_compress_noalloc: the truncated SVD of one m x n block at Frobenius error eps (an
 * FP64 one-sided Jacobi SVD; its result matches clr_mat_from_dense with drop threshold 0 to
 * within eps, and the rank may differ by one where the singular-value tail crosses eps), for
 * callers that must not allocate device memory: code running while a CUDA stream is being captured into a graph,
 * real-time or embedded hosts whose device memory is planned ahead, and plugins living inside a
 * framework whose allocator owns all device memory.  It calls no cudaMalloc, cudaFree or
 * allocating library routine and needs no context.  The paper has no counterpart: it is a
 * deployment variant, not part of the method.
 *   block        device pointer, m x n column-major, leading dimension ld >= m
 *   m, n         1 .. CLR_MAX_CLUSTER (256); larger sizes return CLR_EINVAL
 *   x_out, w_out device buffers for X (m x min(m,n)) and W (n x min(m,n)), column-major with
 *                leading dimensions m and n; written only when the result is low rank
 *   sigma_out    optional device buffer of min(m,n) singular values, descending
 *   status       device int32[3]: kind (CLR_KIND_*), rank, error flag: 0 ok; 3 non-finite
 *                input (the block is then reported as kind ZERO: read status[2] before
 *                trusting status[0]); 4 the Jacobi sweeps reached max_sweeps before
 *                converging (the truncation is then based on column norms that may be
 *                inexact)
 * Scratch: a fixed 1 MiB device array compiled into the library (2 x 256 x 256 doubles) that
 * every GPU loading the library holds until exit.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  That address is cached for the life of the process: after a
 * cudaDeviceReset of that device the cache is stale and the entry point must not be called
 * again.  Every call shares the array and overwrites it; calls that overlap
 * on the GPU race, so issue them on one stream (or serialise them).  Asynchronous on `stream`. */
int clr_block_compress_noalloc(int device, const double* block, int64_t ld, int m, int n,
                               double eps, int max_sweeps, double* x_out, double* w_out,
                               double* sigma_out, int32_t* status, void* stream);

/* y = A x for dense device vectors (x: n_cols, y: n_rows). */
int clr_matvec(clr_ctx_t ctx, clr_mat_t a, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CLR_H_ */
