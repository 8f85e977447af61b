// K0 -- the product's work list.
//
// The paper's task-based SUMMA (Section 3.2) issues one multiply task per (i,k,j) block
// triple and reduces the partial products into C_ij; on one GPU that task graph becomes a
// triple list built on the device, sorted by C tile (then by k) so that one CTA can own each
// C tile and accumulate its products without atomics (the GEMM-update case of Section 3.2).
// Tiles are screened with the Frobenius-norm estimate of Section 4.1.
#include "clr_internal.h"

namespace clr {

__device__ __forceinline__ int out_rank(int kind, int ra, int rb) {
  // Section 4.1, Eq. 1: Z = W_A^T X_B is contracted on the side of smaller output rank.
  if (kind == T_DL) return rb;
  if (kind == T_LD) return ra;
  if (kind == T_LL) return rb <= ra ? rb : ra;
  return 0;
}

__device__ __forceinline__ unsigned long long triple_flops(int kind, long long m, long long k,
                                                           long long n, long long ra,
                                                           long long rb) {
  if (kind == T_DD) return 2ull * m * k * n;
  if (kind == T_DL) return 2ull * m * k * rb;
  if (kind == T_LD) return 2ull * k * n * ra;
  return 2ull * k * ra * rb + (rb <= ra ? 2ull * m * ra * rb : 2ull * n * ra * rb);
}

// One warp per C tile (I, J), its lanes over the inner clusters K.
// gemm_dacc_bound > 0 (split precision): a tile that would be accumulated densely in FP64
// (ROUTE_DACC) is summed by the tensor-core GEMM instead (ROUTE_DACC_G) when its norm estimate
// sum_K ||A_IK|| ||B_KJ|| is at most gemm_dacc_bound = eps / (16 u_split).
// oz.sa non-null (exact slices): the same when the estimate of the sliced sum's error,
// from the exponents of the tile's rows and columns per K segment, sum over segments
// s of sa[I][s] sb[J][s] (sa[I][s] = sum over rows i of I of 4^e_is), is at most oz.bound2.
__global__ void plan_count_kernel(MatView A, MatView B, Plan p, double eps_sp,
                                  double gemm_dacc_bound, OzDaccRule oz) {
  const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32);
  const int lane = threadIdx.x % 32;
  if (t >= p.nI * p.nJ) return;  // the whole warp
  const int I = t / p.nJ, J = t % p.nJ;
  const int m = A.row_off[I + 1] - A.row_off[I];
  const int n = B.col_off[J + 1] - B.col_off[J];
  bool pass = true;
  double est = 0.0;
  if (eps_sp > 0.0 || gemm_dacc_bound > 0.0) {
    for (int K = lane; K < p.nK; K += 32) {
      const int ka = A.kind[I * A.nc + K], kb = B.kind[K * B.nc + J];
      if (ka != CLR_KIND_ZERO && kb != CLR_KIND_ZERO)
        est += A.norm[I * A.nc + K] * B.norm[K * B.nc + J];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) est += __shfl_xor_sync(0xffffffffu, est, o);
    if (eps_sp > 0.0) pass = est > eps_sp * (double)m * (double)n;
  }
  int count = 0, has_dd = 0, rsum = 0;
  unsigned long long fl = 0;
  int byk[4] = {0, 0, 0, 0};
  if (pass) {
    for (int K = lane; K < p.nK; K += 32) {
      const int ka = A.kind[I * A.nc + K], kb = B.kind[K * B.nc + J];
      if (ka == CLR_KIND_ZERO || kb == CLR_KIND_ZERO) continue;
      const int kind = (ka == CLR_KIND_DENSE ? 0 : 2) + (kb == CLR_KIND_DENSE ? 0 : 1);
      const int ra = A.rank[I * A.nc + K], rb = B.rank[K * B.nc + J];
      const int k = A.col_off[K + 1] - A.col_off[K];
      ++count;
      byk[kind]++;
      fl += triple_flops(kind, m, k, n, ra, rb);
      if (kind == T_DD) has_dd = 1; else rsum += out_rank(kind, ra, rb);
    }
  }
  count = __reduce_add_sync(0xffffffffu, (unsigned)count);
  rsum = __reduce_add_sync(0xffffffffu, (unsigned)rsum);
  has_dd = __any_sync(0xffffffffu, has_dd);
#pragma unroll
  for (int q = 0; q < 4; ++q) byk[q] = __reduce_add_sync(0xffffffffu, (unsigned)byk[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
  if (lane != 0) return;
  int route = ROUTE_ZERO;
  if (count > 0) {
    int lim = (m < n ? m : n) / 2;
    route = has_dd ? ROUTE_DENSE : (rsum <= lim ? ROUTE_QR : ROUTE_DACC);
    if (route == ROUTE_DACC && gemm_dacc_bound > 0.0 && est <= gemm_dacc_bound) {
      route = ROUTE_DACC_G;
      atomicAdd(&p.counters->n_gemm_dacc, 1ull);
    }
    if (route == ROUTE_DACC && oz.sa) {
      double e2 = 0.0;
      for (int sg = 0; sg < oz.n_seg; ++sg)
        e2 += oz.sa[(int64_t)I * oz.n_seg + sg] * oz.sb[(int64_t)J * oz.n_seg + sg];
      if (e2 <= oz.bound2) {
        route = ROUTE_DACC_G;
        atomicAdd(&p.counters->n_gemm_dacc, 1ull);
      }
    }
  }
  p.t_count[t] = count;
  p.t_route[t] = route;
  p.t_rsum[t] = rsum;
  if (count > 0) {
    atomicAdd(&p.counters->n_triples, (unsigned long long)count);
    for (int q = 0; q < 4; ++q)
      if (byk[q]) atomicAdd(&p.counters->by_kind[q], (unsigned long long)byk[q]);
    atomicAdd(&p.counters->flops, fl);
    atomicAdd(&p.counters->by_mode[has_dd ? 1 : 2], 1ull);
    if (!has_dd) atomicMax(&p.counters->max_rsum, (unsigned long long)rsum);
  } else {
    atomicAdd(&p.counters->by_mode[0], 1ull);
  }
}

// Single-CTA scan: t_start = exclusive prefix sum of t_count, plus the tile lists in tile
// order.  Tile counts are at most a few hundred thousand, so one CTA of 1024 threads walking
// contiguous chunks is enough.
constexpr int kScanThreads = 1024;
constexpr int kScanQ = 5;
constexpr int kCostBuckets = 32;

// log2 bucket of a tile's cost (which = 0: QR route recompression, 1: dense SVD, 2: dense x
// dense products, m n times the tile's number of products).  A dense recompression's cost
// depends on the path the tile takes (dense certificate ~0.4, pivoted QR and the SVD of R
// ~1.1 when stored low rank and ~2 when stored dense, SM cycles per m n min(m, n) on the
// lattice iterates), known only once it ran: the cycles
// measured the last time a tile of this matrix was recompressed (Newton-Schulz reuses its
// matrices for the same products every iteration) replace the size estimate (2 m n min(m, n)
// cycles) when present.
__device__ __forceinline__ int cost_bucket(const Plan& p, int t, int which) {
  const int I = t / p.nJ, J = t % p.nJ;
  const long long m = p.row_off[I + 1] - p.row_off[I];
  const long long n = p.col_off[J + 1] - p.col_off[J];
  long long c;
  if (which == 0) {
    const long long R = p.t_rsum[t];
    c = (m + n) * R * R + R * R * R;
  } else if (which == 1) {
    const unsigned kc = p.c_cost ? p.c_cost[t] : 0u;
    c = kc ? (long long)kc << 10 : 2 * m * n * (m < n ? m : n);
  } else {
    c = m * n * (long long)p.t_count[t];
  }
  const int b = c > 0 ? 63 - __clzll(c) : 0;
  return b < kCostBuckets ? b : kCostBuckets - 1;
}

__global__ void __launch_bounds__(kScanThreads) plan_scan_kernel(Plan p, int recompress_dense) {
  __shared__ int sh[kScanQ][kScanThreads];
  const int n = p.nI * p.nJ;
  const int tid = threadIdx.x;
  const int chunk = (n + kScanThreads - 1) / kScanThreads;
  const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
  int s[kScanQ] = {0, 0, 0, 0, 0};
  for (int i = lo; i < hi; ++i) {
    int route = p.t_route[i];
    s[0] += p.t_count[i];
    s[1] += route == ROUTE_DENSE;
    s[2] += p.t_rsum[i] > 0;
    s[3] += route == ROUTE_QR;
    s[4] += route == ROUTE_DACC || route == ROUTE_DACC_G ||
            (route == ROUTE_DENSE && recompress_dense);
  }
  for (int q = 0; q < kScanQ; ++q) sh[q][tid] = s[q];
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partial sums.
  for (int off = 1; off < kScanThreads; off <<= 1) {
    int v[kScanQ];
    for (int q = 0; q < kScanQ; ++q) v[q] = tid >= off ? sh[q][tid - off] : 0;
    __syncthreads();
    for (int q = 0; q < kScanQ; ++q) sh[q][tid] += v[q];
    __syncthreads();
  }
  int base[kScanQ];
  for (int q = 0; q < kScanQ; ++q) base[q] = sh[q][tid] - s[q];
  for (int i = lo; i < hi; ++i) {
    int route = p.t_route[i];
    p.t_start[i] = base[0];
    base[0] += p.t_count[i];
    if (route == ROUTE_DENSE) p.l_dense[base[1]++] = i;
    if (p.t_rsum[i] > 0) p.l_lr[base[2]++] = i;
    if (route == ROUTE_QR) p.l_qr[base[3]++] = i;
    if (route == ROUTE_DACC || route == ROUTE_DACC_G ||
        (route == ROUTE_DENSE && recompress_dense))
      p.l_dcomp[base[4]++] = i;
  }
  if (tid == kScanThreads - 1) {
    p.counters->n_dense = sh[1][tid];
    p.counters->n_lr = sh[2][tid];
    p.counters->n_qr = sh[3][tid];
    p.counters->n_dcomp = sh[4][tid];
    p.counters->n_dacc = 0;
  }
  // The recompression lists and the dense-product list again, largest cost first
  // (longest-processing-time order for the dynamically distributed kernels): a counting sort on
  // log2 of the cost, m n min(m, n) for a dense SVD, (m + n) R^2 for a QR route, m n times the
  // number of products for dense x dense products.  The order within a bucket is immaterial:
  // every tile is processed independently.
  __syncthreads();
  const int n_qr = sh[3][kScanThreads - 1], n_dc = sh[4][kScanThreads - 1];
  const int n_de = sh[1][kScanThreads - 1];
  __shared__ int bcount[3][kCostBuckets], boff[3][kCostBuckets];
  if (tid < 3 * kCostBuckets) (&bcount[0][0])[tid] = 0;
  __syncthreads();
  auto item = [&](int i, int* which) {
    *which = i < n_qr ? 0 : (i < n_qr + n_dc ? 1 : 2);
    return *which == 0 ? p.l_qr[i] : *which == 1 ? p.l_dcomp[i - n_qr]
                                                  : p.l_dense[i - n_qr - n_dc];
  };
  for (int i = tid; i < n_qr + n_dc + n_de; i += kScanThreads) {
    int which;
    const int t = item(i, &which);
    atomicAdd(&bcount[which][cost_bucket(p, t, which)], 1);
  }
  __syncthreads();
  if (tid < 3) {
    int acc = 0;
    for (int b = kCostBuckets - 1; b >= 0; --b) {
      boff[tid][b] = acc;
      acc += bcount[tid][b];
    }
  }
  __syncthreads();
  for (int i = tid; i < n_qr + n_dc + n_de; i += kScanThreads) {
    int which;
    const int t = item(i, &which);
    const int pos = atomicAdd(&boff[which][cost_bucket(p, t, which)], 1);
    (which == 0 ? p.l_qr_s : which == 1 ? p.l_dcomp_s : p.l_dense_s)[pos] = t;
  }
}

// One warp per C tile: its lanes take 32 inner clusters at a time; a ballot gives each
// nonzero triple its place (K order) and a warp scan of the output ranks its first factor
// column in the tile's concatenation.
__global__ void plan_fill_kernel(MatView A, MatView B, Plan p) {
  const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32);
  const int lane = threadIdx.x % 32;
  if (t >= p.nI * p.nJ) return;  // the whole warp
  if (p.t_count[t] == 0) return;
  const int I = t / p.nJ, J = t % p.nJ;
  int64_t pos = p.t_start[t];
  int col = 0;
  for (int K0 = 0; K0 < p.nK; K0 += 32) {
    const int K = K0 + lane;
    int ka = CLR_KIND_ZERO, kb = CLR_KIND_ZERO;
    if (K < p.nK) {
      ka = A.kind[I * A.nc + K];
      kb = B.kind[K * B.nc + J];
    }
    const bool on = ka != CLR_KIND_ZERO && kb != CLR_KIND_ZERO;
    const unsigned mask = __ballot_sync(0xffffffffu, on);
    const int kind = (ka == CLR_KIND_DENSE ? 0 : 2) + (kb == CLR_KIND_DENSE ? 0 : 1);
    const int r = on ? out_rank(kind, A.rank[I * A.nc + K], B.rank[K * B.nc + J]) : 0;
    int incl = r;  // inclusive prefix sum of the output ranks over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (on) {
      Triple tr;
      tr.tile = t;
      tr.k = K;
      tr.kind = kind;
      tr.col = col + incl - r;
      const int64_t at = pos + __popc(mask & ((1u << lane) - 1u));
      if (at < p.max_triples) p.triples[at] = tr; else atomicCAS(&p.counters->err, 0, 2);
    }
    pos += __popc(mask);
    col += __shfl_sync(0xffffffffu, incl, 31);
  }
}

void launch_plan_scan(const Plan& p, int recompress_dense, cudaStream_t st) {
  plan_scan_kernel<<<1, kScanThreads, 0, st>>>(p, recompress_dense);
}

void launch_plan(const MatView& A, const MatView& B, const Plan& p, double eps_sp,
                 int recompress_dense, double gemm_dacc_bound, const OzDaccRule& oz,
                 cudaStream_t st) {
  const int n = p.nI * p.nJ;
  const int threads = 128;  // 4 tiles per block: one warp each
  const int blocks = (int)(((int64_t)n * 32 + threads - 1) / threads);
  cudaMemsetAsync(p.counters, 0, kPlanCountersClear, st);
  plan_count_kernel<<<blocks, threads, 0, st>>>(A, B, p, eps_sp, gemm_dacc_bound, oz);
  plan_scan_kernel<<<1, kScanThreads, 0, st>>>(p, recompress_dense);
  plan_fill_kernel<<<blocks, threads, 0, st>>>(A, B, p);
}

}  // namespace clr
