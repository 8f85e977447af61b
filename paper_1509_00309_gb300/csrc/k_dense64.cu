// FP64 dense tile kernels: dense x dense tile products (the plain-precision form of the
// block GEMM task of Section 3.2, C_ij += A_ik B_kj), reconstruction, and per-tile kind
// bookkeeping.
//
// On GB300 FP64 runs on the CUDA cores at a small fraction of the tensor rate (~2 FMAs per clock
// per SM), so these kernels are FP64-pipe-bound and the work is cut to waste no lanes: a C tile
// (m x n, up to 256 x 256) is split into ceil(m/64) x ceil(n/64) sub-tiles of equal size (at
// most 64 x 64, so a 170-row tile gives three 57-row sub-tiles rather than two full ones and a
// 42-row one); one CTA computes a sub-tile in registers (4 x 4 per thread), walking that tile's
// dense x dense products in k order (deterministic, no atomics).  Sub-tiles are taken from a
// launch-wide counter over the tiles in decreasing cost order (longest-processing-time
// scheduling: tiles differ in size and in their number of products).
#include "clr_internal.h"

namespace clr {

constexpr int kSub = 64;      // sub-tile edge
constexpr int kKc = 16;       // k chunk staged in shared memory
constexpr int kSubPerTile = (CLR_MAX_CLUSTER / kSub) * (CLR_MAX_CLUSTER / kSub);

__global__ void __launch_bounds__(256) dd_fp64_kernel(MatView A, MatView B, MatView C, Plan p) {
  __shared__ double As[kKc][kSub + 1];
  __shared__ double Bs[kKc][kSub + 1];
  __shared__ int sh_next;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int n_items = p.counters->n_dense * kSubPerTile;
  int* sched = &p.counters->sched[3];
  for (int item = next_item(sched, &sh_next); item < n_items;
       item = next_item(sched, &sh_next)) {
    const int t = p.l_dense_s[item / kSubPerTile];
    const int s = item % kSubPerTile;
    const int I = t / p.nJ, J = t % p.nJ;
    const int mt = C.row_off[I + 1] - C.row_off[I];
    const int nt = C.col_off[J + 1] - C.col_off[J];
    // equal sub-tiles of at most kSub x kSub
    const int nsi = (mt + kSub - 1) / kSub, nsj = (nt + kSub - 1) / kSub;
    const int si = s / (CLR_MAX_CLUSTER / kSub), sj = s % (CLR_MAX_CLUSTER / kSub);
    if (si >= nsi || sj >= nsj) continue;
    const int hi = (mt + nsi - 1) / nsi, hj = (nt + nsj - 1) / nsj;
    const int i0 = si * hi, j0 = sj * hj;
    const int m = mt, n = nt;
    const int ie = min(mt, i0 + hi), je = min(nt, j0 + hj);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    const int start = p.t_start[t], count = p.t_count[t];
    for (int q = 0; q < count; ++q) {
      const Triple tr = p.triples[start + q];
      if (tr.kind != T_DD) continue;
      const int K = tr.k;
      const int k = A.col_off[K + 1] - A.col_off[K];
      const double* Ab = A.pool + slot_of(A, I, K, m);   // m x k, column-major
      const double* Bb = B.pool + slot_of(B, K, J, k);   // k x n, column-major
      for (int k0 = 0; k0 < k; k0 += kKc) {
        for (int e = tid; e < kKc * kSub; e += 256) {
          const int r = e % kSub, kk = e / kSub;
          As[kk][r] = (i0 + r < ie && k0 + kk < k) ? Ab[(i0 + r) + (int64_t)(k0 + kk) * m] : 0.0;
          const int kk2 = e % kKc, c = e / kKc;
          Bs[kk2][c] = (j0 + c < je && k0 + kk2 < k) ? Bb[(k0 + kk2) + (int64_t)(j0 + c) * k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKc; ++kk) {
          double av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
      }
    }
    double* D = C.pool + slot_of(C, I, J, m);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int r = i0 + ty + 16 * a, c = j0 + tx + 16 * b;
        if (r < ie && c < je) D[r + (int64_t)c * m] = acc[a][b];
      }
  }
}

void launch_dd_fp64(const MatView& A, const MatView& B, const MatView& C, const Plan& p,
                    int grid, cudaStream_t st) {
  dd_fp64_kernel<<<grid, 256, 0, st>>>(A, B, C, p);
}

// After planning: kinds of tiles that get no contribution (zero) or a dense accumulation.
__global__ void set_route_kinds_kernel(MatView C, Plan p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nI * p.nJ) return;
  const int route = p.t_route[t];
  const int I = t / p.nJ, J = t % p.nJ;
  const int m = C.row_off[I + 1] - C.row_off[I];
  const int n = C.col_off[J + 1] - C.col_off[J];
  if (route == ROUTE_ZERO) {
    C.kind[t] = CLR_KIND_ZERO;
    C.rank[t] = 0;
    C.norm[t] = 0.0;
  } else if (route == ROUTE_DENSE) {
    C.kind[t] = CLR_KIND_DENSE;
    C.rank[t] = m < n ? m : n;
    C.norm[t] = 0.0;  // a sum of squares when the dense kernel's epilogue forms the norms
  }
}

void launch_set_route_kinds(const MatView& C, const Plan& p, cudaStream_t st) {
  const int n = p.nI * p.nJ;
  set_route_kinds_kernel<<<(n + 127) / 128, 128, 0, st>>>(C, p);
}

// Frobenius norms of the dense-accumulated tiles (those not recompressed afterwards).
__global__ void __launch_bounds__(256) dense_tile_norms_kernel(MatView C, Plan p) {
  __shared__ double red[8];
  const int n_items = p.counters->n_dense;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int t = p.l_dense[it];
    const int I = t / p.nJ, J = t % p.nJ;
    const int m = C.row_off[I + 1] - C.row_off[I];
    const int n = C.col_off[J + 1] - C.col_off[J];
    const double* D = C.pool + slot_of(C, I, J, m);
    double s = 0.0;
    for (int e = threadIdx.x; e < m * n; e += 256) s = fma(D[e], D[e], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int i = 0; i < 8; ++i) tot += red[i];
      C.norm[t] = sqrt(tot);
    }
    __syncthreads();
  }
}

void launch_dense_tile_norms(const MatView& C, const Plan& p, cudaStream_t st) {
  dense_tile_norms_kernel<<<1024, 256, 0, st>>>(C, p);
}

__global__ void sqrt_dense_norms_kernel(MatView C, Plan p) {
  const int n_items = p.counters->n_dense;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n_items; it += gridDim.x * blockDim.x) {
    const int t = p.l_dense[it];
    C.norm[t] = sqrt(C.norm[t]);
  }
}

void launch_sqrt_dense_norms(const MatView& C, const Plan& p, cudaStream_t st) {
  sqrt_dense_norms_kernel<<<64, 256, 0, st>>>(C, p);
}

}  // namespace clr
