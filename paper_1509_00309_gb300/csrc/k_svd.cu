// K5 -- recompression of C tiles (FP64), and the truncated SVD used to build CLR matrices.
//
// Section 4.1 recompresses a low-rank sum X W^T by QR of both factors, X = Q_X R_X and
// W = Q_W R_W, a low-rank decomposition of the small core M = R_X R_W^T, and re-expansion
// X' = Q_X X_M, W' = Q_W W_M.  The decomposition of M is taken to be its SVD (the paper does
// not name it); truncation keeps the smallest rank whose Frobenius error is <= eps, with the
// singular values on the left factor (X' = Q_X U_r S_r, W' = Q_W V_r).  A block whose rank
// exceeds floor(min(m,n)/2) is stored dense.
//
// One CTA (8 warps) handles one tile:
//   Householder QR         LAPACK-style reflectors H = I - tau v v^T, v_0 = 1;
//   one-sided Jacobi SVD   Hestenes rotations on column pairs, round-robin ordering so a
//                          round's pairs are disjoint (one warp per pair), until no pair has
//                          |g_a.g_b| > tol ||g_a|| ||g_b|| or the sweep limit is reached.
// Working arrays live in the tile's workspace slot (2 m n doubles per tile, enough for
// either route).
#include <cfloat>
#include <mutex>

#include "clr_internal.h"

namespace clr {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kWarps; ++i) s += sh[i];
  __syncthreads();
  return s;
}

// In-place Householder QR of the p x q column-major matrix a (ld lda), p >= q.  R is left in
// the upper triangle, the reflector vectors (without their unit first entry) below it.
__device__ void householder_qr(double* a, int p, int q, int64_t lda, double* tau, double* sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int j = 0; j < q; ++j) {
    double* col = a + (int64_t)j * lda;
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < p; i += kThreads) part += col[i] * col[i];
    const double s = block_sum(part, sh);
    const double x0 = col[j];
    double t = 0.0, beta = x0, v0 = 1.0;
    if (s > 0.0) {
      beta = -copysign(sqrt(x0 * x0 + s), x0);
      v0 = x0 - beta;
      t = (beta - x0) / beta;
    }
    __syncthreads();
    if (s > 0.0) {
      const double inv = 1.0 / v0;
      for (int i = j + 1 + threadIdx.x; i < p; i += kThreads) col[i] *= inv;
    }
    if (threadIdx.x == 0) {
      col[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int c = j + 1 + w; c < q; c += kWarps) {
        double* y = a + (int64_t)c * lda;
        double d = 0.0;
        for (int i = j + 1 + l; i < p; i += 32) d += col[i] * y[i];
        d = warp_sum(d) + y[j];
        const double f = t * d;
        if (l == 0) y[j] -= f;
        for (int i = j + 1 + l; i < p; i += 32) y[i] -= f * col[i];
      }
    }
    __syncthreads();
  }
}

// y (p x r, ld ldy) <- Q y with Q = H_0 H_1 ... H_{q-1} from householder_qr.
__device__ void apply_q(const double* v, int p, int q, int64_t ldv, const double* tau,
                        double* y, int r, int64_t ldy) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int j = q - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      const double* vj = v + (int64_t)j * ldv;
      for (int c = w; c < r; c += kWarps) {
        double* yc = y + (int64_t)c * ldy;
        double d = 0.0;
        for (int i = j + 1 + l; i < p; i += 32) d += vj[i] * yc[i];
        d = warp_sum(d) + yc[j];
        const double f = t * d;
        if (l == 0) yc[j] -= f;
        for (int i = j + 1 + l; i < p; i += 32) yc[i] -= f * vj[i];
      }
    }
    __syncthreads();
  }
}

// One-sided Jacobi on the q columns of g (p x q, ld ldg); v (q x q, ld ldv) accumulates the
// rotations (initialised to I here unless reset_v is false).  On return g = U S and the input
// equals g v^T (times the initial v^T when v is not reset).  T is float or double; the
// convergence threshold is the type's epsilon times sqrt(p) (times tol_scale); pairs whose inner
// product is below floor2 are left alone.
template <typename T>
__device__ int jacobi_svd(T* g, int p, int q, int64_t ldg, T* v, int64_t ldv,
                          int max_sweeps, int* sh_flag, bool reset_v = true,
                          T tol_scale = T(1), T floor2 = T(0)) {
  // Column norms squared, kept in shared memory: recomputed exactly at every sweep start and
  // refreshed (fused into the rotation pass) for the two columns of every rotated pair, so a
  // pair costs one inner product unless it is rotated.
  __shared__ T nrm2[CLR_MAX_CLUSTER];
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (reset_v) {
    for (int e = threadIdx.x; e < q * q; e += kThreads)
      v[(e % q) + (int64_t)(e / q) * ldv] = (e % q == e / q) ? T(1) : T(0);
    __syncthreads();
  }
  const int qq = q + (q & 1);  // even number of slots; slot q is a dummy when q is odd
  const T eps_t = sizeof(T) == 4 ? T(FLT_EPSILON) : T(DBL_EPSILON);
  const T tol = eps_t * sqrt(T(p)) * tol_scale;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int c = w; c < q; c += kWarps) {
      const T* gc = g + (int64_t)c * ldg;
      T s2 = 0;
      for (int i = l; i < p; i += 32) s2 = fma(gc[i], gc[i], s2);
      s2 = warp_sum(s2);
      if (l == 0) nrm2[c] = s2;
    }
    if (threadIdx.x == 0) *sh_flag = 0;
    __syncthreads();
    for (int round = 0; round < qq - 1; ++round) {
      for (int k = w; k < qq / 2; k += kWarps) {
        int a, b;
        if (k == 0) {
          a = round;
          b = qq - 1;
        } else {
          a = (round + k) % (qq - 1);
          b = (round - k + (qq - 1)) % (qq - 1);
        }
        if (a >= q || b >= q) continue;
        const T al = nrm2[a], be = nrm2[b];
        const T scale = sqrt(al) * sqrt(be);
        // both columns at the noise floor: |g_a . g_b| <= scale <= floor2, nothing to do
        if (scale == T(0) || scale <= floor2) continue;
        T* ga = g + (int64_t)a * ldg;
        T* gb = g + (int64_t)b * ldg;
        T ga_gb = 0;
        for (int i = l; i < p; i += 32) ga_gb = fma(ga[i], gb[i], ga_gb);
        ga_gb = warp_sum(ga_gb);
        if (fabs(ga_gb) <= tol * scale || fabs(ga_gb) <= floor2) continue;
        const T zeta = (be - al) / (T(2) * ga_gb);
        const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T sn = c * t;
        T na = 0, nb = 0;
        for (int i = l; i < p; i += 32) {
          const T x = ga[i], y = gb[i];
          const T xa = c * x - sn * y, yb = sn * x + c * y;
          ga[i] = xa;
          gb[i] = yb;
          na = fma(xa, xa, na);
          nb = fma(yb, yb, nb);
        }
        na = warp_sum(na);
        nb = warp_sum(nb);
        T* va = v + (int64_t)a * ldv;
        T* vb = v + (int64_t)b * ldv;
        for (int i = l; i < q; i += 32) {
          const T x = va[i], y = vb[i];
          va[i] = c * x - sn * y;
          vb[i] = sn * x + c * y;
        }
        if (l == 0) {
          nrm2[a] = na;
          nrm2[b] = nb;
          *sh_flag = 1;
        }
      }
      __syncthreads();
    }
    const int rotated = *sh_flag;
    __syncthreads();
    if (!rotated) break;
  }
  return sweep;
}

struct SvdShared {
  double red[kWarps];
  double sigma[CLR_MAX_CLUSTER];    // by column
  double sorted[CLR_MAX_CLUSTER];   // descending
  int perm[CLR_MAX_CLUSTER];        // sorted position -> column
  int flag;
  int rank;
  double kept_sq;
};

// Column norms of g, their descending order, and the truncation rank at eps.
__device__ void sort_and_truncate(const double* g, int p, int q, int64_t ldg, double eps,
                                  SvdShared& sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int c = w; c < q; c += kWarps) {
    const double* gc = g + (int64_t)c * ldg;
    double s = 0.0;
    for (int i = l; i < p; i += 32) s = fma(gc[i], gc[i], s);
    s = warp_sum(s);
    if (l == 0) sh.sigma[c] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += kThreads) {
    const double sj = sh.sigma[j];
    int pos = 0;
    for (int i = 0; i < q; ++i) {
      const double si = sh.sigma[i];
      pos += (si > sj) || (si == sj && i < j);
    }
    sh.perm[pos] = j;
    sh.sorted[pos] = sj;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // smallest r with sqrt(sum_{i >= r} s_i^2) <= eps
    double tail = 0.0;
    int r = q;
    for (int i = q - 1; i >= 0; --i) {
      const double nt = tail + sh.sorted[i] * sh.sorted[i];
      if (sqrt(nt) <= eps) {
        tail = nt;
        r = i;
      } else {
        break;
      }
    }
    if (q == 0) r = 0;
    double kept = 0.0;
    for (int i = 0; i < r; ++i) kept += sh.sorted[i] * sh.sorted[i];
    sh.rank = r;
    sh.kept_sq = kept;
  }
  __syncthreads();
}

// Read-only view of the p x q working matrix: element (i, j) = src[i * s_r + j * s_c], or of its
// transpose when tr is set.
struct SrcView {
  const double* src;
  int64_t s_r, s_c;
  bool tr;
  __device__ __forceinline__ double at(int i, int j) const {
    return tr ? src[(int64_t)j * s_r + (int64_t)i * s_c] : src[(int64_t)i * s_r + (int64_t)j * s_c];
  }
};

// Mixed-precision one-sided Jacobi SVD of the p x q (p >= q) matrix A given by `a`:
//  1. FP32 sweeps on a copy (FP32 runs far faster than FP64 on this part) until converged at
//     FP32 accuracy, accumulating V32;
//  2. V = V32 orthonormalised in FP64 (modified Gram-Schmidt) and G = A V in FP64, so A and G
//     have the same singular values and G's columns are nearly orthogonal;
//  3. FP64 sweeps continuing on (G, V) -- a few from this start.
// Pairs whose inner product is below the noise floor are not rotated: p u ||A||_F in FP32, and
// max(p u ||A||_F, 1e-3 eps) in FP64 (columns that small cannot move a truncation at eps).
// On return g = U S and A = g v^T in FP64.  g (p x q doubles) also serves as the FP32 scratch
// (p q + q^2 floats).
//
// Certified dense exit (dense_h >= 0): the block is stored dense when its eps-rank exceeds
// dense_h, i.e. when the singular-value tail sqrt(sum_{i >= dense_h} s_i^2) exceeds eps.  After
// the FP32 phase every sorted column norm c_i of G32 is within delta of s_i(A), with
//   delta = 2 u32 ||A||_F (4 q sqrt(p) + p sqrt(q) + 2 s32 q + 1)
// (backward error of s32 FP32 sweeps of rotations, the rounding of A to FP32, and the residual
// non-orthogonality of G32's columns: pairs within 4 u32 sqrt(p) of orthogonal or below the FP32
// noise floor).  So tail(A) >= tail(c) - sqrt(q - dense_h) delta, and when that exceeds eps the
// FP64 phase could only confirm "dense": it is skipped and the function returns 1.
__device__ int svd_mixed(const SrcView& a, int p, int q, double* g, double* v, int max_sweeps,
                         double eps, int dense_h, double fro, SvdShared& sh,
                         unsigned long long* jstats) {
  float* g32 = reinterpret_cast<float*>(g);
  float* v32 = g32 + (int64_t)p * q;
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int e = threadIdx.x; e < p * q; e += kThreads) g32[e] = (float)a.at(e % p, e / p);
  __syncthreads();
  const float floor32 = (float)((double)p * FLT_EPSILON * fro);
  const int sw32 = jacobi_svd<float>(g32, p, q, p, v32, q, max_sweeps, &sh.flag, true, 4.0f,
                                     floor32 * floor32);
  if (dense_h >= 0 && dense_h < q) {
    for (int c = w; c < q; c += kWarps) {
      const float* gc = g32 + (int64_t)c * p;
      double s2 = 0.0;
      for (int i = l; i < p; i += 32) s2 = fma((double)gc[i], (double)gc[i], s2);
      s2 = warp_sum(s2);
      if (l == 0) sh.sigma[c] = sqrt(s2);
    }
    __syncthreads();
    double part = 0.0;
    for (int j = threadIdx.x; j < q; j += kThreads) {
      const double sj = sh.sigma[j];
      int pos = 0;
      for (int i = 0; i < q; ++i) {
        const double si = sh.sigma[i];
        pos += (si > sj) || (si == sj && i < j);
      }
      if (pos >= dense_h) part = fma(sj, sj, part);
    }
    const double tail = sqrt(block_sum(part, sh.red));
    const double delta = 2.0 * FLT_EPSILON * fro *
                         (4.0 * q * sqrt((double)p) + p * sqrt((double)q) + 2.0 * sw32 * q + 1.0);
    if (tail - sqrt((double)(q - dense_h)) * delta > eps) {
      if (jstats && threadIdx.x == 0) {
        atomicAdd(&jstats[0], 1ull);
        atomicAdd(&jstats[1], (unsigned long long)sw32);
        atomicAdd(&jstats[3], 1ull);
      }
      return 1;
    }
  }
  // FP64 refinement
  for (int e = threadIdx.x; e < q * q; e += kThreads) v[e] = (double)v32[e];
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    double* vj = v + (int64_t)j * q;
    double part = 0.0;
    for (int i = threadIdx.x; i < q; i += kThreads) part = fma(vj[i], vj[i], part);
    const double nrm = sqrt(block_sum(part, sh.red));
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = threadIdx.x; i < q; i += kThreads) vj[i] *= inv;
    __syncthreads();
    for (int k = j + 1 + w; k < q; k += kWarps) {
      double* vk = v + (int64_t)k * q;
      double d = 0.0;
      for (int i = l; i < q; i += 32) d = fma(vj[i], vk[i], d);
      d = warp_sum(d);
      for (int i = l; i < q; i += 32) vk[i] = fma(-d, vj[i], vk[i]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < p * q; e += kThreads) {
    const int i = e % p, j = e / p;
    const double* vj = v + (int64_t)j * q;
    double s2 = 0.0;
    for (int k = 0; k < q; ++k) s2 = fma(a.at(i, k), vj[k], s2);
    g[e] = s2;
  }
  __syncthreads();
  // FP64 noise floor, raised to 1e-3 eps: columns below it hold less than 1e-6 eps^2 each, so
  // their mutual (non-)orthogonality cannot move a truncation decision at eps except within a
  // hair of the threshold, while orthogonalising them costs most of the sweeps
  const double floor64 = fmax((double)p * DBL_EPSILON * fro, 1e-3 * eps);
  const int sw64 = jacobi_svd<double>(g, p, q, p, v, q, max_sweeps, &sh.flag, false, 1.0,
                                      floor64 * floor64);
  if (jstats && threadIdx.x == 0) {
    atomicAdd(&jstats[0], 1ull);
    atomicAdd(&jstats[1], (unsigned long long)sw32);
    atomicAdd(&jstats[2], (unsigned long long)sw64);
  }
  return 0;
}

// ---------------------------------------------------------------------------------------------
// ROUTE_QR tiles: X_cat (m x R) and W_cat (n x R) in the workspace slot.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) compress_qr_kernel(MatView C, const int* list,
                                                               const int* count,
                                                               const int* rsum, double* ws,
                                                               double eps, int max_sweeps,
                                                               unsigned long long* jstats) {
  __shared__ SvdShared sh;
  const int n_items = *count;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int t = list[it];
    const int I = t / C.nc, J = t % C.nc;
    const int m = C.row_off[I + 1] - C.row_off[I];
    const int n = C.col_off[J + 1] - C.col_off[J];
    const int R = rsum[t];
    const int64_t sC = slot_of(C, I, J, m);
    double* Xc = ws + 2 * sC;
    double* Wc = Xc + (int64_t)m * R;
    double* tauX = Wc + (int64_t)n * R;
    double* tauW = tauX + R;
    double* M = tauW + R;
    double* V = M + (int64_t)R * R;
    double* G = V + (int64_t)R * R;
    householder_qr(Xc, m, R, m, tauX, sh.red);
    householder_qr(Wc, n, R, n, tauW, sh.red);
    // M = R_X R_W^T (both upper triangular R x R)
    for (int e = threadIdx.x; e < R * R; e += kThreads) {
      const int a = e % R, b = e / R;
      double s = 0.0;
      for (int c = (a > b ? a : b); c < R; ++c)
        s = fma(Xc[a + (int64_t)c * m], Wc[b + (int64_t)c * n], s);
      M[e] = s;
    }
    __syncthreads();
    {
      double part = 0.0;
      for (int e = threadIdx.x; e < R * R; e += kThreads) part = fma(M[e], M[e], part);
      const double mfro = sqrt(block_sum(part, sh.red));
      SrcView mv{M, 1, R, false};
      svd_mixed(mv, R, R, G, V, max_sweeps, eps, -1, mfro, sh, jstats);
    }
    sort_and_truncate(G, R, R, R, eps, sh);
    const int r = sh.rank;
    double* Xo = C.pool + sC;
    double* Wo = Xo + (int64_t)m * r;
    for (int e = threadIdx.x; e < m * r; e += kThreads) {
      const int i = e % m, c = e / m;
      Xo[e] = i < R ? G[i + (int64_t)sh.perm[c] * R] : 0.0;
    }
    for (int e = threadIdx.x; e < n * r; e += kThreads) {
      const int j = e % n, c = e / n;
      Wo[e] = j < R ? V[j + (int64_t)sh.perm[c] * R] : 0.0;
    }
    __syncthreads();
    apply_q(Xc, m, R, m, tauX, Xo, r, m);
    apply_q(Wc, n, R, n, tauW, Wo, r, n);
    if (threadIdx.x == 0) {
      C.kind[t] = r > 0 ? CLR_KIND_LR : CLR_KIND_ZERO;
      C.rank[t] = r;
      C.norm[t] = sqrt(sh.kept_sq);
    }
    __syncthreads();
  }
}

void launch_compress_qr(const MatView& C, const int* list, const int* count, const int* rsum,
                        double* ws, double eps, int max_sweeps, int grid, int* err,
                        unsigned long long* jstats, cudaStream_t st) {
  (void)err;
  compress_qr_kernel<<<grid, kThreads, 0, st>>>(C, list, count, rsum, ws, eps, max_sweeps,
                                                 jstats);
}

// ---------------------------------------------------------------------------------------------
// Dense truncated SVD of whole blocks (ROUTE_DACC tiles, recompressed dense tiles, building a
// CLR matrix from a dense one).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) compress_dense_kernel(
    MatView C, const int* list, const int* count, const double* src, int64_t lds, double* ws,
    double eps, double drop_norm, int dense_only, int max_sweeps, int* err,
    unsigned long long* jstats) {
  __shared__ SvdShared sh;
  const int n_items = list ? *count : C.nr * C.nc;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int t = list ? list[it] : it;
    const int I = t / C.nc, J = t % C.nc;
    const int m = C.row_off[I + 1] - C.row_off[I];
    const int n = C.col_off[J + 1] - C.col_off[J];
    const int64_t sC = slot_of(C, I, J, m);
    double* slot = C.pool + sC;
    const double* S = src ? src + (int64_t)C.row_off[I] * lds + C.col_off[J] : slot;
    const int64_t s_r = src ? lds : 1;   // element (i,j) at S[i * s_r + j * s_c]
    const int64_t s_c = src ? 1 : m;
    const bool tr = m < n;
    const int p = tr ? n : m, q = tr ? m : n;
    double* G = ws + 2 * sC;             // p x q, ld p (also the FP32 scratch)
    double* V = G + (int64_t)m * n;      // q x q, ld q
    double part = 0.0;
    for (int e = threadIdx.x; e < m * n; e += kThreads) {
      int i, j;
      if (src) { i = e / n; j = e % n; } else { i = e % m; j = e / m; }
      const double x = S[i * s_r + j * s_c];
      part = fma(x, x, part);
    }
    const double nsq = block_sum(part, sh.red);
    if (!isfinite(nsq)) {
      if (threadIdx.x == 0) atomicExch(err, 3);
    }
    const double nrm = sqrt(nsq);
    int kind;
    if (!(nrm >= drop_norm) || nsq == 0.0 || !isfinite(nsq)) {
      kind = CLR_KIND_ZERO;
      if (threadIdx.x == 0) { C.kind[t] = kind; C.rank[t] = 0; C.norm[t] = 0.0; }
      __syncthreads();
      continue;
    }
    int r = q;
    if (!dense_only) {
      const SrcView view{S, s_r, s_c, tr};
      const int early_dense =
          svd_mixed(view, p, q, G, V, max_sweeps, eps, q / 2, nrm, sh, jstats);
      if (!early_dense) {
        sort_and_truncate(G, p, q, p, eps, sh);
        r = sh.rank;
      }
    }
    const int lim = q / 2;
    if (r == 0) {
      if (threadIdx.x == 0) { C.kind[t] = CLR_KIND_ZERO; C.rank[t] = 0; C.norm[t] = 0.0; }
    } else if (dense_only || r > lim) {
      if (src) {
        for (int e = threadIdx.x; e < m * n; e += kThreads) {
          const int i = e % m, j = e / m;
          slot[e] = S[i * s_r + j * s_c];
        }
      }
      if (threadIdx.x == 0) { C.kind[t] = CLR_KIND_DENSE; C.rank[t] = q; C.norm[t] = nrm; }
    } else {
      double* Xo = slot;
      double* Wo = slot + (int64_t)m * r;
      if (!tr) {
        // G = U S (m x n), V (n x n):  X = (U S)_r, W = V_r
        for (int e = threadIdx.x; e < m * r; e += kThreads) {
          const int i = e % m, c = e / m;
          Xo[e] = G[i + (int64_t)sh.perm[c] * p];
        }
        for (int e = threadIdx.x; e < n * r; e += kThreads) {
          const int j = e % n, c = e / n;
          Wo[e] = V[j + (int64_t)sh.perm[c] * q];
        }
      } else {
        // G = S^T V' = U' S (n x m): block = V' S U'^T -> X = V'_r S_r, W = U'_r
        for (int e = threadIdx.x; e < m * r; e += kThreads) {
          const int i = e % m, c = e / m;
          Xo[e] = V[i + (int64_t)sh.perm[c] * q] * sh.sorted[c];
        }
        for (int e = threadIdx.x; e < n * r; e += kThreads) {
          const int j = e % n, c = e / n;
          Wo[e] = G[j + (int64_t)sh.perm[c] * p] / sh.sorted[c];
        }
      }
      if (threadIdx.x == 0) {
        C.kind[t] = CLR_KIND_LR;
        C.rank[t] = r;
        C.norm[t] = sqrt(sh.kept_sq);
      }
    }
    __syncthreads();
  }
}

void launch_compress_dense(const MatView& C, const int* list, const int* count,
                           const double* src, int64_t lds, double* ws, double eps,
                           double drop_norm, int dense_only, int max_sweeps, int grid,
                           int* err, unsigned long long* jstats, cudaStream_t st) {
  compress_dense_kernel<<<grid, kThreads, 0, st>>>(C, list, count, src, lds, ws, eps,
                                                   drop_norm, dense_only, max_sweeps, err,
                                                   jstats);
}

// ---------------------------------------------------------------------------------------------
// Block Frobenius norms: dense directly, low rank as sqrt(sum_ab (X^T X)_ab (W^T W)_ab).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) block_norms_kernel(MatView M) {
  __shared__ double red[kWarps];
  const int t = blockIdx.x;
  const int I = t / M.nc, J = t % M.nc;
  const int m = M.row_off[I + 1] - M.row_off[I];
  const int n = M.col_off[J + 1] - M.col_off[J];
  const int kind = M.kind[t];
  const double* s = M.pool + slot_of(M, I, J, m);
  double part = 0.0;
  if (kind == CLR_KIND_DENSE) {
    for (int e = threadIdx.x; e < m * n; e += kThreads) part = fma(s[e], s[e], part);
  } else if (kind == CLR_KIND_LR) {
    const int r = M.rank[t];
    const double* X = s;
    const double* W = s + (int64_t)m * r;
    for (int e = threadIdx.x; e < r * r; e += kThreads) {
      const int a = e % r, b = e / r;
      double gx = 0.0, gw = 0.0;
      for (int i = 0; i < m; ++i) gx = fma(X[i + (int64_t)a * m], X[i + (int64_t)b * m], gx);
      for (int j = 0; j < n; ++j) gw = fma(W[j + (int64_t)a * n], W[j + (int64_t)b * n], gw);
      part = fma(gx, gw, part);
    }
  }
  const double tot = block_sum(part, red);
  if (threadIdx.x == 0) M.norm[t] = kind == CLR_KIND_ZERO ? 0.0 : sqrt(fmax(tot, 0.0));
}

// Frobenius norm of every block's slot read as a dense block (kinds not yet known).
__global__ void __launch_bounds__(kThreads) block_norms_dense_kernel(MatView M) {
  __shared__ double red[kWarps];
  const int t = blockIdx.x;
  const int I = t / M.nc, J = t % M.nc;
  const int m = M.row_off[I + 1] - M.row_off[I];
  const int n = M.col_off[J + 1] - M.col_off[J];
  const double* s = M.pool + slot_of(M, I, J, m);
  double part = 0.0;
  for (int e = threadIdx.x; e < m * n; e += kThreads) part = fma(s[e], s[e], part);
  const double tot = block_sum(part, red);
  if (threadIdx.x == 0) M.norm[t] = sqrt(tot);
}

void launch_block_norms_dense(const MatView& M, cudaStream_t st) {
  block_norms_dense_kernel<<<M.nr * M.nc, kThreads, 0, st>>>(M);
}

void launch_block_norms(const MatView& M, cudaStream_t st) {
  block_norms_kernel<<<M.nr * M.nc, kThreads, 0, st>>>(M);
}

// alpha * M in place: dense values or the X factor, and the norms.
__global__ void scale_blocks_kernel(MatView M, double alpha) {
  const int t = blockIdx.x;
  const int I = t / M.nc, J = t % M.nc;
  const int m = M.row_off[I + 1] - M.row_off[I];
  const int n = M.col_off[J + 1] - M.col_off[J];
  const int kind = M.kind[t];
  double* s = M.pool + slot_of(M, I, J, m);
  int64_t len = kind == CLR_KIND_DENSE ? (int64_t)m * n
              : kind == CLR_KIND_LR ? (int64_t)m * M.rank[t] : 0;
  for (int64_t e = threadIdx.x; e < len; e += blockDim.x) s[e] *= alpha;
  if (threadIdx.x == 0) M.norm[t] *= fabs(alpha);
}

void launch_scale_blocks(const MatView& M, double alpha, cudaStream_t st) {
  scale_blocks_kernel<<<M.nr * M.nc, 256, 0, st>>>(M, alpha);
}

}  // namespace clr

// =============================================================================================
// Allocation-free truncated SVD of one block (clr_block_compress_noalloc).
//
// Same computation as compress_dense_kernel for a single block, but its working memory (the
// block copy G and the rotation matrix V) lives in a fixed file-scope device array instead of a
// caller- or context-allocated workspace, so the entry point never allocates.  The array holds
// CLR_MAX_CLUSTER^2 doubles for G and as many for V (1 MiB), is loaded with every GPU that
// loads this library, and is shared by every call: G is fully rewritten and V reset to the
// identity by each call, so no stale contents are read, but calls that overlap on the GPU
// (different streams, concurrent host threads) race on it.
// =============================================================================================
namespace clr {
namespace {

constexpr int64_t kNoAllocScratchDoubles = 2LL * CLR_MAX_CLUSTER * CLR_MAX_CLUSTER;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// status[0] = kind, status[1] = rank, status[2] = error flag (3: non-finite input)
__global__ void __launch_bounds__(kThreads) compress_block_noalloc_kernel(
    const double* src, int64_t lds, int m, int n, double eps, int max_sweeps, double* scratch,
    double* x_out, double* w_out, double* sigma_out, int* status) {
  __shared__ SvdShared sh;
  const bool tr = m < n;
  const int p = tr ? n : m, q = tr ? m : n;
  double* G = scratch;                                   // p x q, ld p
  double* V = scratch + (int64_t)CLR_MAX_CLUSTER * CLR_MAX_CLUSTER;  // q x q, ld q
  double part = 0.0;
  for (int e = threadIdx.x; e < m * n; e += kThreads) {
    const int i = e % m, j = e / m;
    const double x = src[i + (int64_t)j * lds];
    part = fma(x, x, part);
    if (tr) G[j + (int64_t)i * p] = x; else G[i + (int64_t)j * p] = x;
  }
  const double nsq = block_sum(part, sh.red);
  if (threadIdx.x == 0) status[2] = isfinite(nsq) ? 0 : 3;
  if (!isfinite(nsq) || nsq == 0.0) {
    if (threadIdx.x == 0) { status[0] = CLR_KIND_ZERO; status[1] = 0; }
    return;
  }
  jacobi_svd(G, p, q, p, V, q, max_sweeps, &sh.flag);
  sort_and_truncate(G, p, q, p, eps, sh);
  const int r = sh.rank;
  if (sigma_out)
    for (int c = threadIdx.x; c < q; c += kThreads) sigma_out[c] = sh.sorted[c];
  if (r == 0) {
    if (threadIdx.x == 0) { status[0] = CLR_KIND_ZERO; status[1] = 0; }
    return;
  }
  if (r > q / 2) {
    if (threadIdx.x == 0) { status[0] = CLR_KIND_DENSE; status[1] = q; }
    return;
  }
  if (!tr) {
    for (int e = threadIdx.x; e < m * r; e += kThreads)
      x_out[e] = G[(e % m) + (int64_t)sh.perm[e / m] * p];
    for (int e = threadIdx.x; e < n * r; e += kThreads)
      w_out[e] = V[(e % n) + (int64_t)sh.perm[e / n] * q];
  } else {
    for (int e = threadIdx.x; e < m * r; e += kThreads)
      x_out[e] = V[(e % m) + (int64_t)sh.perm[e / m] * q] * sh.sorted[e / m];
    for (int e = threadIdx.x; e < n * r; e += kThreads)
      w_out[e] = G[(e % n) + (int64_t)sh.perm[e / n] * p] / sh.sorted[e / n];
  }
  if (threadIdx.x == 0) { status[0] = CLR_KIND_LR; status[1] = r; }
}

}  // namespace
}  // namespace clr

extern "C" int clr_block_compress_noalloc(int device, const double* block, int64_t ld, int m,
                                          int n, double eps, int max_sweeps, double* x_out,
                                          double* w_out, double* sigma_out, int32_t* status,
                                          void* stream) {
  using namespace clr;
  if (!block || !x_out || !w_out || !status) return CLR_EINVAL;
  if (m < 1 || n < 1 || m > CLR_MAX_CLUSTER || n > CLR_MAX_CLUSTER) return CLR_EINVAL;
  if (ld < m || !(eps >= 0.0) || max_sweeps < 1) return CLR_EINVAL;
  if (device < 0 || device >= kNoAllocMaxDevices) return CLR_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return CLR_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return CLR_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        if (prev != device) cudaSetDevice(prev);
        return CLR_ECUDA;
      }
      g_noalloc_ptr[device] = (double*)ptr;
    }
    scratch = g_noalloc_ptr[device];
  }
  compress_block_noalloc_kernel<<<1, kThreads, 0, (cudaStream_t)stream>>>(
      block, ld, m, n, eps, max_sweeps, scratch, x_out, w_out, sigma_out, (int*)status);
  const cudaError_t e = cudaGetLastError();
  if (prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? CLR_OK : CLR_ECUDA;
}
