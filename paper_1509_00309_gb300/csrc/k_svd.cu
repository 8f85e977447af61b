// K5 -- recompression of C tiles (FP64), and the truncated SVD used to build CLR matrices.
//
// Section 4.1 recompresses a low-rank sum X W^T by QR of both factors, X = Q_X R_X and
// W = Q_W R_W, a low-rank decomposition of the small core M = R_X R_W^T, and re-expansion
// X' = Q_X X_M, W' = Q_W W_M.  The decomposition of M is taken to be its SVD (the paper does
// not name it); truncation keeps the smallest rank whose Frobenius error is <= eps, with the
// singular values on the left factor (X' = Q_X U_r S_r, W' = Q_W V_r).  A block whose rank
// exceeds floor(min(m,n)/2) is stored dense.
//
// One CTA (16 warps) handles one tile at a time, taking tiles from a launch-wide counter:
//   Householder QR         LAPACK-style reflectors H = I - tau v v^T, v_0 = 1;
//   one-sided Jacobi SVD   Hestenes rotations on column pairs, round-robin ordering so a
//                          round's pairs are disjoint (one warp per pair), until no pair has
//                          |g_a.g_b| > tol ||g_a|| ||g_b|| or the sweep limit is reached
//                          (mixed FP32/FP64 stages, svd_mixed);
//   rank-revealing QR      the paper's construction for building from dense (option).
// FP64 working arrays live in the tile's workspace slot (2 m n doubles per tile, enough for
// either route); the FP32 copies of the mixed-precision SVD in a per-CTA scratch (L1-cached).
#include <cfloat>
#include <mutex>

#include "clr_internal.h"

namespace clr {

constexpr int kThreads = 512;
// index of the per-path cycle counters in the profiling counters (third block of 8)
constexpr int kPathCounters = 16;
// compress_dense_kernel's full-SVD stages while profiling (block 3 of the counters): cycles of
// the pivoted QR attempt, the five stages of svd_mixed, truncation and stores; then the count
constexpr int kFullStageCounters = 24;
// the same for the pre-reduced path (block 4): the QR, the five stages of svd_mixed on R^T,
// truncation, recovery and the factors' stores; then the count
constexpr int kPreStageCounters = 32;
constexpr int kWarps = kThreads / 32;
constexpr int kFp64SweepCap = 0;  // FP64 sweeps of svd_mixed when the right factor is recovered

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

// Per-pair arithmetic of the Jacobi sweeps.  FP64 runs at 1/64 of the FP32 rate on this part
// and each FP64 instruction of a warp occupies its sub-partition's FP64 pipe for many cycles,
// so the scalar steps avoid FP64 square roots and most divisions: the tests compare squares,
// the rotation's tangent t is found in FP32 from zeta (its accuracy only sets how far one
// rotation reduces the pair's inner product) and c = (1 + t^2)^-1/2 is refined in FP64 by two
// Newton steps from the FP32 seed, so that c^2 + s^2 = 1 to FP64 rounding and the rotation is
// orthogonal.
// In FP32 the hardware approximations (a few ulp) serve throughout: the FP32 stages only find
// rotations that the FP64 stages apply and refine.
__device__ __forceinline__ float rt_sqrt(float x) {
  return x > 0.f ? (x <= FLT_MAX ? x * rsqrtf(x) : x) : 0.f;
}

__device__ __forceinline__ bool pair_below_floor(float al, float be, float f2) {
  const float s = rt_sqrt(al * be);
  return s == 0.f || s <= f2;
}
__device__ __forceinline__ bool pair_below_floor(double al, double be, double f2) {
  const double p2 = al * be;
  return p2 == 0.0 || p2 <= f2 * f2;
}

// |g| <= tol |g_a| |g_b| or |g| <= floor2
__device__ __forceinline__ bool pair_converged(float al, float be, float g, float tol, float f2) {
  const float s = rt_sqrt(al * be);
  return fabsf(g) <= tol * s || fabsf(g) <= f2;
}
__device__ __forceinline__ bool pair_converged(double al, double be, double g, double tol,
                                               double f2) {
  const double g2 = g * g;
  return g2 <= tol * tol * (al * be) || g2 <= f2 * f2;
}

// Rutishauser's rotation: zeta = (b - a) / 2g, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t.
// (for |zeta| > 2^40, where zeta^2 may overflow, the asymptote 1 / (2 zeta))
__device__ __forceinline__ float tangent_of(float zeta) {
  if (fabsf(zeta) > 0x1p40f) return __fdividef(0.5f, zeta);
  return copysignf(__fdividef(1.f, fabsf(zeta) + rt_sqrt(1.f + zeta * zeta)), zeta);
}
__device__ __forceinline__ float rot_tangent(float d, float g) {
  return tangent_of(__fdividef(d, 2.f * g));
}
__device__ __forceinline__ void rotation(float al, float be, float g, float& c, float& s,
                                         float& t) {
  t = rot_tangent(be - al, g);
  c = rsqrtf(1.f + t * t);
  s = c * t;
}
__device__ __forceinline__ void rotation(double al, double be, double g, double& c, double& s,
                                         double& t) {
  // zeta in FP64 (the operands may lie far outside the FP32 range).  For a large angle
  // (|cos| > 1e-3: the first sweeps of a fresh start, nearly parallel columns) the tangent in
  // FP64, since a rotation that is off by u32 there leaves a leak that is large relative to the
  // smaller column; for the small angles of a refinement in FP32 where |zeta| < 2^100, else its
  // asymptote 1 / (2 zeta).
  const double zeta = (be - al) / (2.0 * g);
  if (g * g > 1e-6 * (al * be)) {
    t = copysign(1.0 / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0))), zeta);
  } else if (fabs(zeta) < 0x1p100) {
    t = (double)tangent_of((float)zeta);
  } else {
    t = 0.5 / zeta;
  }
  const double u = fma(t, t, 1.0);
  double r = (double)rsqrtf((float)u);
  r = r * fma(-0.5 * u, r * r, 1.5);
  r = r * fma(-0.5 * u, r * r, 1.5);
  c = r;
  s = r * t;
}

// One-sided Jacobi on the q columns of g (p x q, ld ldg); v (q x q, ld ldv) accumulates the
// rotations (initialised to I here unless reset_v is false; not accumulated when v is null).
// On return g = U S and the input
// equals g v^T (times the initial v^T when v is not reset).  T is float or double; the
// convergence threshold is the type's epsilon times sqrt(p) (times tol_scale); pairs whose inner
// product is below floor2 are left alone.
// A pair found converged (or below the floor) is checked again only once one of its columns has
// been rotated: each pair meets at the same round of every sweep (cyclic round-robin order), so
// when neither column has been rotated since the pair's check one sweep earlier, its inner
// product is the one that check computed and the pair is skipped.  Late sweeps, and the
// refinement of columns that are already orthogonal to each other, then touch only the pairs
// of recently rotated columns.
template <typename T>
__device__ int jacobi_svd(T* g, int p, int q, int64_t ldg, T* v, int64_t ldv,
                          int max_sweeps, int* sh_flag, bool reset_v = true,
                          T tol_scale = T(1), T floor2 = T(0)) {
  // Column norms squared, kept in shared memory: recomputed exactly at every sweep start and
  // refreshed (fused into the rotation pass) for the two columns of every rotated pair, so a
  // pair costs one inner product unless it is rotated.
  __shared__ T nrm2[CLR_MAX_CLUSTER];
  // per column: the step (sweep * (qq - 1) + round) of its last rotation, -1 if none
  __shared__ int last_rot[CLR_MAX_CLUSTER];
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (reset_v && v) {
    for (int e = threadIdx.x; e < q * q; e += kThreads)
      v[(e % q) + (int64_t)(e / q) * ldv] = (e % q == e / q) ? T(1) : T(0);
    __syncthreads();
  }
  const int qq = q + (q & 1);  // even number of slots; slot q is a dummy when q is odd
  const T eps_t = sizeof(T) == 4 ? T(FLT_EPSILON) : T(DBL_EPSILON);
  const T tol = eps_t * sqrt(T(p)) * tol_scale;
  for (int c = threadIdx.x; c < q; c += kThreads) last_rot[c] = -1;
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
          a = round + k;
          if (a >= qq - 1) a -= qq - 1;
          b = round - k;
          if (b < 0) b += qq - 1;
        }
        if (a >= q || b >= q) continue;
        const int step = sweep * (qq - 1) + round;
        // neither column rotated since this pair's check one sweep ago (step - (qq - 1))
        if (sweep > 0 && last_rot[a] < step - (qq - 1) && last_rot[b] < step - (qq - 1))
          continue;
        const T al = nrm2[a], be = nrm2[b];
        // both columns at the noise floor: |g_a . g_b| <= |g_a| |g_b| <= floor2, nothing to do
        if (pair_below_floor(al, be, floor2)) continue;
        T* ga = g + (int64_t)a * ldg;
        T* gb = g + (int64_t)b * ldg;
        // The working copies live in global scratch (L2 for the largest blocks): the two
        // columns stay in registers between the inner product and the rotation, and in FP32
        // the two columns of v are fetched before the rotation is formed, so that their latency
        // overlaps it (in FP64 the registers that takes would spill)
        constexpr int kPer = CLR_MAX_CLUSTER / 32;
        constexpr bool kPrefetchV = sizeof(T) == 4;
        T xa[kPer], xb[kPer];
        T ga_gb = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int i = l + 32 * j;
          xa[j] = i < p ? ga[i] : T(0);
          xb[j] = i < p ? gb[i] : T(0);
          ga_gb = fma(xa[j], xb[j], ga_gb);
        }
        ga_gb = warp_sum(ga_gb);
        if (pair_converged(al, be, ga_gb, tol, floor2)) continue;
        T* va = v ? v + (int64_t)a * ldv : nullptr;
        T* vb = v ? v + (int64_t)b * ldv : nullptr;
        T ya[kPrefetchV ? kPer : 1], yb[kPrefetchV ? kPer : 1];
        if constexpr (kPrefetchV) {
          if (v) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
              const int i = l + 32 * j;
              ya[j] = i < q ? va[i] : T(0);
              yb[j] = i < q ? vb[i] : T(0);
            }
          }
        }
        T c, sn, t;
        rotation(al, be, ga_gb, c, sn, t);
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int i = l + 32 * j;
          if (i < p) {
            ga[i] = c * xa[j] - sn * xb[j];
            gb[i] = sn * xa[j] + c * xb[j];
          }
        }
        // new squared norms: a - t g and b + t g exactly; recomputed from the rotated columns
        // when the update cancels (a column losing more than 63/64 of its square)
        T na = al - t * ga_gb, nb = be + t * ga_gb;
        if (!(na > al * T(0.015625)) || !(nb > be * T(0.015625))) {
          __syncwarp();
          T sa = 0, sb = 0;
          for (int i = l; i < p; i += 32) {
            sa = fma(ga[i], ga[i], sa);
            sb = fma(gb[i], gb[i], sb);
          }
          na = warp_sum(sa);
          nb = warp_sum(sb);
        }
        if (v) {
          if constexpr (kPrefetchV) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
              const int i = l + 32 * j;
              if (i < q) {
                va[i] = c * ya[j] - sn * yb[j];
                vb[i] = sn * ya[j] + c * yb[j];
              }
            }
          } else {
            for (int i = l; i < q; i += 32) {
              const T x = va[i], y = vb[i];
              va[i] = c * x - sn * y;
              vb[i] = sn * x + c * y;
            }
          }
        }
        if (l == 0) {
          nrm2[a] = na;
          nrm2[b] = nb;
          last_rot[a] = step;
          last_rot[b] = step;
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
  int v_tracked;  // svd_mixed: 1 when v holds the right singular vectors (else recover_right)
  int ls_recover; // svd_mixed: 1 when G's kept columns may be non-orthogonal (FP64 sweep cap
                  // reached): the right factor needs the least-squares form (ls_solve)
  int rank;
  double kept_sq;
  // pivoted QR pre-reduction (compress_by_pivoted_qr): reflector coefficients and column order
  double qr_tau[CLR_MAX_CLUSTER];
  int qr_perm[CLR_MAX_CLUSTER];
  int qr_pivot;
  double cert;    // tail_lower_bound_sq's result
  // compress_by_pivoted_qr: each column's trailing norm^2 when it was last summed exactly (the
  // downdated norms are recomputed once they fall below kDowndateFloor of it), and the FMAs
  // of those recomputations
  double qr_nref[CLR_MAX_CLUSTER];
  unsigned long long qr_recomputed;
};
// Downdated column norms^2 are summed again exactly once they fall below this fraction of the
// last exact value: a downdate nu'^2 = nu^2 - r^2 carries an absolute error of a few u nu_ref^2,
// so the relative error stays below ~1e-9 between recomputations.
constexpr double kDowndateFloor = 1e-6;

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

// v (q x q, ld q) <- the columns of the FP32 matrix v32 orthonormalised in FP64 (modified
// Gram-Schmidt).
__device__ void orthonormalise_fp64(const float* v32, double* v, int q, SvdShared& sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
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
}

// g (p x q, ld p) = A v in FP64 (register-tiled, cta_gemm_tiled).
__device__ void project_fp64(const SrcView& a, int p, int q, const double* v, double* g) {
  const int64_t a_i = a.tr ? a.s_c : a.s_r, a_k = a.tr ? a.s_r : a.s_c;
  cta_gemm_tiled<kThreads>(p, q, q, a.src, a_i, a_k, v, 1, q, g, p, false);
  __syncthreads();
}

// y (q x r, ld q) = A^T G_r in FP64, G_r the r kept columns of g (p x q, ld p) in the order
// perm; with G_r = U_r S_r this is V_r S_r^2.  G_r is first gathered into `gather` (p r
// doubles, not overlapping g or y) so that the product runs register-tiled.
__device__ void recover_right(const SrcView& a, int p, int q, const double* g, const int* perm,
                              int r, double* y, double* gather) {
  for (int e = threadIdx.x; e < p * r; e += kThreads) {
    const int k = e % p, c = e / p;
    gather[e] = g[k + (int64_t)perm[c] * p];
  }
  __syncthreads();
  // y(j, c) = sum_k A(k, j) G_r(k, c)
  const int64_t a_j = a.tr ? a.s_r : a.s_c, a_k = a.tr ? a.s_c : a.s_r;
  cta_gemm_tiled<kThreads>(q, r, p, a.src, a_j, a_k, gather, 1, p, y, q, false);
  __syncthreads();
}

// y (q x r, ld q) <- y (G_r^T G_r)^-1 in FP64, G_r the r kept columns of g (p x q, ld p) in the
// order perm, with norms d: the least-squares right factor when G_r is not orthogonal to FP64
// precision.  The Gram matrix of the normalised columns (unit diagonal, off-diagonal at the
// FP32 stages' tolerance, so well conditioned) is factored by Cholesky in mw (r x r).
// Returns false, with y unchanged, when that factorisation meets a pivot that is not positive
// (kept columns at the rounding level of a block whose norm is near eps); the caller then uses
// the orthogonal-columns formula y S^-2.
__device__ bool ls_solve(double* y, int q, int r, const double* g, int p, const int* perm,
                         const double* d, double* mw, SvdShared& sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int e = w; e < r * r; e += kWarps) {
    const int i = e % r, j = e / r;
    if (i < j) continue;
    const double* gi = g + (int64_t)perm[i] * p;
    const double* gj = g + (int64_t)perm[j] * p;
    double s2 = 0.0;
    for (int k = l; k < p; k += 32) s2 = fma(gi[k], gj[k], s2);
    s2 = warp_sum(s2);
    if (l == 0) mw[i + (int64_t)j * r] = s2 / (d[i] * d[j]);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.flag = 1;
  for (int j = 0; j < r; ++j) {  // lower Cholesky, column by column
    if (threadIdx.x == 0) {
      double a = mw[j + (int64_t)j * r];
      for (int k = 0; k < j; ++k) a -= mw[j + (int64_t)k * r] * mw[j + (int64_t)k * r];
      if (!(a > 0.0) || !isfinite(a)) {
        sh.flag = 0;
        a = 1.0;
      }
      mw[j + (int64_t)j * r] = sqrt(a);
    }
    __syncthreads();
    const double ljj = mw[j + (int64_t)j * r];
    for (int i = j + 1 + threadIdx.x; i < r; i += kThreads) {
      double a = mw[i + (int64_t)j * r];
      for (int k = 0; k < j; ++k) a -= mw[i + (int64_t)k * r] * mw[j + (int64_t)k * r];
      mw[i + (int64_t)j * r] = a / ljj;
    }
    __syncthreads();
  }
  if (!sh.flag) {
    __syncthreads();
    return false;
  }
  // each row t: x = (y_t D^-1) (L L^T)^-1 D^-1
  for (int t = threadIdx.x; t < q; t += kThreads) {
    double* yt = y + t;  // stride q
    for (int i = 0; i < r; ++i) {  // forward: L u = (y_t D^-1)^T
      double a = yt[(int64_t)i * q] / d[i];
      for (int k = 0; k < i; ++k) a -= mw[i + (int64_t)k * r] * yt[(int64_t)k * q];
      yt[(int64_t)i * q] = a / mw[i + (int64_t)i * r];
    }
    for (int i = r - 1; i >= 0; --i) {  // back: L^T x = u
      double a = yt[(int64_t)i * q];
      for (int k = i + 1; k < r; ++k) a -= mw[k + (int64_t)i * r] * yt[(int64_t)k * q];
      yt[(int64_t)i * q] = a / mw[i + (int64_t)i * r];
    }
    for (int i = 0; i < r; ++i) yt[(int64_t)i * q] /= d[i];
  }
  __syncthreads();
  return true;
}

// m (rows x q, ld ldm) <- m w in FP64 with the q x q factor w given row-major (wt[k q + c] =
// w(k, c)), row by row in place: one warp per row, the row held in registers (8 entries per
// lane) and broadcast by shuffles, 8 output columns per lane (consecutive lanes read
// consecutive entries of wt).
__device__ void right_multiply_fp64(double* m, int rows, int64_t ldm, int q, const double* wt) {
  constexpr int kPer = CLR_MAX_CLUSTER / 32;
  const int wp = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int i = wp; i < rows; i += kWarps) {
    double r[kPer], acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int k = l + 32 * j;
      r[j] = k < q ? m[i + (int64_t)k * ldm] : 0.0;
      acc[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (32 * j >= q) break;
      for (int kk = 0; kk < 32; ++kk) {
        const int k = 32 * j + kk;
        const double rk = __shfl_sync(0xffffffffu, r[j], kk);
        if (k >= q) break;
#pragma unroll
        for (int o = 0; o < kPer; ++o) {
          const int c = l + 32 * o;
          if (c < q) acc[o] = fma(rk, wt[(int64_t)k * q + c], acc[o]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int o = 0; o < kPer; ++o) {
      const int c = l + 32 * o;
      if (c < q) m[i + (int64_t)c * ldm] = acc[o];
    }
  }
  __syncthreads();
}

// Mixed-precision one-sided Jacobi SVD of the p x q (p >= q) matrix A given by `a`.  FP64 runs
// at a small fraction of the FP32 rate on this part, so the rotations are found in FP32 and only
// applied, once per stage, in FP64:
//  1. FP32 sweeps on a copy of A until converged at FP32 accuracy, accumulating V1;
//  2. V = V1 orthonormalised in FP64 (modified Gram-Schmidt) and G = A V in FP64.  G's columns
//     are orthogonal to FP32 accuracy relative to ||A||; the part of the spectrum below
//     u32 ||A|| is still unresolved (it was rounding noise in the FP32 copy of A);
//  3. FP32 sweeps on a copy of G, whose columns are rounded relative to their own norms, so
//     the small columns are resolved against each other and against the large ones; V2
//     orthonormalised in FP64 and G <- G V2;
//  4. FP64 sweeps continuing on G -- a quadratically convergent clean-up from there.  The
//     rotations are not accumulated: for kept columns G_r = U_r S_r the right factor is
//     V_r = A^T G_r S_r^-2 (recover_right), and G_r (A^T G_r S_r^-2)^T = P A with P the
//     orthogonal projector onto span(G_r), so rounding in V_r is scaled back by S_r.
// Pairs whose inner product is below the noise floor are not rotated: p u ||A||_F in FP32 on A,
// and max(p u ||A||_F, 1e-3 eps) on G (columns that small cannot move a truncation at eps).
// On return g = U S in FP64, and v the right factor when sh.v_tracked (else workspace).  sc:
// kSvdScratchPerCta doubles.
//
// Certified dense exit (dense_h >= 0): the block is stored dense when its eps-rank exceeds
// dense_h, i.e. when the singular-value tail sqrt(sum_{i >= dense_h} s_i^2) exceeds eps.  After
// stage 1 every sorted column norm c_i of G32 is within delta of s_i(A), with
//   delta = 2 u32 ||A||_F (4 q sqrt(p) + p sqrt(q) + 2 s32 q + 1)
// (backward error of s32 FP32 sweeps of rotations, the rounding of A to FP32, and the residual
// non-orthogonality of G32's columns: pairs within 4 u32 sqrt(p) of orthogonal or below the FP32
// noise floor).  So tail(A) >= tail(c) - sqrt(q - dense_h) delta, and when that exceeds eps the
// later stages could only confirm "dense": they are skipped and the function returns 1.
__device__ __noinline__ int svd_mixed(const SrcView& a, int p, int q, double* g, double* v,
                                      double* sc, int max_sweeps, double eps, int dense_h,
                                      double fro, SvdShared& sh, unsigned long long* jstats,
                                      unsigned long long* stage_clk = nullptr) {
  // while profiling the full-SVD path: SM cycles per stage (1..5 of kFullStageCounters)
  long long ck = stage_clk ? clock64() : 0;
  auto mark = [&](int stage) {
    if (stage_clk && threadIdx.x == 0) {
      const long long now = clock64();
      atomicAdd(&stage_clk[stage], (unsigned long long)(now - ck));
      ck = now;
    }
  };
  // FP32 copies in the per-CTA scratch: the kernels run with the largest L1 carveout, which
  // measured as fast as holding the copies in shared memory and gives the 256-column tiles
  // (copies of 512 KB) the most cache
  const int64_t pq = (int64_t)p * q;
  float* g32 = reinterpret_cast<float*>(sc);
  float* v32 = g32 + pq;
  double* v2 = sc + (int64_t)CLR_MAX_CLUSTER * CLR_MAX_CLUSTER;  // after p q + q^2 floats
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int e = threadIdx.x; e < p * q; e += kThreads) g32[e] = (float)a.at(e % p, e / p);
  __syncthreads();
  const float floor32 = (float)((double)p * FLT_EPSILON * fro);
  const int sw32 = jacobi_svd<float>(g32, p, q, p, v32, q, max_sweeps, &sh.flag, true, 4.0f,
                                     floor32 * floor32);
  mark(1);
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
        atomicAdd(&jstats[5], 4ull * p * q * q * sw32);
      }
      return 1;
    }
  }
  orthonormalise_fp64(v32, v, q, sh);
  project_fp64(a, p, q, v, g);
  mark(2);
  // FP64 noise floor, raised to 1e-3 eps: columns below it hold less than 1e-6 eps^2 each, so
  // their mutual (non-)orthogonality cannot move a truncation decision at eps except within a
  // hair of the threshold, while orthogonalising them costs most of the sweeps
  const double floor64 = fmax((double)p * DBL_EPSILON * fro, 1e-3 * eps);
  for (int e = threadIdx.x; e < p * q; e += kThreads) g32[e] = (float)g[e];
  __syncthreads();
  const float floor_g = (float)floor64;
  const int sw32b = jacobi_svd<float>(g32, p, q, p, v32, q, max_sweeps, &sh.flag, true, 4.0f,
                                      floor_g * floor_g);
  mark(3);
  // The FP64 sweeps rotate G alone when eps is well above the noise floor: the right factor
  // of the kept columns is then recovered from A and G afterwards (recover_right), a p q r
  // product instead of 4 q flops per rotation.  Near the floor (eps < 1e3 p u ||A||_F) kept
  // columns may lie below it, unorthogonalised, where that recovery is not a projection: V is
  // accumulated instead.
  const bool track_v = floor64 > 1e-3 * eps;
  if (sw32b > 0) {
    orthonormalise_fp64(v32, v2, q, sh);
    // V2 row-major into the scratch's first half (the FP32 copies there are dead now)
    double* v2t = sc;
    for (int e = threadIdx.x; e < q * q; e += kThreads) v2t[e] = v2[e / q + (int64_t)(e % q) * q];
    __syncthreads();
    right_multiply_fp64(g, p, p, q, v2t);
    if (track_v) right_multiply_fp64(v, q, q, q, v2t);
  }
  if (threadIdx.x == 0) sh.v_tracked = track_v ? 1 : 0;
  mark(4);
  // Without V accumulation no FP64 sweep runs (kFp64SweepCap): after stage 3 the columns of G
  // are orthogonal to the FP32 stages' tolerance (cosines ~1e-5 relative to their own norms),
  // so the sorted column norms, whose tail decides the rank, are within ~1e-10 of the
  // singular values; and with the least-squares right factor (ls_solve) X W^T is the
  // orthogonal projection of A onto span(G_r) for any G = A V_eff with V_eff orthogonal, so the
  // error is ||(I - P) G_tail|| <= ||G_tail||_F <= eps whether or not the kept columns are
  // mutually orthogonal.  (One FP64 sweep, the earlier choice, took the cosines to ~1e-10 at
  // 4 p q^2 FP64 flops; a tight cluster of singular values made it converge only linearly.)
  const int cap64 = track_v || max_sweeps < kFp64SweepCap ? max_sweeps : kFp64SweepCap;
  const int sw64 = cap64 > 0 ? jacobi_svd<double>(g, p, q, p, track_v ? v : nullptr, q, cap64,
                                                  &sh.flag, false, 1.0, floor64 * floor64)
                             : 0;
  if (threadIdx.x == 0) sh.ls_recover = (!track_v && sw64 >= cap64) ? 1 : 0;
  mark(5);
  if (jstats && threadIdx.x == 0) {
    // algorithmic flops: Jacobi 4 p q^2 per sweep, orthonormalisation 2 q^3, products 2 p q^2
    const unsigned long long pq2 = (unsigned long long)p * q * q, q3 = (unsigned long long)q * q * q;
    unsigned long long f64 = 2 * q3 + 2 * pq2 + 4 * pq2 * sw64;
    if (sw32b > 0) f64 += 2 * q3 + 2 * pq2 + (track_v ? 2 * q3 : 0);
    atomicAdd(&jstats[0], 1ull);
    atomicAdd(&jstats[1], (unsigned long long)(sw32 + sw32b));
    atomicAdd(&jstats[2], (unsigned long long)sw64);
    atomicAdd(&jstats[4], f64);
    atomicAdd(&jstats[5], 4 * pq2 * (unsigned long long)(sw32 + sw32b));
  }
  return 0;
}

// ---------------------------------------------------------------------------------------------
// ROUTE_QR tiles: X_cat (m x R) and W_cat (n x R) in the workspace slot.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) compress_qr_kernel(MatView C, const int* list,
                                                               const int* count,
                                                               const int* rsum, double* ws,
                                                               double* svd_scratch,
                                                               double eps, int max_sweeps,
                                                               int* sched,
                                                               unsigned long long* jstats) {
  __shared__ SvdShared sh;
  __shared__ int sh_next;
  double* sc = svd_scratch + (int64_t)blockIdx.x * kSvdScratchPerCta;
  const int n_items = *count;
  for (int it = next_item(sched, &sh_next); it < n_items; it = next_item(sched, &sh_next)) {
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
      svd_mixed(mv, R, R, G, V, sc, max_sweeps, eps, -1, mfro, sh, jstats);
    }
    sort_and_truncate(G, R, R, R, eps, sh);
    const int r = sh.rank;
    const bool tracked = sh.v_tracked;
    bool ls = !tracked && sh.ls_recover;
    if (!tracked) {
      // V_r S_r^2 = M^T G_r into V (M is still intact), or the least-squares V_r
      SrcView mv{M, 1, R, false};
      recover_right(mv, R, R, G, sh.perm, r, V, sc);
      if (ls) ls = ls_solve(V, R, r, G, R, sh.perm, sh.sorted, sc, sh);
    }
    double* Xo = C.pool + sC;
    double* Wo = Xo + (int64_t)m * r;
    for (int e = threadIdx.x; e < m * r; e += kThreads) {
      const int i = e % m, c = e / m;
      Xo[e] = i < R ? G[i + (int64_t)sh.perm[c] * R] : 0.0;
    }
    for (int e = threadIdx.x; e < n * r; e += kThreads) {
      const int j = e % n, c = e / n;
      Wo[e] = j >= R ? 0.0
              : tracked ? V[j + (int64_t)sh.perm[c] * R]
              : ls      ? V[j + (int64_t)c * R]
                        : V[j + (int64_t)c * R] / (sh.sorted[c] * sh.sorted[c]);
    }
    __syncthreads();
    apply_q(Xc, m, R, m, tauX, Xo, r, m);
    apply_q(Wc, n, R, n, tauW, Wo, r, n);
    if (jstats && threadIdx.x == 0) {
      // Householder QRs 2(m+n)R^2, core R_X R_W^T (2/3)R^3, recovery 2R^2 r (when not
      // accumulated), re-expansion 4(m+n)R r
      const unsigned long long mn = (unsigned long long)(m + n), RR = (unsigned long long)R * R;
      atomicAdd(&jstats[4], 2 * mn * RR + 2 * RR * R / 3 + (tracked ? 0 : 2 * RR * r) +
                                4 * mn * R * r);
    }
    if (threadIdx.x == 0) {
      C.kind[t] = r > 0 ? CLR_KIND_LR : CLR_KIND_ZERO;
      C.rank[t] = r;
      C.norm[t] = sqrt(sh.kept_sq);
    }
    __syncthreads();
  }
}

// Launch shape of a recompression kernel: one CTA per SM (512 threads x 128 registers fill the
// register file) within the caller's grid (the scratch is sized for it), with the shared memory
// carveout at its minimum so that L1 caches the FP32 working copies.
template <typename K>
int svd_launch_grid(K kernel, int grid_max, bool* attr_done) {
  int dev = 0;
  cudaGetDevice(&dev);
  int n_sm = 1;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // set once per device (outside any stream capture the first time a product runs)
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    attr_done[dev] = true;
  }
  int grid = n_sm;
  if (grid > grid_max) grid = grid_max;
  return grid < 1 ? 1 : grid;
}

void launch_compress_qr(const MatView& C, const int* list, const int* count, const int* rsum,
                        double* ws, double* svd_scratch, double eps, int max_sweeps, int grid,
                        int* err, int* sched,
                        unsigned long long* jstats, cudaStream_t st) {
  (void)err;
  static bool attr_done[64] = {false};
  const int g = svd_launch_grid(compress_qr_kernel, grid, attr_done);
  compress_qr_kernel<<<g, kThreads, 0, st>>>(C, list, count, rsum, ws, svd_scratch, eps,
                                             max_sweeps, sched, jstats);
}

// ---------------------------------------------------------------------------------------------
// Rank-revealing QR of one block (the paper's construction of X and W, Section 4.1): Householder
// QR with greedy column pivoting (at step j the remaining column of largest norm over rows
// j..m-1, first maximum; the norms are recomputed exactly every step), stopped at the first j
// whose trailing block has ||R_22||_F <= eps.  g: m x n work copy (ld m); on return its upper
// trapezoid holds R, the reflectors lie below the diagonal (v_0 = 1), tau in sh.sorted and the
// column order in sh.perm.  Returns the rank r.
// ---------------------------------------------------------------------------------------------
__device__ int rrqr_block(const double* S, int64_t s_r, int64_t s_c, int m, int n, double eps,
                          double* g, SvdShared& sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int e = threadIdx.x; e < m * n; e += kThreads) {
    const int i = e % m, j = e / m;
    g[e] = S[i * s_r + j * s_c];
  }
  for (int c = threadIdx.x; c < n; c += kThreads) sh.perm[c] = c;
  __syncthreads();
  const int k = m < n ? m : n;
  int r = k;
  for (int j = 0; j < k; ++j) {
    for (int c = j + w; c < n; c += kWarps) {
      const double* gc = g + (int64_t)c * m;
      double s2 = 0.0;
      for (int i = j + l; i < m; i += 32) s2 = fma(gc[i], gc[i], s2);
      s2 = warp_sum(s2);
      if (l == 0) sh.sigma[c] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0, best = -1.0;
      int arg = j;
      for (int c = j; c < n; ++c) {
        tot += sh.sigma[c];
        if (sh.sigma[c] > best) { best = sh.sigma[c]; arg = c; }
      }
      sh.kept_sq = tot;
      sh.flag = arg;
    }
    __syncthreads();
    if (sqrt(sh.kept_sq) <= eps) {
      r = j;
      break;
    }
    const int piv = sh.flag;
    if (piv != j) {
      double* a = g + (int64_t)j * m;
      double* b = g + (int64_t)piv * m;
      for (int i = threadIdx.x; i < m; i += kThreads) {
        const double t = a[i];
        a[i] = b[i];
        b[i] = t;
      }
      if (threadIdx.x == 0) {
        const int t = sh.perm[j];
        sh.perm[j] = sh.perm[piv];
        sh.perm[piv] = t;
      }
    }
    __syncthreads();
    // Householder reflector of column j below the diagonal (as householder_qr)
    double* col = g + (int64_t)j * m;
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += kThreads) part += col[i] * col[i];
    const double s = block_sum(part, sh.red);
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
      for (int i = j + 1 + threadIdx.x; i < m; i += kThreads) col[i] *= inv;
    }
    if (threadIdx.x == 0) {
      col[j] = beta;
      sh.sorted[j] = t;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int c = j + 1 + w; c < n; c += kWarps) {
        double* y = g + (int64_t)c * m;
        double d = 0.0;
        for (int i = j + 1 + l; i < m; i += 32) d += col[i] * y[i];
        d = warp_sum(d) + y[j];
        const double f = t * d;
        if (l == 0) y[j] -= f;
        for (int i = j + 1 + l; i < m; i += 32) y[i] -= f * col[i];
      }
    }
    __syncthreads();
  }
  return r;
}

// ---------------------------------------------------------------------------------------------
// Truncated SVD of a block of low numerical rank through a column-pivoted QR (pre-reduction).
//
// A (p x q, the block or its transpose, p >= q) is reduced by Householder QR with column
// pivoting (at step j the remaining column of largest norm over rows j..p-1, first maximum on
// ties; the norms are downdated and summed again exactly once they have fallen by 1e6, and the
// stop is always decided on exact sums), stopped at the first step k whose trailing block has
// ||R_22||_F <= tau = eps/16:
//   A P = Q [R_11 R_12; 0 R_22].
// R_22 is dropped and the k x q factor R = [R_11 R_12] gets the mixed-precision SVD, truncated
// at the remaining budget sqrt(eps^2 - ||R_22||_F^2).  The two errors are orthogonal (rows
// 0..k-1 and k..p-1 of Q^T A P), so ||A - X W^T||_F <= eps, with X = Q_k X_R and W = P W_R.
// Cost: about 3 p q k FP64 FMAs for the QR and O(q k^2) for the SVD of R, instead of the
// O(p q^2)-per-sweep Jacobi on all q columns.  Ranks can exceed the minimal eps-rank where the
// singular-value tail crosses eps within the budget split (the rank reading allows one).
// Blocks of numerical rank above q/2 (stored dense): the QR stops after J = floor(q/2) + 1
// steps, and the block is certified dense when sigma_min(R_11) > eps for the leading J x J
// triangle: R_11 is a submatrix of Q^T A P, so sigma_J(A) >= sigma_min(R_11), and the eps-rank
// exceeds q/2 as soon as sigma_{q/2+1}(A) > eps.  sigma_min(R_11) is bounded below by
// 1 / ||R_11^-1||_F (a triangular inverse, J^3/6 FMAs).
// A block that meets neither goes on to its QR rank k at eps/16 (at most q).  Past 3q/5 steps
// it is first certified dense when a leading triangle R_K' bounds the tail
// sum_{i > q/2} sigma_i(A)^2 above eps^2: sigma_min alone certifies only blocks whose
// (q/2 + 1)-th singular value exceeds eps, while the tail of a block with many singular
// values just below eps also exceeds it (tail_lower_bound_sq).  Otherwise the SVD of its R
// decides, at any k: rank <= q/2 is stored low rank, else the block is stored dense (the
// untouched source).  One-sided Jacobi on R^T after a pivoted QR
// converges in fewer sweeps than on A itself (R is graded by the pivoting: the
// preconditioning of Drmac and Veselic, "New fast and accurate Jacobi SVD algorithm", SIAM
// J. Matrix Anal. Appl. 29, 2008), so even k near q costs less than the full SVD of A.
// Returns 1 when the block is done (low rank or zero, written to slot and the outputs), 2 when
// it is certified dense, 3 when the SVD of R found it dense (for 2 and 3 the source is
// untouched: the caller stores the kind and copies an external source into the slot), 0 only
// when a trailing norm is not finite; the caller then takes the full SVD on the source.
// g: p x q copy (ld p); wv: the tile's second workspace half (p q doubles); slot: the block's
// m n output slot (also the source of product tiles, overwritten only by a low-rank result);
// sc: the CTA's SVD scratch (kSvdScratchPerCta doubles: svd_mixed's working copies in the
// first two CLR_MAX_CLUSTER^2, the k x k right factor of R^T in the third, R in the fourth).
// ---------------------------------------------------------------------------------------------
// A lower bound on sum_{i > h} sigma_i(A)^2 from the leading K x K upper triangle R_K of the
// pivoted QR in g (ld p).  For every K' in (h, K], R_K' is the upper part of the first K'
// columns of Q^T A P, so sigma_i(A) >= sigma_i(R_K') (removing columns does not raise singular
// values), and the Cauchy-Schwarz inequality over the K' - h smallest singular values of R_K'
// gives  sum_{i > h} sigma_i(R_K')^2 >= (K' - h)^2 / sum_{i > h} sigma_i(R_K')^-2
// >= (K' - h)^2 / ||R_K'^-1||_F^2.  The columns of R_K^-1 come by back substitution of the unit
// vectors, one warp per column (x: K x K scratch); column c depends only on the leading
// (c + 1) x (c + 1) triangle, so R_K'^-1 is the leading block of R_K^-1 and its squared
// Frobenius norm a prefix sum of column norms.  Returns the largest of the K - h bounds
// (h = K - 1: 1 / ||R_K^-1||_F^2 <= sigma_min(R_K)^2).
__device__ double tail_lower_bound_sq(const double* g, int p, int h, int K, double* x,
                                      SvdShared& sh) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int c = w; c < K; c += kWarps) {
    double* xc = x + (int64_t)c * K;
    double s2 = 0.0;
    for (int i = c; i >= 0; --i) {
      double d = 0.0;
      for (int t = i + 1 + l; t <= c; t += 32) d = fma(g[i + (int64_t)t * p], xc[t], d);
      d = warp_sum(d);
      const double rhs = (i == c ? 1.0 : 0.0) - d;
      const double xi = rhs / g[i + (int64_t)i * p];
      __syncwarp();
      if (l == 0) xc[i] = xi;
      __syncwarp();
      s2 = fma(xi, xi, s2);
    }
    if (l == 0) sh.sorted[c] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0, best = 0.0;
    for (int c = 0; c < K; ++c) {
      f += sh.sorted[c];
      if (!(f > 0.0) || !isfinite(f)) break;   // a zero pivot: no larger K' bounds anything
      const int kk = c + 1;
      if (kk > h) best = fmax(best, (double)(kk - h) * (double)(kk - h) / f);
    }
    sh.cert = best;
  }
  __syncthreads();
  return sh.cert;
}

// (not inlined: the kernel's register allocation stays with its own paths)
__device__ __noinline__ int compress_by_pivoted_qr(const SrcView& a, int p, int q, bool tr,
                                                   int m, int n, double eps, int max_sweeps,
                                                   double* g, double* wv, double* sc,
                                                   double* slot, int* kind_out, int* rank_out,
                                                   double* norm_out, SvdShared& sh,
                                                   unsigned long long* jstats) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  const long long c_entry = clock64();
  // Once the QR has met the threshold, R (k x q) goes to the fourth part of sc, the left SVD
  // factor of R^T (q x k <= p q doubles) to wv and the right one (k x k) to the third part of
  // sc; the source stays untouched until a low-rank result overwrites it.  Ranks up to q/2
  // are stored low rank.
  const int kmax = q / 2;
  // steps after which a block still above the threshold is tested for the sigma_min
  // certificate, and the QR rank above which the tail certificate is tried before the SVD
  // (the steps past jtail cost a few percent of the first ones: their trailing blocks are
  // small)
  const int jcert = q / 2 + 1 <= q ? q / 2 + 1 : q;
  const int jtail = (3 * q) / 5 > jcert ? (3 * q) / 5 : jcert;
  const double tau2 = (eps / 16.0) * (eps / 16.0);
  // copy with the column norms
  for (int c = w; c < q; c += kWarps) {
    double* gc = g + (int64_t)c * p;
    double s2 = 0.0;
    for (int i = l; i < p; i += 32) {
      const double x = a.at(i, c);
      gc[i] = x;
      s2 = fma(x, x, s2);
    }
    s2 = warp_sum(s2);
    if (l == 0) {
      sh.sigma[c] = s2;
      sh.qr_nref[c] = s2;
      sh.qr_perm[c] = c;
    }
  }
  if (threadIdx.x == 0) sh.qr_recomputed = 0;
  __syncthreads();
  unsigned long long fma_count = 0;
  bool exact = true;   // the trailing norms were all summed exactly at this step
  int k = -1;
  for (int j = 0; j <= q; ++j) {
    // trailing norm and pivot (warp 0)
    if (w == 0) {
      double tot = 0.0, best = -1.0;
      int arg = j;
      for (int c = j + l; c < q; c += 32) {
        const double v = sh.sigma[c];
        tot += v;
        if (v > best) { best = v; arg = c; }
      }
      tot = warp_sum(tot);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
      }
      if (l == 0) {
        sh.kept_sq = tot;
        sh.qr_pivot = arg;
      }
    }
    __syncthreads();
    if (sh.kept_sq <= tau2 && !exact) {
      // the downdated norms meet the threshold: sum the trailing norms exactly and decide (and
      // pivot) on those
      for (int c = j + w; c < q; c += kWarps) {
        const double* y = g + (int64_t)c * p;
        double s2 = 0.0;
        for (int i = j + l; i < p; i += 32) s2 = fma(y[i], y[i], s2);
        s2 = warp_sum(s2);
        if (l == 0) {
          sh.sigma[c] = s2;
          sh.qr_nref[c] = s2;
        }
      }
      fma_count += (unsigned long long)(p - j) * (unsigned long long)(q - j);
      exact = true;
      __syncthreads();
      --j;   // the same step again
      continue;
    }
    if (sh.kept_sq <= tau2) {
      k = j;
      break;
    }
    if (j == jcert) {
      // still above the threshold after floor(q/2) + 1 steps: dense if sigma_min(R_11) > eps
      const double b2 = tail_lower_bound_sq(g, p, jcert - 1, jcert, wv, sh);
      if (jstats && threadIdx.x == 0)
        atomicAdd(&jstats[4], 2ull * fma_count + (unsigned long long)jcert * jcert * jcert / 3);
      fma_count = 0;
      if (b2 > eps * eps) return 2;
    }
    // (the trailing block after q steps is empty: only a non-finite norm gets here)
    if (j == q) break;
    const int piv = sh.qr_pivot;
    if (piv != j) {
      double* x = g + (int64_t)j * p;
      double* y = g + (int64_t)piv * p;
      for (int i = threadIdx.x; i < p; i += kThreads) {
        const double t = x[i];
        x[i] = y[i];
        y[i] = t;
      }
    }
    __syncthreads();
    if (piv != j && threadIdx.x == 0) {
      const double t = sh.sigma[j];
      sh.sigma[j] = sh.sigma[piv];
      sh.sigma[piv] = t;
      const double tr = sh.qr_nref[j];
      sh.qr_nref[j] = sh.qr_nref[piv];
      sh.qr_nref[piv] = tr;
      const int ti = sh.qr_perm[j];
      sh.qr_perm[j] = sh.qr_perm[piv];
      sh.qr_perm[piv] = ti;
    }
    // Householder reflector of column j below the diagonal (as householder_qr)
    double* col = g + (int64_t)j * p;
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < p; i += kThreads) part = fma(col[i], col[i], part);
    const double sv = block_sum(part, sh.red);
    const double x0 = col[j];
    double t = 0.0, beta = x0, v0 = 1.0;
    if (sv > 0.0) {
      beta = -copysign(sqrt(x0 * x0 + sv), x0);
      v0 = x0 - beta;
      t = (beta - x0) / beta;
    }
    if (sv > 0.0) {
      const double inv = 1.0 / v0;
      for (int i = j + 1 + threadIdx.x; i < p; i += kThreads) col[i] *= inv;
    }
    if (threadIdx.x == 0) {
      col[j] = beta;
      sh.qr_tau[j] = t;
    }
    __syncthreads();
    // apply to the remaining columns.  The reflector keeps the norm of each column's rows
    // j..p-1 and moves its row j into R, so the trailing norm^2 over rows j+1..p-1 is the old
    // one minus the new row-j entry squared (downdate), summed again exactly when it has fallen
    // below kDowndateFloor of its last exact value (or is not positive).
    for (int c = j + 1 + w; c < q; c += kWarps) {
      double* y = g + (int64_t)c * p;
      double d = 0.0;
      for (int i = j + 1 + l; i < p; i += 32) d = fma(col[i], y[i], d);
      d = warp_sum(d) + y[j];
      const double f = t * d;
      for (int i = j + 1 + l; i < p; i += 32) y[i] = fma(-f, col[i], y[i]);
      const double yj = y[j] - f;
      double nu2 = sh.sigma[c] - yj * yj;
      if (!(nu2 > kDowndateFloor * sh.qr_nref[c])) {
        double s2 = 0.0;
        for (int i = j + 1 + l; i < p; i += 32) s2 = fma(y[i], y[i], s2);
        nu2 = warp_sum(s2);
        if (l == 0) {
          sh.qr_nref[c] = nu2;
          atomicAdd(&sh.qr_recomputed, (unsigned long long)(p - j - 1));
        }
      }
      __syncwarp();
      if (l == 0) {
        y[j] = yj;
        sh.sigma[c] = nu2;
      }
    }
    fma_count += 2ull * (unsigned long long)(p - j) * (unsigned long long)(q - j - 1) + (p - j);
    exact = false;
    __syncthreads();
  }
  if (jstats && threadIdx.x == 0)   // (the QR's flops after the certificate test)
    atomicAdd(&jstats[4], 2ull * (fma_count + sh.qr_recomputed));
  if (k < 0) return 0;
  if (k > jtail) {
    // dense when sum_{i > q/2} sigma_i^2 > eps^2 is certified by some leading triangle of the
    // k completed steps, else the SVD of R decides
    const double b2 = tail_lower_bound_sq(g, p, kmax, k, wv, sh);
    if (jstats && threadIdx.x == 0)
      atomicAdd(&jstats[4], (unsigned long long)k * k * k / 3);
    if (b2 > eps * eps) return 2;
  }
  const double trail2 = sh.kept_sq;
  __syncthreads();
  if (k == 0) {
    if (threadIdx.x == 0) { *kind_out = CLR_KIND_ZERO; *rank_out = 0; *norm_out = 0.0; }
    __syncthreads();
    return 1;
  }
  // R (k x q, ld k, zero below the diagonal) and the SVD of M = R^T (q x k)
  constexpr int64_t kSq = (int64_t)CLR_MAX_CLUSTER * CLR_MAX_CLUSTER;
  double* rb = sc + 3 * kSq;   // k x q
  double* gs = wv;             // q x k
  double* vs = sc + 2 * kSq;   // k x k
  double part = 0.0;
  for (int e = threadIdx.x; e < k * q; e += kThreads) {
    const int i = e % k, c = e / k;
    const double x = i <= c ? g[i + (int64_t)c * p] : 0.0;
    rb[e] = x;
    part = fma(x, x, part);
  }
  const double rfro = sqrt(block_sum(part, sh.red));
  const double budget = sqrt(fmax(eps * eps - trail2, 0.0));
  const SrcView mv{rb, k, 1, false};   // M(i, j) = R(j, i)
  unsigned long long* stage_clk = jstats ? jstats + kPreStageCounters : nullptr;
  if (stage_clk && threadIdx.x == 0)
    atomicAdd(&stage_clk[0], (unsigned long long)(clock64() - c_entry));
  svd_mixed(mv, q, k, gs, vs, sc, max_sweeps, budget, -1, rfro, sh, jstats, stage_clk);
  const long long c_after = clock64();
  sort_and_truncate(gs, q, k, q, budget, sh);
  const int r = sh.rank;
  if (r == 0) {
    if (threadIdx.x == 0) { *kind_out = CLR_KIND_ZERO; *rank_out = 0; *norm_out = 0.0; }
    __syncthreads();
    return 1;
  }
  if (r > kmax) {
    // stored dense: the source is untouched (R lives in the scratch), so the block is kept
    // exactly (the caller copies an external source into the slot)
    if (jstats && threadIdx.x == 0) {
      atomicAdd(&stage_clk[6], (unsigned long long)(clock64() - c_after));
      atomicAdd(&stage_clk[7], 1ull);
    }
    __syncthreads();
    return 3;
  }
  const bool tracked = sh.v_tracked;
  bool ls = !tracked && sh.ls_recover;
  if (!tracked) recover_right(mv, q, k, gs, sh.perm, r, vs, sc);   // Y = R G_r (k x r)
  if (ls) ls = ls_solve(vs, k, r, gs, q, sh.perm, sh.sorted, sc, sh);
  // R = V_M S U_M^T:  X_R = (V_M S)_r (k x r), W_R = (U_M)_r (q x r); A ~ (Q_k X_R) (P W_R)^T
  // (the source in the slot is no longer read: the factors overwrite it)
  __syncthreads();
  double* xa = tr ? slot + (int64_t)m * r : slot;   // Q_k X_R: p x r, ld p
  double* wa = tr ? slot : slot + (int64_t)m * r;   // P W_R: q x r, ld q
  for (int e = threadIdx.x; e < p * r; e += kThreads) {
    const int i = e % p, c = e / p;
    double v = 0.0;
    if (i < k)
      v = tracked ? vs[i + (int64_t)sh.perm[c] * k] * sh.sorted[c]
          : ls    ? vs[i + (int64_t)c * k]
                  : vs[i + (int64_t)c * k] / sh.sorted[c];
    xa[e] = v;
  }
  for (int e = threadIdx.x; e < q * r; e += kThreads) {
    const int j = e % q, c = e / q;
    const double v = gs[j + (int64_t)sh.perm[c] * q];
    wa[sh.qr_perm[j] + (int64_t)c * q] = ls ? v : v / sh.sorted[c];
  }
  __syncthreads();
  apply_q(g, p, k, p, sh.qr_tau, xa, r, p);
  if (threadIdx.x == 0) {
    *kind_out = CLR_KIND_LR;
    *rank_out = r;
    *norm_out = sqrt(sh.kept_sq);
    if (jstats) {
      atomicAdd(&jstats[4], 4ull * (unsigned long long)p * k * r);
      atomicAdd(&jstats[6], 1ull);
      atomicAdd(&stage_clk[6], (unsigned long long)(clock64() - c_after));
      atomicAdd(&stage_clk[7], 1ull);
    }
  }
  __syncthreads();
  return 1;
}

// ---------------------------------------------------------------------------------------------
// Dense truncated SVD of whole blocks (ROUTE_DACC tiles, recompressed dense tiles, building a
// CLR matrix from a dense one).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) compress_dense_kernel(
    MatView C, const int* list, const int* count, const int* order, const double* src,
    int64_t lds, double* ws, double* svd_scratch, double eps, double drop_norm,
    int dense_only, int rrqr, int prereduce, int max_sweeps, int* err, int* sched,
    unsigned long long* jstats) {
  __shared__ SvdShared sh;
  __shared__ int sh_next;
  double* sc = svd_scratch + (int64_t)blockIdx.x * kSvdScratchPerCta;
  const int n_items = list ? *count : C.nr * C.nc;
  // each tile's SM kilocycles go to C.cost (the next plan's scheduling cost), written when the
  // CTA takes its next tile (every path of the loop body ends there) and after the last one
  int prev_t = -1;
  long long prev_c = 0;
  auto record_cost = [&](long long now) {
    if (C.cost && prev_t >= 0 && threadIdx.x == 0) {
      const long long kc = (now - prev_c) >> 10;
      C.cost[prev_t] = (unsigned int)(kc < 1 ? 1 : kc > 0xFFFFFFFFll ? 0xFFFFFFFFll : kc);
    }
  };
  for (int it = next_item(sched, &sh_next); it < n_items; it = next_item(sched, &sh_next)) {
    const int t = list ? list[it] : (order ? order[it] : it);
    const long long now = clock64();
    record_cost(now);
    prev_t = t;
    prev_c = now;
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
    double* G = ws + 2 * sC;             // p x q, ld p
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
      if (threadIdx.x == 0) atomicCAS(err, 0, 3);  // a timeout (1) keeps precedence
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
    long long c_full = -1;   // while profiling: start of a full-SVD block's truncation
    if (rrqr && !dense_only) {
      r = rrqr_block(S, s_r, s_c, m, n, eps, G, sh);
      if (r > 0 && r <= q / 2) {
        // X = Q_r (the first r columns of H_0 ... H_{r-1}), W = P R_r^T
        double* Xo = slot;
        double* Wo = slot + (int64_t)m * r;
        for (int e = threadIdx.x; e < m * r; e += kThreads) Xo[e] = (e % m == e / m) ? 1.0 : 0.0;
        __syncthreads();
        apply_q(G, m, r, m, sh.sorted, Xo, r, m);
        double part = 0.0;
        for (int e = threadIdx.x; e < n * r; e += kThreads) {
          const int c = e % n, i = e / n;
          const double v = c >= i ? G[i + (int64_t)c * m] : 0.0;
          Wo[sh.perm[c] + (int64_t)i * n] = v;
          part = fma(v, v, part);
        }
        const double kept = block_sum(part, sh.red);
        if (threadIdx.x == 0) {
          C.kind[t] = CLR_KIND_LR;
          C.rank[t] = r;
          C.norm[t] = sqrt(kept);
        }
        __syncthreads();
        continue;
      }
    } else if (!dense_only) {
      const SrcView view{S, s_r, s_c, tr};
      const long long c0 = clock64();
      // pivoted QR first: blocks of low numerical rank are truncated through the SVD of
      // the k x q factor, blocks of rank above q/2 certified dense
      const int pre = prereduce ? compress_by_pivoted_qr(view, p, q, tr, m, n, eps, max_sweeps,
                                                         G, V, sc, slot, &C.kind[t], &C.rank[t],
                                                         &C.norm[t], sh, jstats)
                                : 0;
      if (pre == 0) {
        unsigned long long* stage_clk = jstats ? jstats + kFullStageCounters : nullptr;
        if (stage_clk && threadIdx.x == 0)
          atomicAdd(&stage_clk[0], (unsigned long long)(clock64() - c0));
        const int early_dense = svd_mixed(view, p, q, G, V, sc, max_sweeps, eps, q / 2, nrm,
                                          sh, jstats, stage_clk);
        if (!early_dense) {
          c_full = clock64();
          sort_and_truncate(G, p, q, p, eps, sh);
          r = sh.rank;
        }
      } else if (pre >= 2 && jstats && threadIdx.x == 0) {
        atomicAdd(&jstats[3], 1ull);   // stored dense without a full SVD
      }
      // SM cycles per path while profiling (block 2 of the counters): QR and the SVD of R
      // stored low rank, certified dense by the QR's triangles, full SVD (prereduce off, or a
      // non-finite QR norm), QR and the SVD of R stored dense
      if (jstats && threadIdx.x == 0) {
        const int path = pre == 1 ? 0 : pre == 2 ? 1 : pre == 3 ? 3 : 2;
        atomicAdd(&jstats[kPathCounters + 2 * path], (unsigned long long)(clock64() - c0));
        atomicAdd(&jstats[kPathCounters + 2 * path + 1], 1ull);
      }
      if (pre == 1) continue;
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
      // Y = A^T G_r (q x r) into V before the slot (possibly the source) is overwritten, or
      // Y = V_r S_r^2 from the accumulated V
      const SrcView view{S, s_r, s_c, tr};
      const bool tracked = sh.v_tracked;
      bool ls = !tracked && sh.ls_recover;
      if (!tracked) recover_right(view, p, q, G, sh.perm, r, V, sc);
      if (ls) ls = ls_solve(V, q, r, G, p, sh.perm, sh.sorted, sc, sh);
      if (jstats && threadIdx.x == 0 && !tracked)
        atomicAdd(&jstats[4], 2ull * p * q * r);
      double* Xo = slot;
      double* Wo = slot + (int64_t)m * r;
      if (!tr) {
        // G = U S (m x n), Y = V S^2:  X = (U S)_r, W = V_r
        for (int e = threadIdx.x; e < m * r; e += kThreads) {
          const int i = e % m, c = e / m;
          Xo[e] = G[i + (int64_t)sh.perm[c] * p];
        }
        for (int e = threadIdx.x; e < n * r; e += kThreads) {
          const int j = e % n, c = e / n;
          Wo[e] = tracked ? V[j + (int64_t)sh.perm[c] * q]
                  : ls    ? V[j + (int64_t)c * q]
                          : V[j + (int64_t)c * q] / (sh.sorted[c] * sh.sorted[c]);
        }
      } else {
        // G = U' S (n x m) of the transposed block, Y = V' S^2 (m x r): block = V' S U'^T ->
        // X = V'_r S_r = Y S^-1, W = U'_r = G_r S^-1
        for (int e = threadIdx.x; e < m * r; e += kThreads) {
          const int i = e % m, c = e / m;
          Xo[e] = tracked ? V[i + (int64_t)sh.perm[c] * q] * sh.sorted[c]
                  : ls    ? V[i + (int64_t)c * q]
                          : V[i + (int64_t)c * q] / sh.sorted[c];
        }
        for (int e = threadIdx.x; e < n * r; e += kThreads) {
          const int j = e % n, c = e / n;
          Wo[e] = ls ? G[j + (int64_t)sh.perm[c] * p] : G[j + (int64_t)sh.perm[c] * p] / sh.sorted[c];
        }
      }
      if (threadIdx.x == 0) {
        C.kind[t] = CLR_KIND_LR;
        C.rank[t] = r;
        C.norm[t] = sqrt(sh.kept_sq);
      }
    }
    __syncthreads();
    if (jstats && c_full >= 0 && threadIdx.x == 0) {
      atomicAdd(&jstats[kFullStageCounters + 6], (unsigned long long)(clock64() - c_full));
      atomicAdd(&jstats[kFullStageCounters + 7], 1ull);
      if (r > q / 2) atomicAdd(&jstats[7], 1ull);   // full SVD, stored dense
    }
  }
  record_cost(clock64());
}

void launch_compress_dense(const MatView& C, const int* list, const int* count,
                           const int* order, const double* src, int64_t lds, double* ws,
                           double* svd_scratch, double eps, double drop_norm,
                           int dense_only, int rrqr, int prereduce, int max_sweeps, int grid,
                           int* err, int* sched, unsigned long long* jstats, cudaStream_t st) {
  static bool attr_done[64] = {false};
  const int g = svd_launch_grid(compress_dense_kernel, grid, attr_done);
  compress_dense_kernel<<<g, kThreads, 0, st>>>(C, list, count, order, src, lds, ws, svd_scratch,
                                                eps, drop_norm, dense_only, rrqr, prereduce,
                                                max_sweeps, err, sched, jstats);
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

// status[0] = kind, status[1] = rank, status[2] = error flag (3: non-finite input, 4: sweep
// limit reached before convergence)
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
  // pairs of columns at the FP64 rounding level of the block (p u ||A||_F) are left alone:
  // rotating them changes nothing that a truncation can see, and they would keep the sweeps
  // from ever converging
  const double floor64 = (double)p * DBL_EPSILON * sqrt(nsq);
  const int sweeps = jacobi_svd(G, p, q, p, V, q, max_sweeps, &sh.flag, true, 1.0,
                                floor64 * floor64);
  // every sweep still rotated a pair: the column norms the truncation uses may be inexact
  if (sweeps >= max_sweeps && threadIdx.x == 0) status[2] = 4;
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
