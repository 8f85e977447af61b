// K6/K7 -- CLR linear combination (the T_n polynomial of Section 4.2 is
// (15 I - 10 X_n + 3 X_n^2) / 8), distance to the identity (NS convergence test), CLR
// matrix-vector products (alpha estimate) and transposes (adjoint products).
#include "clr_internal.h"

namespace clr {

constexpr int kT = 256;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double bsum(double v, double* sh) {
  v = wsum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += sh[i];
  __syncthreads();
  return s;
}

// Route of each output block of out = a X + b Y + diag I (rules of Section 4.1 low-rank
// addition; see clr.h).
__global__ void lincomb_route_kernel(double a, MatView X, double b, MatView Y, double diag,
                                     Plan p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nI * p.nJ) return;
  const int I = t / p.nJ, J = t % p.nJ;
  const int m = X.row_off[I + 1] - X.row_off[I];
  const int n = X.col_off[J + 1] - X.col_off[J];
  int kx = X.kind[t], ky = Y.kind[t];
  if (a == 0.0) kx = CLR_KIND_ZERO;
  if (b == 0.0) ky = CLR_KIND_ZERO;
  const bool shift = I == J && diag != 0.0;
  int route = ROUTE_ZERO, rs = 0;
  if (kx == CLR_KIND_ZERO && ky == CLR_KIND_ZERO && !shift) {
    route = ROUTE_ZERO;
  } else if (!shift && (kx == CLR_KIND_ZERO || ky == CLR_KIND_ZERO)) {
    route = -1;  // exact scaled copy
  } else if (shift || kx == CLR_KIND_DENSE || ky == CLR_KIND_DENSE) {
    route = ROUTE_DENSE;
  } else {
    const int R = X.rank[t] + Y.rank[t];
    const int lim = (m < n ? m : n) / 2;
    if (R <= lim) { route = ROUTE_QR; rs = R; } else { route = ROUTE_DACC; }
  }
  p.t_count[t] = 0;
  p.t_route[t] = route < 0 ? ROUTE_ZERO : route;
  p.t_rsum[t] = rs;
  // the copy case is re-derived by the apply kernel from the operand kinds
}

__global__ void __launch_bounds__(kT) lincomb_apply_kernel(double a, MatView X, double b,
                                                           MatView Y, double diag, MatView O,
                                                           Plan p, double* ws) {
  __shared__ double red[kT / 32];
  const int t = blockIdx.x;
  const int I = t / p.nJ, J = t % p.nJ;
  const int m = X.row_off[I + 1] - X.row_off[I];
  const int n = X.col_off[J + 1] - X.col_off[J];
  int kx = X.kind[t], ky = Y.kind[t];
  if (a == 0.0) kx = CLR_KIND_ZERO;
  if (b == 0.0) ky = CLR_KIND_ZERO;
  const bool shift = I == J && diag != 0.0;
  const int64_t sl = slot_of(O, I, J, m);
  const double* xs = X.pool + sl;
  const double* ys = Y.pool + sl;
  double* os = O.pool + sl;
  const int route = p.t_route[t];
  const int rx = X.rank[t], ry = Y.rank[t];
  if (kx == CLR_KIND_ZERO && ky == CLR_KIND_ZERO && !shift) {
    if (threadIdx.x == 0) { O.kind[t] = CLR_KIND_ZERO; O.rank[t] = 0; O.norm[t] = 0.0; }
    return;
  }
  if (!shift && (kx == CLR_KIND_ZERO || ky == CLR_KIND_ZERO)) {
    const bool fromx = ky == CLR_KIND_ZERO;
    const MatView& S = fromx ? X : Y;
    const double c = fromx ? a : b;
    const double* ss = fromx ? xs : ys;
    const int kind = S.kind[t], r = S.rank[t];
    if (kind == CLR_KIND_DENSE) {
      for (int e = threadIdx.x; e < m * n; e += kT) os[e] = c * ss[e];
    } else {
      for (int e = threadIdx.x; e < m * r; e += kT) os[e] = c * ss[e];
      for (int e = threadIdx.x; e < n * r; e += kT) os[m * r + e] = ss[m * r + e];
    }
    if (threadIdx.x == 0) { O.kind[t] = kind; O.rank[t] = r; O.norm[t] = fabs(c) * S.norm[t]; }
    return;
  }
  if (route == ROUTE_QR) {
    const int R = rx + ry;
    double* Xc = ws + 2 * sl;
    double* Wc = Xc + (int64_t)m * R;
    for (int e = threadIdx.x; e < m * rx; e += kT) Xc[e] = a * xs[e];
    for (int e = threadIdx.x; e < m * ry; e += kT) Xc[m * rx + e] = b * ys[e];
    for (int e = threadIdx.x; e < n * rx; e += kT) Wc[e] = xs[m * rx + e];
    for (int e = threadIdx.x; e < n * ry; e += kT) Wc[n * rx + e] = ys[m * ry + e];
    return;
  }
  // dense sum (ROUTE_DENSE or ROUTE_DACC)
  double part = 0.0;
  for (int e = threadIdx.x; e < m * n; e += kT) {
    const int i = e % m, j = e / m;
    double v = 0.0;
    if (kx == CLR_KIND_DENSE) {
      v = a * xs[e];
    } else if (kx == CLR_KIND_LR) {
      double s = 0.0;
      for (int c = 0; c < rx; ++c) s = fma(xs[i + c * m], xs[m * rx + j + c * n], s);
      v = a * s;
    }
    if (ky == CLR_KIND_DENSE) {
      v = fma(b, ys[e], v);
    } else if (ky == CLR_KIND_LR) {
      double s = 0.0;
      for (int c = 0; c < ry; ++c) s = fma(ys[i + c * m], ys[m * ry + j + c * n], s);
      v = fma(b, s, v);
    }
    if (shift && i == j) v += diag;
    os[e] = v;
    part = fma(v, v, part);
  }
  const double nsq = bsum(part, red);
  if (threadIdx.x == 0) {
    O.kind[t] = CLR_KIND_DENSE;
    O.rank[t] = m < n ? m : n;
    O.norm[t] = sqrt(nsq);
  }
}

void launch_plan_scan(const Plan& p, int recompress_dense, cudaStream_t st);

void launch_lincomb_plan(double a, const MatView& X, double b, const MatView& Y, double diag,
                         const MatView& O, const Plan& p, double* ws, int recompress_dense,
                         cudaStream_t st) {
  const int n = p.nI * p.nJ;
  cudaMemsetAsync(p.counters, 0, kPlanCountersClear, st);
  lincomb_route_kernel<<<(n + 127) / 128, 128, 0, st>>>(a, X, b, Y, diag, p);
  launch_plan_scan(p, recompress_dense, st);
  lincomb_apply_kernel<<<n, kT, 0, st>>>(a, X, b, Y, diag, O, p, ws);
}

// Per block: ||M_IJ - delta_IJ I||_F^2, then a deterministic single-CTA sum.
__global__ void __launch_bounds__(kT) identity_distance_block_kernel(MatView M, double* part) {
  __shared__ double red[kT / 32];
  const int t = blockIdx.x;
  const int I = t / M.nc, J = t % M.nc;
  const int m = M.row_off[I + 1] - M.row_off[I];
  const int n = M.col_off[J + 1] - M.col_off[J];
  const int kind = M.kind[t];
  if (I != J) {
    if (threadIdx.x == 0) part[t] = M.norm[t] * M.norm[t];
    return;
  }
  const double* s = M.pool + slot_of(M, I, J, m);
  double acc = 0.0;
  if (kind == CLR_KIND_DENSE) {
    for (int e = threadIdx.x; e < m * n; e += kT) {
      const double v = s[e] - ((e % m) == (e / m) ? 1.0 : 0.0);
      acc = fma(v, v, acc);
    }
  } else if (kind == CLR_KIND_LR) {
    // ||X W^T||^2 - 2 tr(X W^T) + m
    const int r = M.rank[t];
    for (int e = threadIdx.x; e < m * r; e += kT) {
      const int i = e % m, c = e / m;
      acc -= 2.0 * s[e] * s[m * r + i + c * n];
    }
  }
  const double tot = bsum(acc, red);
  if (threadIdx.x == 0) {
    if (kind == CLR_KIND_DENSE) part[t] = tot;
    else if (kind == CLR_KIND_LR) part[t] = M.norm[t] * M.norm[t] + tot + (double)m;
    else part[t] = (double)m;
  }
}

__global__ void __launch_bounds__(1024) sum_kernel(const double* part, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = wsum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) tot += red[i];
    *out = tot;
  }
}

void launch_identity_distance(const MatView& X, double* out_sq, cudaStream_t st) {
  // out_sq[0] receives the sum; out_sq[1 ...] holds the per-block parts
  const int nb = X.nr * X.nc;
  identity_distance_block_kernel<<<nb, kT, 0, st>>>(X, out_sq + 1);
  sum_kernel<<<1, 1024, 0, st>>>(out_sq + 1, nb, out_sq);
}

// y_I = sum_J M_IJ x_J, one CTA per block-row.
__global__ void __launch_bounds__(kT) matvec_kernel(MatView M, const double* x, double* y) {
  __shared__ double acc[CLR_MAX_CLUSTER];
  __shared__ double tw[CLR_MAX_CLUSTER / 2];
  const int I = blockIdx.x;
  const int m = M.row_off[I + 1] - M.row_off[I];
  for (int i = threadIdx.x; i < m; i += kT) acc[i] = 0.0;
  __syncthreads();
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  for (int J = 0; J < M.nc; ++J) {
    const int t = I * M.nc + J;
    const int kind = M.kind[t];
    if (kind == CLR_KIND_ZERO) continue;
    const int n = M.col_off[J + 1] - M.col_off[J];
    const double* s = M.pool + slot_of(M, I, J, m);
    const double* xj = x + M.col_off[J];
    if (kind == CLR_KIND_DENSE) {
      for (int i = threadIdx.x; i < m; i += kT) {
        double v = 0.0;
        for (int j = 0; j < n; ++j) v = fma(s[i + (int64_t)j * m], xj[j], v);
        acc[i] += v;
      }
    } else {
      const int r = M.rank[t];
      const double* W = s + (int64_t)m * r;
      for (int c = w; c < r; c += kT / 32) {
        double v = 0.0;
        for (int j = l; j < n; j += 32) v = fma(W[j + (int64_t)c * n], xj[j], v);
        v = wsum(v);
        if (l == 0) tw[c] = v;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += kT) {
        double v = 0.0;
        for (int c = 0; c < r; ++c) v = fma(s[i + (int64_t)c * m], tw[c], v);
        acc[i] += v;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < m; i += kT) y[M.row_off[I] + i] = acc[i];
}

void launch_matvec(const MatView& M, const double* x, double* y, cudaStream_t st) {
  matvec_kernel<<<M.nr, kT, 0, st>>>(M, x, y);
}

// T = S^T: block (J,I) of T is block (I,J) of S transposed (dense) or with X and W swapped.
__global__ void transpose_kernel(MatView S, MatView T) {
  const int t = blockIdx.x;
  const int I = t / S.nc, J = t % S.nc;
  const int m = S.row_off[I + 1] - S.row_off[I];
  const int n = S.col_off[J + 1] - S.col_off[J];
  const int kind = S.kind[t], r = S.rank[t];
  const double* s = S.pool + slot_of(S, I, J, m);
  const int tt = J * T.nc + I;
  double* d = T.pool + slot_of(T, J, I, n);
  if (kind == CLR_KIND_DENSE) {
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
      const int i = e % m, j = e / m;
      d[j + (int64_t)i * n] = s[e];
    }
  } else if (kind == CLR_KIND_LR) {
    for (int e = threadIdx.x; e < n * r; e += blockDim.x) d[e] = s[(int64_t)m * r + e];
    for (int e = threadIdx.x; e < m * r; e += blockDim.x) d[(int64_t)n * r + e] = s[e];
  }
  if (threadIdx.x == 0) {
    T.kind[tt] = kind;
    T.rank[tt] = r;
    T.norm[tt] = S.norm[t];
  }
}

void launch_transpose(const MatView& S, const MatView& T, cudaStream_t st) {
  transpose_kernel<<<S.nr * S.nc, 256, 0, st>>>(S, T);
}

}  // namespace clr
