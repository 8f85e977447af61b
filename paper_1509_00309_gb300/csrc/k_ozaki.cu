// K1 (FP64-accurate) -- dense x dense tile products on the tensor cores by exact slices.
//
// Method: the error-free transformation of matrix products of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012): every row of A and of B^T
// is scaled by a power of two so that its entries lie in (-1, 1) and cut into fixed-point
// slices whose products, and the sums of those products over a bounded number of terms, are
// exact in the tensor cores' FP32 accumulator.
//
// Slices.  Row i of the A panel has exponent e_i (|a_ik| < 2^e_i for every k of the row's
// staged blocks).  v = round(a 2^(47 - e_i)) is an integer of magnitude <= 2^47; its balanced
// base-64 digits d_0 .. d_7 (d_1..d_7 in [-32, 31], d_0 in [-32, 32]) satisfy
//   a / 2^e_i = sum_s d_s 2^(-5 - 6 s) + r,   |r| <= 2^-48,
// and each digit is an integer of magnitude <= 32, exact in bf16.  The same for B with
// exponents f_j.
// Products.  C_ij = 2^(e_i + f_j - 10) sum_g 2^(-6 g) G_g with G_g = sum_{s + t = g} sum_k
// d_s(a_ik) d_t(b_jk): pairs with s + t <= 7 are kept (36 products of bf16 slices), the rest is
// below the truncation.  Every product of two digits is an integer of magnitude <= 2^10, so a
// sum over K_seg = 1024 values of k and the g + 1 <= 8 pairs of a group stays within
// 8 * 1024 * 2^10 = 2^23: the FP32 accumulator holds it exactly.  The error against the exact
// product is at most K 2^-44 2^(e_i + f_j) (truncation of both operands and the dropped pairs),
// about 2^-48 sqrt(K) 2^(e_i + f_j) for independent rounding: FP64-like relative to the rows'
// and columns' largest entries.
//
// Kernel (one CTA per SM, persistent over 128 x 32 output tiles):
//   warp 0     TMA producer: per 32-wide k chunk the 8 slices of the A tile (128 x 32) and of
//              the B tile (32 x 32), 64-byte swizzle, into one of two pipeline stages;
//   warp 1     allocates all 512 TMEM columns: two sets of eight 128 x 32 FP32 accumulators
//              (one per weight group g, side by side), and issues tcgen05.mma (M=128, K=16,
//              kind::f16, bf16 in, FP32 accumulate) for the 36 slice pairs as 8 MMAs per K16
//              step: slice s of A against the B slices t = 0 .. 7 - s at once (N = 32 (8 - s)),
//              which writes groups s .. 7 together.  Each A slice is then read from shared
//              memory once per MMA instead of once per pair (with one MMA per pair the tensor
//              unit was bound by operand fetch: busy 68% of the time with its math pipe at
//              28%).  Consecutive K segments alternate between the two sets;
//   warps 2-9  epilogue: after every K segment of 1024 the eight exact group sums of its set
//              are read from TMEM and added, scaled by 2^(e_i + f_j - 10 - 6 g) with the
//              segment's exponents, into FP64 registers (16 per thread), while the MMAs of the
//              next segment fill the other set (with one set, 128 x 64 tiles, this FP64 fold
//              took a third of the kernel's time); after the tile's last segment the values are
//              stored into the C tiles the GEMM serves (route DENSE or DACC_G).
// Every mbarrier wait is bounded as in the split-precision kernel; on a timeout the kernel
// raises the error flag, drains its copies and MMAs (bounded) and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "clr_internal.h"

namespace clr {

namespace oz {

constexpr int S = kOzakiSlices;  // 8
constexpr int BM = 128;
constexpr int BN = kOzakiTileN;      // 32
constexpr int BK = 32;               // 32 bf16 = 64 bytes: one 64B-swizzle row
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t A_TILE = BM * BK * 2;   // 8192 B
constexpr uint32_t B_TILE = BN * BK * 2;   // 2048 B
constexpr uint32_t STAGE = S * (A_TILE + B_TILE);
constexpr int STAGES = 2;
constexpr uint32_t SMEM_DATA = STAGE * STAGES;
constexpr uint32_t SMEM_TOTAL = SMEM_DATA + 1024 /*barriers*/ + 1024 /*align*/;
constexpr int GROUPS = S;            // weight groups g = s + t <= S - 1
constexpr int ACC_COLS = GROUPS * BN;   // one accumulator set: the eight groups side by side
constexpr int NBUF = 2;                 // two sets: a segment's MMAs overlap the last one's fold
constexpr int EPC = BN / 2;             // output columns per epilogue thread
constexpr int SEG_CHUNKS = 32;       // K segment of 1024: exact FP32 group sums
constexpr int SEG_K = SEG_CHUNKS * BK;
constexpr int kPassSegments = kOzakiPassK / SEG_K;   // K segments per launch (ozaki_gemm_dd)
static_assert(kOzakiPassK % SEG_K == 0, "a launch covers whole K segments");
// the staging kernels' k tiles (256, 128 and 4 x 256 wide) never straddle a segment
static_assert(SEG_K == 1024 && SEG_K == kOzakiSegK, "staging tiles assume K segments of 1024");
constexpr int TMEM_COLS = 512;
constexpr unsigned long long kDrainNs = 2000000000ull;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on the phase of parity `parity`; false on timeout (after limit_ns) or abort.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                          unsigned long long limit_ns) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(b))
      : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, rows of 64 bytes with 64-byte swizzle,
// 8-row groups 512 bytes apart (stride byte offset); leading byte offset unused.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n
// (a multiple of 16 up to 256).
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
constexpr int kMaxSlicesPerMma = 256 / BN;   // B slices one MMA covers (N <= 256)
static_assert(NBUF * GROUPS * BN == 512, "the accumulator sets fill the 512 TMEM columns");

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Epi {
  double* pool;
  const int* row_off;
  const int* row_tile_of;
  const int* col_tile_of;
  const int* t_route;
  const int* ea;   // row exponents of A (M_pad), sentinel for rows without dense entries
  const int* eb;   // row exponents of the B panel = column exponents of C (N_pad)
  int nJ;
  int64_t n_rows, n_cols;
};

// Linear tile id -> (m block, n block), grouped along m for L2 reuse across concurrent CTAs.
__device__ __forceinline__ void tile_coords(int id, int n_m, int n_n, int* mb, int* nb) {
  constexpr int G = 8;   // 8 x 19 tiles of 128 x 32 per wave: the least panel bytes
  const int per_group = G * n_n;
  const int g = id / per_group;
  const int first = g * G;
  const int gs = min(G, n_m - first);
  const int r = id - g * per_group;
  *mb = first + r % gs;
  *nb = r / gs;
}

// Exponents of rows without entries (the staging's sentinel) scale only zero digits: 0.
__device__ __forceinline__ int clamp_exp(int e) { return e < -1100 ? 0 : e; }

// 2^x: built from its bits in the normal range, by ldexp outside it.
__device__ __forceinline__ double pow2(int x) {
  if (x >= -1022 && x <= 1023) return __longlong_as_double((long long)(x + 1023) << 52);
  return ldexp(1.0, x);
}

__global__ void __launch_bounds__(THREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, Epi epi, int n_m, int n_n,
                      int k_begin, int k_end, int accumulate, int M_pad, int N_pad,
                      const int* active, int* err,
                      unsigned long long wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + SMEM_DATA);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;     // per accumulator set
  uint64_t* tempty = tfull + NBUF;
  uint64_t* drain = tempty + NBUF;
  uint32_t* tmem_holder = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // the active tiles in raster order (oz_compact_kernel): active[0] of them at active[1..]
  const int n_act = active[0];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            saddr(tmem_holder)),
        "r"(TMEM_COLS)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int s = 0;
      uint32_t phase = 0;
      uint32_t issued_parity[STAGES];
      bool issued[STAGES];
      for (int i = 0; i < STAGES; ++i) issued[i] = false;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < n_act; it += gridDim.x) {
        const int tile = active[1 + it];
        int mb, nb;
        tile_coords(tile, n_m, n_n, &mb, &nb);
        for (int kc = k_begin; kc < k_end; ++kc) {
          if (!mbar_wait(&empty[s], phase ^ 1, abort_flag, wait_ns)) { ok = false; break; }
          unsigned char* st = smem + (size_t)s * STAGE;
          mbar_expect_tx(&full[s], STAGE);
          issued[s] = true;
          issued_parity[s] = phase;
          for (int t = 0; t < S; ++t)
            tma_load_2d(st + t * A_TILE, &tmA, kc * BK, t * M_pad + mb * BM, &full[s]);
          for (int t = 0; t < S; ++t)
            tma_load_2d(st + S * A_TILE + t * B_TILE, &tmB, kc * BK, t * N_pad + nb * BN,
                        &full[s]);
          if (++s == STAGES) { s = 0; phase ^= 1; }
        }
      }
      if (!ok) {
        // copies in flight land before the CTA exits (bounded)
        for (int i = 0; i < STAGES; ++i)
          if (issued[i]) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try(&full[i], issued_parity[i]) && gtimer() - t0 < kDrainNs) {
            }
          }
        atomicExch(err, 1);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t phase = 0;
      int seg_count = 0;  // segments issued by this CTA
      bool ok = true;
      bool any = false;
      for (int it = blockIdx.x; ok && it < n_act; it += gridDim.x) {
        for (int k0 = k_begin; ok && k0 < k_end; k0 += SEG_CHUNKS) {
          const int k1 = min(k_end, k0 + SEG_CHUNKS);
          // the epilogue has read the group sums of the segment before last from this set
          const int bset = seg_count & 1;
          const uint32_t tp = (seg_count >> 1) & 1;
          if (!mbar_wait(&tempty[bset], tp ^ 1, abort_flag, wait_ns)) { ok = false; break; }
          fence_after();
          const uint32_t acc_base = tmem_base + (uint32_t)(bset * ACC_COLS);
          for (int kc = k0; kc < k1; ++kc) {
            if (!mbar_wait(&full[s], phase, abort_flag, wait_ns)) { ok = false; break; }
            fence_after();
            const uint32_t st = saddr(smem + (size_t)s * STAGE);
            // A slice s times the consecutive B slices t = 0 .. 7 - s in one MMA of
            // N = 32 (8 - s): its output columns land in the accumulators of groups s .. 7,
            // which are consecutive in TMEM.  The MMA of s = 0 covers every group, so it alone
            // starts a segment (accumulate off).
#pragma unroll
            for (int k16 = 0; k16 < BK / 16; ++k16) {
#pragma unroll 1
              for (int sa = 0; sa < S; ++sa) {
                const uint32_t a_addr = st + sa * A_TILE + k16 * 32;
                for (int t0 = 0; t0 < S - sa; t0 += kMaxSlicesPerMma) {
                  const int cnt = min(kMaxSlicesPerMma, S - sa - t0);
                  const uint32_t d_tmem = acc_base + (uint32_t)((sa + t0) * BN);
                  const uint32_t b_addr = st + S * A_TILE + t0 * B_TILE + k16 * 32;
                  const uint32_t acc = (kc != k0 || sa != 0 || k16 != 0) ? 1u : 0u;
                  umma_bf16(d_tmem, sdesc(a_addr), sdesc(b_addr), idesc_n(cnt * BN), acc);
                }
              }
            }
            umma_commit(&empty[s]);
            any = true;
            if (++s == STAGES) { s = 0; phase ^= 1; }
          }
          if (!ok) break;
          umma_commit(&tfull[bset]);
          ++seg_count;
        }
      }
      if (!ok) {
        if (any) {
          // wait (bounded) for the MMAs already issued before TMEM is released
          umma_commit(drain);
          const unsigned long long t0 = gtimer();
          while (!mbar_try(drain, 0) && gtimer() - t0 < kDrainNs) {
          }
        }
        atomicExch(err, 1);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    const int quarter = warp % 4;          // TMEM lanes 32*quarter .. 32*quarter+31
    const int half = (warp - 2) / 4;       // columns EPC*half .. EPC*half+EPC-1
    const int rl = quarter * 32 + lane;    // row within the tile
    int seg_count = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_act; it += gridDim.x) {
      const int tile = active[1 + it];
      int mb, nb;
      tile_coords(tile, n_m, n_n, &mb, &nb);
      double acc[EPC];
#pragma unroll
      for (int j = 0; j < EPC; ++j) acc[j] = 0.0;
      const int64_t row = (int64_t)mb * BM + rl;
      const int64_t col0 = (int64_t)nb * BN + half * EPC;
      for (int k0 = k_begin; k0 < k_end; k0 += SEG_CHUNKS) {
        // this segment's scale of every entry: 2^(e_i + f_j - 10) with the exponents of its
        // own K range (row i of A, column j of B over the segment's columns / rows)
        const int sg = k0 / SEG_CHUNKS;
        const int er = clamp_exp(epi.ea[(int64_t)sg * M_pad + row]) - 10;
        int ex[EPC];
#pragma unroll
        for (int j = 0; j < EPC; ++j)
          ex[j] = er + clamp_exp(epi.eb[(int64_t)sg * N_pad + col0 + j]);
        const int bset = seg_count & 1;
        int got = 0;
        if (lane == 0)
          got = mbar_wait(&tfull[bset], (seg_count >> 1) & 1, abort_flag, wait_ns) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        fence_after();
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(bset * ACC_COLS + half * EPC);
        // the fold of this set overlaps the MMAs of the next segment into the other set
#pragma unroll 1
        for (int g = 0; g < GROUPS; ++g) {
          uint32_t r[EPC];
          tmem_ld16(tbase + (uint32_t)(g * BN), r);
#pragma unroll
          for (int j = 0; j < EPC; ++j)
            acc[j] = fma((double)__uint_as_float(r[j]), pow2(ex[j] - 6 * g), acc[j]);
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[bset]);
        ++seg_count;
      }
      if (!ok) break;
      if (row < epi.n_rows) {
        const int I = epi.row_tile_of[row];
        const int mI = epi.row_off[I + 1] - epi.row_off[I];
        const int64_t rowbase = (int64_t)epi.row_off[I] * epi.n_cols + (row - epi.row_off[I]);
        const int* route_row = epi.t_route + (int64_t)I * epi.nJ;
#pragma unroll
        for (int j = 0; j < EPC; ++j) {
          const int64_t col = col0 + j;
          if (col < epi.n_cols) {
            const int J = epi.col_tile_of[col];
            const int route = route_row[J];
            if (route == ROUTE_DENSE || route == ROUTE_DACC_G) {
              double* o = epi.pool + rowbase + col * mI;
              *o = accumulate ? *o + acc[j] : acc[j];
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// GEMM tile t is active when it overlaps at least one C tile the GEMM forms: one with a
// dense x dense product, or a densely accumulated low-rank sum routed to the tensor cores.
__global__ void oz_tile_active_kernel(const int* row_tile_of, const int* col_tile_of, int nc,
                                      const int* t_route, int n_m, int n_n, int64_t n_rows,
                                      int64_t n_cols, unsigned char* active) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_m * n_n) return;
  int mb, nb;
  tile_coords(t, n_m, n_n, &mb, &nb);
  const int64_t r0 = (int64_t)mb * BM, r1 = (r0 + BM < n_rows) ? r0 + BM : n_rows;
  const int64_t c0 = (int64_t)nb * BN, c1 = (c0 + BN < n_cols) ? c0 + BN : n_cols;
  unsigned char on = 0;
  if (r0 < n_rows && c0 < n_cols) {
    const int i0 = row_tile_of[r0], i1 = row_tile_of[r1 - 1];
    const int j0 = col_tile_of[c0], j1 = col_tile_of[c1 - 1];
    for (int I = i0; I <= i1 && !on; ++I)
      for (int J = j0; J <= j1; ++J)
        if (t_route[(int64_t)I * nc + J] == ROUTE_DENSE ||
            t_route[(int64_t)I * nc + J] == ROUTE_DACC_G) {
          on = 1;
          break;
        }
  }
  active[t] = on;
}

// The active tiles' ids in raster order: out[0] = their number, out[1..] = the ids (one CTA
// of 1024 threads, a ballot and warp scan per chunk of 1024 flags).  The persistent GEMM CTAs
// then stride over active tiles only, so each gets the same number of tiles whatever the
// pattern of inactive ones.
__global__ void __launch_bounds__(1024) oz_compact_kernel(const unsigned char* flags, int n,
                                                          int* out) {
  __shared__ int ws[32];
  __shared__ int chunk_total;
  __shared__ int base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const int f = i < n ? flags[i] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, f != 0);
    const int pre = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) ws[wid] = __popc(m);
    __syncthreads();
    if (wid == 0) {
      const int v = ws[lane];
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      ws[lane] = incl - v;
      if (lane == 31) chunk_total = incl;
    }
    __syncthreads();
    if (f) out[1 + base + ws[wid] + pre] = i;
    __syncthreads();
    if (threadIdx.x == 0) base += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = base;
}

// ---------------------------------------------------------------------------------------------
// Staging: exponents, then digits.  Dense blocks and the reconstructions X W^T of low-rank
// blocks are staged (zero blocks stay zero), so that the GEMM forms the whole sum
// sum_K A_IK B_KJ of every C tile it serves.  Exponents are per row (of A) or column (of B)
// and K segment of SEG_K: exps[segment * rows_pad + row].
// ---------------------------------------------------------------------------------------------
// x with |a| < 2^x for a finite nonzero a (from the FP64 exponent field; subnormals count as
// 2^-1022), or INT_MIN for zero.
__device__ __forceinline__ int exp_bound(double a) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const int E = (int)((bits >> 52) & 0x7FF);
  if ((bits << 1) == 0) return INT_MIN;
  return (E ? E : 1) - 1022;
}

// The 8 balanced digits of a relative to 2^e (see the file header), as bf16 bit patterns,
// most significant first.
__device__ __forceinline__ void oz_digits(double a, int e, unsigned short (&out)[S]) {
  long long v = 0;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  if ((bits << 1) != 0 && e > -1100) {
    const int E = (int)((bits >> 52) & 0x7FF);
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (E ? (1ull << 52) : 0ull);
    const int x = (E ? E : 1) - 1075;          // |a| = mant 2^x
    const int sh = x - e + 47;                 // v = mant 2^sh, < 2^47 since |a| < 2^e
    unsigned long long m;
    if (sh >= 0) m = mant << sh;
    else if (sh > -63) m = (mant + (1ull << (-sh - 1))) >> (-sh);   // nearest, ties up
    else m = 0;
    v = (bits >> 63) ? -(long long)m : (long long)m;
  }
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const long long d = ((v + 32) & 63) - 32;
    out[s] = (unsigned short)(__float_as_uint((float)d) >> 16);
    v = (v - d) >> 6;
  }
  out[0] = (unsigned short)(__float_as_uint((float)v) >> 16);
}

// A: exponent of every row over its dense blocks, per K segment.  32 rows x 256 k per CTA
// (threads along rows: the block-row panels are column-major).
__global__ void __launch_bounds__(256) oz_exp_a_kernel(MatView M, const int* row_idx,
                                                       const int* col_idx, int* ea,
                                                       int64_t rows_pad, int64_t cols_pad) {
  __shared__ int red[8][32];
  const int64_t tiles_r = rows_pad / 32;
  const int64_t r = (int64_t)(blockIdx.x % tiles_r) * 32 + threadIdx.x % 32;
  const int64_t k0 = (int64_t)(blockIdx.x / tiles_r) * 256;
  const int ty = threadIdx.x / 32;
  int e = INT_MIN;
  if (r < M.n_rows) {
    const int R = row_idx[r];
    const int mR = M.row_off[R + 1] - M.row_off[R];
    const int64_t rbase = (int64_t)M.row_off[R] * M.n_cols + (r - M.row_off[R]);
    const int* kind_row = M.kind + (int64_t)R * M.nc;
    for (int i = 0; i < 32; ++i) {
      const int64_t k = k0 + ty + 8 * i;
      if (k < M.n_cols && kind_row[col_idx[k]] == CLR_KIND_DENSE)
        e = max(e, exp_bound(M.pool[rbase + k * mR]));
    }
  }
  red[ty][threadIdx.x % 32] = e;
  __syncthreads();
  if (ty == 0) {
    for (int i = 1; i < 8; ++i) e = max(e, red[i][threadIdx.x % 32]);
    if (r < rows_pad && e != INT_MIN) atomicMax(&ea[(k0 / SEG_K) * rows_pad + r], e);
  }
}

// B: exponent of every panel row j (column j of B) over k: one CTA per (j, K segment).
__global__ void __launch_bounds__(256) oz_exp_b_kernel(MatView M, const int* row_idx,
                                                       const int* col_idx, int* eb,
                                                       int64_t rows_pad, int64_t cols_pad) {
  __shared__ int red[8];
  const int64_t j = blockIdx.x;
  int e = INT_MIN;
  if (j < M.n_cols) {
    const int Cc = col_idx[j];
    for (int q = 0; q < 4; ++q) {
      const int64_t k = ((int64_t)blockIdx.y * 1024) + q * 256 + threadIdx.x;
      if (k < M.n_rows && k < cols_pad) {
        const int R = row_idx[k];
        if (M.kind[R * M.nc + Cc] == CLR_KIND_DENSE) {
          const int mR = M.row_off[R + 1] - M.row_off[R];
          e = max(e, exp_bound(M.pool[(int64_t)M.row_off[R] * M.n_cols + (k - M.row_off[R]) +
                                      j * mR]));
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < 8; ++i) e = max(e, red[i]);
    if (e != INT_MIN) atomicMax(&eb[(int64_t)blockIdx.y * rows_pad + j], e);
  }
}

// A digits: a 32 (rows) x 128 (k) tile through shared memory (column-major source, K-major
// panel), 4 consecutive k per thread and plane.
__global__ void __launch_bounds__(256) oz_digits_a_kernel(MatView M, const int* row_idx,
                                                          const int* col_idx, const int* ea,
                                                          unsigned short* panels,
                                                          int64_t rows_pad, int64_t cols_pad) {
  constexpr int TK = 128;
  __shared__ double tile[32][TK + 1];
  __shared__ int s_col[TK];
  const int64_t tiles_r = rows_pad / 32;
  const int64_t r0 = (int64_t)(blockIdx.x % tiles_r) * 32;
  const int64_t k0 = (int64_t)(blockIdx.x / tiles_r) * TK;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
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
  if (threadIdx.x < TK)
    s_col[threadIdx.x] = k0 + threadIdx.x < M.n_cols ? col_idx[k0 + threadIdx.x] : -1;
  __syncthreads();
  for (int i = 0; i < TK / 8; ++i) {
    const int cc = ty + 8 * i;
    const int C = s_col[cc];
    tile[tx][cc] =
        rin && C >= 0 && kind_row[C] == CLR_KIND_DENSE ? M.pool[rbase + (k0 + cc) * mR] : 0.0;
  }
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = r0 + rr;
    const int e = ea[(k0 / SEG_K) * rows_pad + i];
    const int64_t k = k0 + 4 * tx;
    unsigned long long packed[S];
#pragma unroll
    for (int t = 0; t < S; ++t) packed[t] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned short d[S];
      oz_digits(tile[rr][4 * tx + q], e, d);
#pragma unroll
      for (int t = 0; t < S; ++t) packed[t] |= (unsigned long long)d[t] << (16 * q);
    }
#pragma unroll
    for (int t = 0; t < S; ++t)
      *reinterpret_cast<unsigned long long*>(panels + t * plane + i * cols_pad + k) = packed[t];
  }
}

// B digits: panel[j][k] = B(k, j); 4 consecutive k per thread (contiguous in the source).
__global__ void __launch_bounds__(256) oz_digits_b_kernel(MatView M, const int* row_idx,
                                                          const int* col_idx, const int* eb,
                                                          unsigned short* panels,
                                                          int64_t rows_pad, int64_t cols_pad) {
  const int64_t j = blockIdx.x;
  const int64_t k = ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * 4;
  if (k >= cols_pad) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < M.n_cols) {
    const int Cc = col_idx[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t kk = k + q;
      if (kk < M.n_rows) {
        const int R = row_idx[kk];
        if (M.kind[R * M.nc + Cc] == CLR_KIND_DENSE) {
          const int mR = M.row_off[R + 1] - M.row_off[R];
          v[q] = M.pool[(int64_t)M.row_off[R] * M.n_cols + (kk - M.row_off[R]) + j * mR];
        }
      }
    }
  }
  const int e = eb[(int64_t)blockIdx.y * rows_pad + j];   // blockIdx.y: the K segment
  unsigned long long packed[S];
#pragma unroll
  for (int t = 0; t < S; ++t) packed[t] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned short d[S];
    oz_digits(v[q], e, d);
#pragma unroll
    for (int t = 0; t < S; ++t) packed[t] |= (unsigned long long)d[t] << (16 * q);
  }
  const int64_t plane = rows_pad * cols_pad;
#pragma unroll
  for (int t = 0; t < S; ++t)
    *reinterpret_cast<unsigned long long*>(panels + t * plane + j * cols_pad + k) = packed[t];
}

// Low-rank blocks: their reconstructions X W^T, once, in FP64 into a scratch image of M laid
// out like its pool (block (R, C) at row_off[R] n_cols + m col_off[C], column-major): one CTA
// per block of M (blocks of another kind return at once), the register-tiled CTA product.
// Then the exponents and the digits read the image.  a_mode: panel row = M's row, panel k =
// M's column (threads along j); else panel row = M's column, panel k = M's row (threads along
// i).
struct LrBlock {
  const double* v;   // the reconstruction (m x n, ld m)
  int m, n;
  int64_t row0, col0;
};
__device__ __forceinline__ bool lr_block(const MatView& M, const double* recon, int b,
                                         LrBlock* o) {
  if (M.kind[b] != CLR_KIND_LR) return false;
  const int R = b / M.nc, Cc = b % M.nc;
  o->m = M.row_off[R + 1] - M.row_off[R];
  o->n = M.col_off[Cc + 1] - M.col_off[Cc];
  o->v = recon + (int64_t)M.row_off[R] * M.n_cols + (int64_t)o->m * M.col_off[Cc];
  o->row0 = M.row_off[R];
  o->col0 = M.col_off[Cc];
  return true;
}

__global__ void __launch_bounds__(256) oz_lr_recon_kernel(MatView M, double* recon) {
  const int b = blockIdx.x;
  if (M.kind[b] != CLR_KIND_LR) return;
  const int R = b / M.nc, Cc = b % M.nc;
  const int m = M.row_off[R + 1] - M.row_off[R];
  const int n = M.col_off[Cc + 1] - M.col_off[Cc];
  const int r = M.rank[b];
  const int64_t slot = (int64_t)M.row_off[R] * M.n_cols + (int64_t)m * M.col_off[Cc];
  const double* x = M.pool + slot;             // m x r, ld m
  const double* w = x + (int64_t)m * r;        // n x r, ld n
  // out(i, j) = sum_q X(i, q) W(j, q)
  cta_gemm_tiled<256>(m, n, r, x, 1, m, w, n, 1, recon + slot, m, false);
}

__global__ void __launch_bounds__(256) oz_exp_lr_kernel(MatView M, const double* recon,
                                                        int* exps, int64_t rows_pad,
                                                        int a_mode) {
  __shared__ int red[CLR_MAX_CLUSTER][2];   // per panel row: the block's (at most) 2 segments
  LrBlock L;
  if (!lr_block(M, recon, blockIdx.x, &L)) return;
  const int np = a_mode ? L.m : L.n;
  const int64_t k0 = a_mode ? L.col0 : L.row0;    // the block's first panel k
  const int s0 = (int)(k0 / SEG_K);
  for (int i = threadIdx.x; i < np; i += blockDim.x) red[i][0] = red[i][1] = INT_MIN;
  __syncthreads();
  for (int e = threadIdx.x; e < L.m * L.n; e += blockDim.x) {
    const int i = a_mode ? e / L.n : e % L.m;
    const int j = a_mode ? e % L.n : e / L.m;
    const int x = exp_bound(L.v[i + (int64_t)j * L.m]);
    const int64_t k = k0 + (a_mode ? j : i);
    if (x != INT_MIN) atomicMax(&red[a_mode ? i : j][(int)(k / SEG_K) - s0], x);
  }
  __syncthreads();
  const int64_t p0 = a_mode ? L.row0 : L.col0;
  for (int i = threadIdx.x; i < np; i += blockDim.x)
    for (int h = 0; h < 2; ++h)
      if (red[i][h] != INT_MIN) atomicMax(&exps[(int64_t)(s0 + h) * rows_pad + p0 + i], red[i][h]);
}

__global__ void __launch_bounds__(256) oz_digits_lr_kernel(MatView M, const double* recon,
                                                           const int* exps,
                                                           unsigned short* panels,
                                                           int64_t rows_pad, int64_t cols_pad,
                                                           int a_mode) {
  LrBlock L;
  if (!lr_block(M, recon, blockIdx.x, &L)) return;
  const int64_t plane = rows_pad * cols_pad;
  for (int e = threadIdx.x; e < L.m * L.n; e += blockDim.x) {
    const int i = a_mode ? e / L.n : e % L.m;
    const int j = a_mode ? e % L.n : e / L.m;
    const int64_t prow = a_mode ? L.row0 + i : L.col0 + j;
    const int64_t k = a_mode ? L.col0 + j : L.row0 + i;
    unsigned short d[S];
    oz_digits(L.v[i + (int64_t)j * L.m], exps[(k / SEG_K) * rows_pad + prow], d);
#pragma unroll
    for (int t = 0; t < S; ++t) panels[t * plane + prow * cols_pad + k] = d[t];
  }
}

// Per cluster and K segment: the sum over the cluster's rows (columns) of 4^e, e their
// exponents in that segment (rows without entries there count 0; past 2^1023 the sum is
// infinite, which routes nothing to the GEMM).  One warp per (cluster, segment).
__global__ void oz_scale_sums_kernel(const int* exps, int64_t rows_pad, const int* off, int n_cl,
                                     int n_seg, double* out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (t >= (int64_t)n_cl * n_seg) return;
  const int c = (int)(t / n_seg), sg = (int)(t % n_seg);
  double sum = 0.0;
  for (int i = off[c] + lane; i < off[c + 1]; i += 32) {
    const int e = exps[(int64_t)sg * rows_pad + i];
    if (e > -1100) sum += ldexp(1.0, 2 * e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) out[t] = sum;
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                             const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                             const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_panel(EncodeFn fn, CUtensorMap* tm, void* base, int64_t k_pad, int64_t rows,
                  uint32_t box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(k_pad * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace oz

void launch_ozaki_stage(const MatView& M, const int* row_idx, const int* col_idx, void* panels,
                        int* exps, double* recon, int64_t rows_pad, int64_t cols_pad,
                        int a_mode, cudaStream_t st) {
  using namespace oz;
  unsigned short* pn = (unsigned short*)panels;
  // sentinel exponent (bytes 0x80: a large negative int) for rows without entries in a segment
  const int64_t n_seg = (cols_pad + SEG_K - 1) / SEG_K;
  cudaMemsetAsync(exps, 0x80, (size_t)(n_seg * rows_pad) * sizeof(int), st);
  const unsigned nb = (unsigned)(M.nr * M.nc);
  if (a_mode) {
    const unsigned ne = (unsigned)((rows_pad / 32) * ((cols_pad + 255) / 256));
    oz_exp_a_kernel<<<ne, 256, 0, st>>>(M, row_idx, col_idx, exps, rows_pad, cols_pad);
  } else {
    const dim3 ne((unsigned)rows_pad, (unsigned)n_seg);
    oz_exp_b_kernel<<<ne, 256, 0, st>>>(M, row_idx, col_idx, exps, rows_pad, cols_pad);
  }
  oz_lr_recon_kernel<<<nb, 256, 0, st>>>(M, recon);
  oz_exp_lr_kernel<<<nb, 256, 0, st>>>(M, recon, exps, rows_pad, a_mode);
  if (a_mode) {
    const unsigned nd = (unsigned)((rows_pad / 32) * (cols_pad / 128));
    oz_digits_a_kernel<<<nd, 256, 0, st>>>(M, row_idx, col_idx, exps, pn, rows_pad, cols_pad);
  } else {
    const dim3 nd((unsigned)rows_pad, (unsigned)((cols_pad / 4 + 255) / 256));
    oz_digits_b_kernel<<<nd, 256, 0, st>>>(M, row_idx, col_idx, exps, pn, rows_pad, cols_pad);
  }
  // (after the dense pass, which writes zeros at the low-rank blocks' entries)
  oz_digits_lr_kernel<<<nb, 256, 0, st>>>(M, recon, exps, pn, rows_pad, cols_pad, a_mode);
}

void launch_ozaki_scale_sums(const int* exps, int64_t rows_pad, const int* off, int n_cl,
                             int n_seg, double* out, cudaStream_t st) {
  const int64_t warps = (int64_t)n_cl * n_seg;
  oz::oz_scale_sums_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
      exps, rows_pad, off, n_cl, n_seg, out);
}

int ozaki_gemm_dd(const OzakiGemmArgs& a, cudaStream_t st, std::string* why) {
  using namespace oz;
  if (!a.encode_fn) {
    if (why) *why = "driver TMA encoder unavailable";
    return CLR_ENOTSUP;
  }
  if (a.M_pad % BM || a.N_pad % BN || a.K_pad % 128 || (int64_t)S * a.M_pad > (1ll << 31) ||
      (int64_t)S * a.N_pad > (1ll << 31)) {
    if (why) *why = "bad panel padding";
    return CLR_EINVAL;
  }
  EncodeFn fn = (EncodeFn)a.encode_fn;
  CUtensorMap tmA, tmB;
  if (!encode_panel(fn, &tmA, a.a_panels, a.K_pad, (int64_t)S * a.M_pad, BM) ||
      !encode_panel(fn, &tmB, a.b_panels, a.K_pad, (int64_t)S * a.N_pad, BN)) {
    if (why) *why = "cuTensorMapEncodeTiled failed";
    return CLR_ECUDA;
  }
  const int n_m = (int)(a.M_pad / BM), n_n = (int)(a.N_pad / BN);
  const int num_k = (int)(a.K_pad / BK);
  const MatView& C = *a.C;
  oz_tile_active_kernel<<<(n_m * n_n + 127) / 128, 128, 0, st>>>(
      a.row_tile_of, a.col_tile_of, C.nc, a.p->t_route, n_m, n_n, C.n_rows, C.n_cols,
      a.tile_active);
  oz_compact_kernel<<<1, 1024, 0, st>>>(a.tile_active, n_m * n_n, a.active_list);
  Epi epi;
  epi.pool = C.pool;
  epi.row_off = C.row_off;
  epi.row_tile_of = a.row_tile_of;
  epi.col_tile_of = a.col_tile_of;
  epi.t_route = a.p->t_route;
  epi.ea = a.ea;
  epi.eb = a.eb;
  epi.nJ = C.nc;
  epi.n_rows = C.n_rows;
  epi.n_cols = C.n_cols;
  // set once per device (outside any stream capture the first time a product runs)
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_TOTAL);
    if (e != cudaSuccess) {
      if (why) *why = cudaGetErrorString(e);
      return CLR_ECUDA;
    }
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
  }
  const int grid = std::max(1, std::min(a.n_sm, n_m * n_n));
  // K in passes of kPassSegments segments, the later passes adding into C: the CTAs of a wave
  // share their operand slabs through L2 only while they are at about the same k, and over a
  // long K they drift apart (at N = 32768 in one pass the kernel streamed every slab from
  // DRAM); a pass's slabs for one wave, (8 x 128 + 19 x 32) rows x 2048 x 16 B = 53 MB, stay
  // in L2.  Each later pass reads and writes C once more (16 N^2 bytes).
  const int pass = kPassSegments * SEG_CHUNKS;
  for (int k0 = 0; k0 < num_k; k0 += pass) {
    ozaki_gemm_kernel<<<grid, THREADS, SMEM_TOTAL, st>>>(
        tmA, tmB, epi, n_m, n_n, k0, std::min(num_k, k0 + pass), k0 > 0 ? 1 : 0,
        (int)a.M_pad, (int)a.N_pad, a.active_list, a.err, a.wait_ns > 0 ? a.wait_ns : kDrainNs);
  }
  return CLR_OK;
}

}  // namespace clr
