// K1 (split precision) -- dense x dense tile products on the 5th-generation tensor cores.
//
// The dense blocks of A and B are staged as bf16 term panels (k_split_stage.cu); the product
// of the dense parts is sum_{(p,q)} A_p B_q^T over the term pairs of the split (bf16x3:
// (0,0) (0,1) (1,0); bf16x6: every p + q <= 2), accumulated in FP32 in tensor memory.  The
// epilogue converts to FP64 and writes only into C tiles whose route is dense (tiles with a
// dense x dense contribution, Section 3.2's GEMM update); other regions of the GEMM grid are
// discarded, and GEMM tiles that touch no dense C tile are skipped.
//
// Kernel structure (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0      TMA producer: per 32-wide k chunk loads every term tile of A (128 x 32) and
//               B (256 x 32) with 64-byte swizzle into one pipeline stage;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and issues
//               tcgen05.mma (M=128, N=256, K=16, kind::f16, bf16 in, f32 accumulate);
//   warps 2-9   epilogue: two warps per TMEM lane quarter, each owning 128 of the 256 columns.
//
// Accumulation in segments: the tensor core's FP32 accumulation loses about 2^-26 of the
// partial sum per MMA (measured), so a chain of thousands of MMAs into one accumulator costs
// ~1e-4 relative accuracy.  The k loop of a tile is therefore cut into segments of about 96
// MMAs; the MMA warp alternates the two TMEM accumulators segment by segment, and the
// epilogue adds each finished segment into FP32 registers with round-to-nearest adds (128
// per thread) while the next segment runs.  After the last segment the registers are
// converted to FP64 and stored into the C block pool (column-major blocks: consecutive lanes
// -> consecutive rows).
// Every mbarrier wait is bounded (wait_ns of %globaltimer, 2 s unless the context sets another
// limit); on a timeout the kernel raises the error flag, stops issuing work, waits (bounded by
// a fixed 2 s, whatever wait_ns is) for its copies and MMAs in flight, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "clr_internal.h"

namespace clr {

namespace sg {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 32;               // 32 bf16 = 64 bytes: one 64B-swizzle row
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t A_TILE = BM * BK * 2;
constexpr uint32_t B_TILE = BN * BK * 2;
constexpr int TMEM_COLS = 512;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

template <int TERMS>
struct Cfg {
  static constexpr uint32_t STAGE = TERMS * (A_TILE + B_TILE);
  static constexpr int STAGES = TERMS == 2 ? 4 : 3;
  static constexpr int NPAIRS = TERMS == 2 ? 3 : 6;
  // k chunks per accumulation segment: NPAIRS * (BK/16) * SEG = 96 MMAs
  static constexpr int SEG = TERMS == 2 ? 16 : 8;
  static constexpr uint32_t SMEM_DATA = STAGE * STAGES;
  static constexpr uint32_t SMEM_TOTAL = SMEM_DATA + 1024 /*barriers*/ + 1024 /*align*/;
};

__device__ __forceinline__ int pair_a(int terms, int i) {
  // bf16x3: (0,0) (0,1) (1,0);  bf16x6: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  const int a3[3] = {0, 0, 1};
  const int a6[6] = {0, 0, 1, 0, 1, 2};
  return terms == 2 ? a3[i] : a6[i];
}
__device__ __forceinline__ int pair_b(int terms, int i) {
  const int b3[3] = {0, 1, 0};
  const int b6[6] = {0, 1, 0, 2, 1, 0};
  return terms == 2 ? b3[i] : b6[i];
}

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
// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Epi {
  double* pool;
  const int* row_off;
  const int* col_off;
  const int* row_tile_of;
  const int* col_tile_of;
  const int* t_route;
  int nJ;
  int64_t n_rows, n_cols;
  // Fused norms (may be null): sums of squares of the values written into route-DENSE C tiles,
  // added per tile (I, J) into norm_sq[I * nJ + J].  Set only when every row cluster has >= 32
  // rows (a warp's rows span at most two) and every column cluster >= 16 columns (a 16-column
  // group spans at most two).
  double* norm_sq;
};

// Adds a warp's partial sums of squares for C column cluster J: lanes whose row cluster is the
// warp's first (I0) and the others (all in I1, at most two clusters per warp) are summed apart;
// lane 0 adds each nonzero total to its tile.  Uniform in the warp.
__device__ __forceinline__ void norm_flush(const Epi& epi, int I, int I0, int I1, int J,
                                           double acc, int lane) {
  if (J < 0) return;
  double a = I == I0 ? acc : 0.0;
  double b = I == I0 ? 0.0 : acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    if (a != 0.0 && I0 >= 0) atomicAdd(&epi.norm_sq[(int64_t)I0 * epi.nJ + J], a);
    if (b != 0.0 && I1 >= 0 && I1 != I0) atomicAdd(&epi.norm_sq[(int64_t)I1 * epi.nJ + J], b);
  }
}

// Linear tile id -> (m block, n block), grouped along m for L2 reuse across concurrent CTAs.
__device__ __forceinline__ void tile_coords(int id, int n_m, int n_n, int* mb, int* nb) {
  constexpr int G = 16;
  const int per_group = G * n_n;
  const int g = id / per_group;
  const int first = g * G;
  const int gs = min(G, n_m - first);
  const int r = id - g * per_group;
  *mb = first + r % gs;
  *nb = r / gs;
}

template <int TERMS, bool NORMS>
__global__ void __launch_bounds__(THREADS, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, Epi epi, int n_m, int n_n,
                      int num_k, int M_pad, int N_pad, const unsigned char* tile_active,
                      int* err, unsigned long long wait_ns) {
  using C = Cfg<TERMS>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::SMEM_DATA);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_holder = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n_tiles = n_m * n_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
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
      uint32_t issued_parity[C::STAGES];
      bool issued[C::STAGES];
      for (int i = 0; i < C::STAGES; ++i) issued[i] = false;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
        if (!tile_active[tile]) continue;
        int mb, nb;
        tile_coords(tile, n_m, n_n, &mb, &nb);
        for (int kc = 0; kc < num_k; ++kc) {
          if (!mbar_wait(&empty[s], phase ^ 1, abort_flag, wait_ns)) { ok = false; break; }
          unsigned char* st = smem + (size_t)s * C::STAGE;
          mbar_expect_tx(&full[s], C::STAGE);
          issued[s] = true;
          issued_parity[s] = phase;
          for (int t = 0; t < TERMS; ++t)
            tma_load_2d(st + t * A_TILE, &tmA, kc * BK, t * M_pad + mb * BM, &full[s]);
          for (int t = 0; t < TERMS; ++t)
            tma_load_2d(st + TERMS * A_TILE + t * B_TILE, &tmB, kc * BK, t * N_pad + nb * BN,
                        &full[s]);
          if (++s == C::STAGES) { s = 0; phase ^= 1; }
        }
      }
      if (!ok) {
        // copies in flight land before the CTA exits (bounded)
        volatile int no_abort = 0;
        for (int i = 0; i < C::STAGES; ++i)
          if (issued[i]) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try(&full[i], issued_parity[i]) && gtimer() - t0 < kTimeoutNs) {
            }
          }
        (void)no_abort;
        atomicExch(err, 1);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t phase = 0;
      int seg_count = 0;  // segments issued by this CTA (accumulator = seg_count & 1)
      bool ok = true;
      bool any = false;
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
        if (!tile_active[tile]) continue;
        for (int k0 = 0; ok && k0 < num_k; k0 += C::SEG) {
          const int k1 = min(num_k, k0 + C::SEG);
          const int b = seg_count & 1;
          const uint32_t tp = (seg_count >> 1) & 1;
          if (!mbar_wait(&tempty[b], tp ^ 1, abort_flag, wait_ns)) { ok = false; break; }
          fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
          for (int kc = k0; kc < k1; ++kc) {
            if (!mbar_wait(&full[s], phase, abort_flag, wait_ns)) { ok = false; break; }
            fence_after();
            const uint32_t st = saddr(smem + (size_t)s * C::STAGE);
#pragma unroll
            for (int pi = 0; pi < C::NPAIRS; ++pi) {
              const uint32_t a_addr = st + pair_a(TERMS, pi) * A_TILE;
              const uint32_t b_addr = st + TERMS * A_TILE + pair_b(TERMS, pi) * B_TILE;
#pragma unroll
              for (int k16 = 0; k16 < BK / 16; ++k16) {
                umma_bf16(d_tmem, sdesc(a_addr + k16 * 32), sdesc(b_addr + k16 * 32), kIdesc,
                          ((kc - k0) | pi | k16) != 0 ? 1u : 0u);
              }
            }
            umma_commit(&empty[s]);
            any = true;
            if (++s == C::STAGES) { s = 0; phase ^= 1; }
          }
          if (!ok) break;
          umma_commit(&tfull[b]);
          ++seg_count;
        }
      }
      if (!ok) {
        if (any) {
          // wait (bounded) for the MMAs already issued before TMEM is released
          umma_commit(drain);
          const unsigned long long t0 = gtimer();
          while (!mbar_try(drain, 0) && gtimer() - t0 < kTimeoutNs) {
          }
        }
        atomicExch(err, 1);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    const int quarter = warp % 4;          // TMEM lanes 32*quarter .. 32*quarter+31
    const int half = (warp - 2) / 4;       // columns 128*half .. 128*half+127
    const int rl = quarter * 32 + lane;    // row within the tile
    int seg_count = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
      if (!tile_active[tile]) continue;
      int mb, nb;
      tile_coords(tile, n_m, n_n, &mb, &nb);
      float hi[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) hi[j] = 0.f;
      for (int k0 = 0; k0 < num_k; k0 += C::SEG) {
        const int b = seg_count & 1;
        const uint32_t tp = (seg_count >> 1) & 1;
        int got = 0;
        if (lane == 0) got = mbar_wait(&tfull[b], tp, abort_flag, wait_ns) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        fence_after();
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(b * BN + half * 128);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint32_t r[16];
          tmem_ld16(tbase + (uint32_t)(c * 16), r);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            hi[c * 16 + j] = __fadd_rn(hi[c * 16 + j], __uint_as_float(r[j]));
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        ++seg_count;
      }
      if (!ok) break;
      const int64_t row = (int64_t)mb * BM + rl;
      const int64_t col0 = (int64_t)nb * BN + half * 128;
      if constexpr (!NORMS) {
        if (row < epi.n_rows) {
          const int I = epi.row_tile_of[row];
          const int mI = epi.row_off[I + 1] - epi.row_off[I];
          const int64_t rowbase = (int64_t)epi.row_off[I] * epi.n_cols + (row - epi.row_off[I]);
          const int* route_row = epi.t_route + (int64_t)I * epi.nJ;
#pragma unroll
          for (int j = 0; j < 128; ++j) {
            const int64_t col = col0 + j;
            if (col < epi.n_cols) {
              const int J = epi.col_tile_of[col];
              if (route_row[J] == ROUTE_DENSE || route_row[J] == ROUTE_DACC_G)
                epi.pool[rowbase + col * mI] = (double)hi[j];
            }
          }
        }
      } else {
        // the same stores, with the sums of squares of route-DENSE values per C tile: per
        // 16-column group (its first and last column clusters Jf, Jl are uniform in the warp),
        // one FP64 partial sum, two where the group crosses a cluster boundary
        const bool valid = row < epi.n_rows;
        int I = -1, mI = 1;
        int64_t rowbase = 0;
        const int* route_row = epi.t_route;
        if (valid) {
          I = epi.row_tile_of[row];
          mI = epi.row_off[I + 1] - epi.row_off[I];
          rowbase = (int64_t)epi.row_off[I] * epi.n_cols + (row - epi.row_off[I]);
          route_row = epi.t_route + (int64_t)I * epi.nJ;
        }
        const int I0 = __shfl_sync(0xffffffffu, I, 0);
        const int I1 = __reduce_max_sync(0xffffffffu, I);
        double acc = 0.0;
        int acc_j = -1;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t cb = col0 + 16 * c;
          if (cb < epi.n_cols) {
            const int64_t ce = cb + 15 < epi.n_cols ? cb + 15 : epi.n_cols - 1;
            const int Jf = epi.col_tile_of[cb], Jl = epi.col_tile_of[ce];
            double sa = 0.0, sb = 0.0;
            if (Jf == Jl) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int64_t col = cb + jj;
                if (valid && col < epi.n_cols) {
                  const int r = route_row[Jf];
                  if (r == ROUTE_DENSE || r == ROUTE_DACC_G) {
                    const double v = (double)hi[16 * c + jj];
                    epi.pool[rowbase + col * mI] = v;
                    if (r == ROUTE_DENSE) sa = fma(v, v, sa);
                  }
                }
              }
            } else {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int64_t col = cb + jj;
                if (valid && col < epi.n_cols) {
                  const int J = epi.col_tile_of[col];
                  const int r = route_row[J];
                  if (r == ROUTE_DENSE || r == ROUTE_DACC_G) {
                    const double v = (double)hi[16 * c + jj];
                    epi.pool[rowbase + col * mI] = v;
                    if (r == ROUTE_DENSE) {
                      if (J == Jf) sa = fma(v, v, sa);
                      else sb = fma(v, v, sb);
                    }
                  }
                }
              }
            }
            if (Jf != acc_j) {
              norm_flush(epi, I, I0, I1, acc_j, acc, lane);
              acc = 0.0;
              acc_j = Jf;
            }
            acc += sa;
            if (Jl != Jf) {
              norm_flush(epi, I, I0, I1, acc_j, acc, lane);
              acc = sb;
              acc_j = Jl;
            }
          }
        }
        norm_flush(epi, I, I0, I1, acc_j, acc, lane);
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

// GEMM tile t is active when it overlaps at least one C tile the GEMM sums (route DENSE or
// DACC_G).
__global__ void tile_active_kernel(const int* row_tile_of, const int* col_tile_of, int nc,
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

template <int TERMS, bool NORMS>
int launch_terms(const SplitGemmArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB,
                 const Epi& epi, int n_m, int n_n, int num_k, cudaStream_t st,
                 std::string* why) {
  const uint32_t smem = Cfg<TERMS>::SMEM_TOTAL;
  // set once per device (outside any stream capture the first time a product runs)
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(split_gemm_kernel<TERMS, NORMS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      if (why) *why = cudaGetErrorString(e);
      return CLR_ECUDA;
    }
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
  }
  const int grid = std::max(1, std::min(a.n_sm, n_m * n_n));
  split_gemm_kernel<TERMS, NORMS><<<grid, THREADS, smem, st>>>(
      tmA, tmB, epi, n_m, n_n, num_k, (int)a.M_pad, (int)a.N_pad, a.tile_active, a.err,
      a.wait_ns > 0 ? a.wait_ns : kTimeoutNs);
  return CLR_OK;
}

}  // namespace sg

int split_gemm_dd(const SplitGemmArgs& a, cudaStream_t st, std::string* why) {
  using namespace sg;
  if (!a.encode_fn) {
    if (why) *why = "driver TMA encoder unavailable";
    return CLR_ENOTSUP;
  }
  if (a.terms != 2 && a.terms != 3) {
    if (why) *why = "terms must be 2 or 3";
    return CLR_EINVAL;
  }
  if (a.M_pad % BM || a.N_pad % BN || a.K_pad % 64 || (int64_t)a.terms * a.N_pad > (1ll << 31)) {
    if (why) *why = "bad panel padding";
    return CLR_EINVAL;
  }
  EncodeFn fn = (EncodeFn)a.encode_fn;
  CUtensorMap tmA, tmB;
  if (!encode_panel(fn, &tmA, a.a_panels, a.K_pad, (int64_t)a.terms * a.M_pad, BM) ||
      !encode_panel(fn, &tmB, a.b_panels, a.K_pad, (int64_t)a.terms * a.N_pad, BN)) {
    if (why) *why = "cuTensorMapEncodeTiled failed";
    return CLR_ECUDA;
  }
  const int n_m = (int)(a.M_pad / BM), n_n = (int)(a.N_pad / BN);
  const int num_k = (int)(a.K_pad / BK);
  const MatView& C = *a.C;
  tile_active_kernel<<<(n_m * n_n + 127) / 128, 128, 0, st>>>(
      a.row_tile_of, a.col_tile_of, C.nc, a.p->t_route, n_m, n_n, C.n_rows, C.n_cols,
      a.tile_active);
  Epi epi;
  epi.pool = C.pool;
  epi.row_off = C.row_off;
  epi.col_off = C.col_off;
  epi.row_tile_of = a.row_tile_of;
  epi.col_tile_of = a.col_tile_of;
  epi.t_route = a.p->t_route;
  epi.nJ = C.nc;
  epi.n_rows = C.n_rows;
  epi.n_cols = C.n_cols;
  epi.norm_sq = a.norm_sq;
  if (epi.norm_sq) {
    if (a.terms == 2) return launch_terms<2, true>(a, tmA, tmB, epi, n_m, n_n, num_k, st, why);
    return launch_terms<3, true>(a, tmA, tmB, epi, n_m, n_n, num_k, st, why);
  }
  if (a.terms == 2) return launch_terms<2, false>(a, tmA, tmB, epi, n_m, n_n, num_k, st, why);
  return launch_terms<3, false>(a, tmA, tmB, epi, n_m, n_n, num_k, st, why);
}

}  // namespace clr
