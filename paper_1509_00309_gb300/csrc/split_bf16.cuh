// Split of a finite FP64 value into bf16 terms, a = a_0 + a_1 (+ a_2) + residual, with
// a_0 = bf16(a), a_1 = bf16(a - a_0), a_2 = bf16(a - a_0 - a_1), every bf16 rounding to nearest
// with ties to even and taken directly from the exact FP64 difference (no double rounding).
// No FP64 arithmetic (on this part it runs at a small fraction of the integer rate): integer
// operations on the bit patterns, and in the paired form one FP32 -> bf16x2 conversion of
// patterns already rounded to odd.  Host and device compile the same code (the host spells the
// conversion out), so the rounding can be checked on the CPU against the format's definition.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define CLR_SPLIT_FN __host__ __device__ __forceinline__
#else
#define CLR_SPLIT_FN static inline
#include <string.h>
#endif

namespace clr {
namespace split {

CLR_SPLIT_FN int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// The high 32 bits of (hi:lo) << n, 0 <= n < 32.
CLR_SPLIT_FN unsigned funnel_left(unsigned lo, unsigned hi, int n) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, (unsigned)n);
#else
  return (unsigned)(((((unsigned long long)hi) << 32 | lo) << n) >> 32);
#endif
}

CLR_SPLIT_FN int clz32(unsigned x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

CLR_SPLIT_FN unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

// Generic rounding: the value R * 2^s (R a signed integer, |R| < 2^62) to the nearest bf16,
// from the format's definition: 8 significant bits, exponent range of binary32, below the
// smallest normal 2^-126 a fixed spacing of 2^-133.  Returns the bf16 bits and, in *Rr, the
// rounded value in units of 2^s (exact), so the caller can form the residual R - Rr.
CLR_SPLIT_FN unsigned short round_generic(long long R, int s, long long* Rr) {
  if (R == 0) {
    *Rr = 0;
    return 0;
  }
  const unsigned short sign = R < 0 ? 0x8000 : 0;
  const unsigned long long mag = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
  const int msb = 63 - clz64(mag);
  int shift = msb - 7;
  const int sub = -133 - s;
  if (shift < sub) shift = sub;
  unsigned long long q;
  if (shift <= 0) {
    q = mag;  // at most 8 significant bits: exact
    shift = 0;
  } else if (shift > 62) {
    q = 0;
  } else {
    const unsigned long long rem = mag & ((1ull << shift) - 1);
    const unsigned long long half = 1ull << (shift - 1);
    q = mag >> shift;
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  if (q == 0) {
    *Rr = 0;
    return sign;
  }
  const long long rr = (long long)(q << shift);
  *Rr = R < 0 ? -rr : rr;
  const int vexp = s + shift;
  const int qb = 63 - clz64(q);  // <= 8
  const int E = qb + vexp;        // exponent of the leading bit
  if (E < -126) return sign | (unsigned short)(q << (vexp + 133));  // subnormal
  const unsigned mant = qb >= 7 ? (unsigned)(q >> (qb - 7)) & 0x7Fu
                                : (unsigned)(q << (7 - qb)) & 0x7Fu;
  return sign | (unsigned short)((E + 127) << 7) | (unsigned short)mant;
}

// Fast rounding of a lower term: R * 2^s with 0 < |R| < 2^45 and every value involved a normal
// bf16 (s >= -126).  The magnitude is normalised so that its leading bit is bit 63; its top 24
// bits, with a sticky bit for everything below (round to odd), form an FP32 bit pattern, and
// rounding that pattern to nearest-even bf16 is then the correctly rounded bf16 of the exact
// value (24 >= 8 + 2 bits: the sticky bit removes double rounding).  *mag_r: the rounded
// magnitude in units of 2^s.
CLR_SPLIT_FN unsigned short round_lower(unsigned long long mag, int s, unsigned long long* mag_r) {
  const int n = clz64(mag);
  const unsigned long long N = mag << n;
  const unsigned top = (unsigned)(N >> 32);
  const unsigned sticky = ((top & 0xFFu) | (unsigned)N) != 0u;
  const unsigned fe = (unsigned)(190 - n + s);  // biased FP32 exponent of the leading bit
  const unsigned fbits = (fe << 23) | ((top >> 8) & 0x7FFFFFu) | sticky;
  const unsigned bf = (fbits + 0x7FFFu + ((fbits >> 16) & 1u)) >> 16;
  if (mag_r) {
    // leading-bit position of the rounded value in units of 2^s (a carry may raise it by one)
    const int p = (int)(bf >> 7) - 127 - s;
    const unsigned long long q = (bf & 0x7Fu) | 0x80u;
    *mag_r = p >= 7 ? q << (p - 7) : mag;  // below 8 significant bits the value is exact
  }
  return (unsigned short)bf;
}

// a = a_0 + ... + a_{TERMS-1} + residual.  Fast path for biased exponents in
// [1023 - 74, 1023 + 126]: a_0 cannot overflow and every nonzero lower term is a normal bf16
// (its leading bit is at or above a's last significand bit, 2^(e - 52) >= 2^-126).
template <int TERMS>
CLR_SPLIT_FN void split_bf16(double x, unsigned short (&out)[TERMS]) {
  const unsigned long long u = bits_of(x);
  const unsigned E = (unsigned)(u >> 52) & 0x7FFu;
  if (E - (1023u - 74u) <= 200u) {
    const unsigned hiW = (unsigned)(u >> 32), loW = (unsigned)u;
    const unsigned short sx = (unsigned short)((hiW >> 16) & 0x8000u);
    // a_0: round the bit pattern at bit 45 (bit 13 of the high word), ties to even; the carry
    // from the low word is 1 exactly when it or the tie-breaking bit is nonzero
    const unsigned b45 = (hiW >> 13) & 1u;
    const unsigned hi0 = (hiW + 0xFFFu + ((loW | b45) != 0u ? 1u : 0u)) & ~0x1FFFu;
    out[0] = sx | (unsigned short)((((hi0 & 0x7FFFFFFFu) - (896u << 20)) >> 13));
    if (TERMS == 1) return;
    // residual in units of a's last bit, 2^(E - 1075): consecutive doubles of one sign are
    // consecutive integers, so the difference of the bit patterns is the difference of the
    // values, also when rounding carried into the exponent.  |residual| <= 2^44: its high
    // word Rh is a small signed integer.
    const int Rh = (int)(hiW - hi0);
    const bool neg = Rh < 0;
    const unsigned ml = neg ? 0u - loW : loW;
    const unsigned mh = neg ? (unsigned)(-Rh) - (loW != 0u ? 1u : 0u) : (unsigned)Rh;
    const int s = (int)E - 1075;
    const unsigned short s1 = neg ? (unsigned short)(sx ^ 0x8000u) : sx;
    if (mh != 0u) {
      // a_1 by 32-bit operations: normalise the magnitude (leading bit to bit 63), keep its top
      // 24 bits with a sticky bit for the rest (round to odd) as an FP32 pattern, round that
      // to nearest-even bf16 (as in round_lower)
      const int n = clz32(mh);
      const unsigned top = funnel_left(ml, mh, n);
      const unsigned sticky = ((top & 0xFFu) | (ml << n)) != 0u ? 1u : 0u;
      const unsigned fbits = ((unsigned)(190 - n + s) << 23) | ((top >> 8) & 0x7FFFFFu) | sticky;
      const unsigned bf = (fbits + 0x7FFFu + ((fbits >> 16) & 1u)) >> 16;
      out[1] = (unsigned short)(bf | s1);
      if (TERMS == 3) {
        const unsigned long long mag = ((unsigned long long)mh << 32) | ml;
        const int p = (int)(bf >> 7) - 127 - s;  // >= 32 here: the rounded value needs no test
        const unsigned long long mr = (unsigned long long)((bf & 0x7Fu) | 0x80u) << (p - 7);
        const long long d = (long long)(mag - mr);
        if (d == 0) {
          out[TERMS - 1] = 0;
        } else {
          const bool n2 = d < 0;
          const unsigned short b = round_lower(n2 ? (unsigned long long)(-d) : (unsigned long long)d,
                                               s, nullptr);
          out[TERMS - 1] = (unsigned short)(b | (n2 ? s1 ^ 0x8000u : s1));
        }
      }
      return;
    }
    // residual below 2^32 units (rare): the 64-bit path
    long long R = neg ? -(long long)ml : (long long)ml;
#pragma unroll
    for (int t = 1; t < TERMS; ++t) {
      if (R == 0) {
        out[t] = 0;
        continue;
      }
      const bool ng = R < 0;
      const unsigned long long mag = ng ? (unsigned long long)(-R) : (unsigned long long)R;
      unsigned long long mr = 0;
      const unsigned short b = round_lower(mag, s, t + 1 < TERMS ? &mr : nullptr);
      out[t] = (unsigned short)(b | (ng ? sx ^ 0x8000u : sx));
      if (t + 1 < TERMS) {
        const long long d = (long long)(mag - mr);
        R = ng ? -d : d;
      }
    }
    return;
  }
  const long long bits = (long long)u;
  const long long frac = bits & ((1ll << 52) - 1);
  const long long M = E == 0 ? frac : (frac | (1ll << 52));
  const int s = E == 0 ? -1074 : (int)E - 1075;
  long long R = bits < 0 ? -M : M;
#pragma unroll
  for (int t = 0; t < TERMS; ++t) {
    long long rr;
    out[t] = round_generic(R, s, &rr);
    R -= rr;
  }
}

// Round two FP32 bit patterns to nearest-even bf16 and pack them, hi in the upper half: one
// cvt.rn.bf16x2.f32 on the device; the same rounding written out on the host.
CLR_SPLIT_FN unsigned cvt_bf16x2(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
  return r;
#else
  const unsigned h = (hi + 0x7FFFu + ((hi >> 16) & 1u)) >> 16;
  const unsigned l = (lo + 0x7FFFu + ((lo >> 16) & 1u)) >> 16;
  return (h << 16) | l;
#endif
}

// FP32 pattern of a magnitude mag * 2^s (mag != 0) rounded to odd at 24 bits, with sign bit
// `sign` (bit 31): rounding it to nearest-even bf16 gives the correctly rounded bf16 of the
// exact value.  fe_base = 190 + s (the biased exponent when the leading bit is bit 63).
CLR_SPLIT_FN unsigned ro24_pattern(unsigned long long mag, int fe_base, unsigned sign) {
  const int n = clz64(mag);
  const unsigned long long N = mag << n;
  const unsigned top = (unsigned)(N >> 32);
  const unsigned sticky = ((top & 0xFFu) | (unsigned)N) != 0u ? 1u : 0u;
  return sign | ((unsigned)(fe_base - n) << 23) | ((top >> 8) & 0x7FFFFFu) | sticky;
}

CLR_SPLIT_FN unsigned min_u32(unsigned a, unsigned b) { return a < b ? a : b; }

// FP32 pattern of a value in the fast range of split_bf16 (high word h, low word l of its bits)
// rounded to odd at 24 bits.  (h - (896 << 20)) << 3 rebiases the exponent from 1023 to 127 and
// drops the sign bit (the magnitude's exponent fits in 8 bits in the fast range).
CLR_SPLIT_FN unsigned ro24_of_double(unsigned h, unsigned l) {
  return (h & 0x80000000u) | ((h - (896u << 20)) << 3) | (l >> 29) |
         min_u32(l & 0x1FFFFFFFu, 1u);
}

// Two consecutive values at once: out[t] = bf16 term t of x1 (upper half) and of x0 (lower
// half), identical to split_bf16 of each.  Every term is formed as an FP32 pattern rounded to
// odd at 24 bits (exact integer operations) and the final rounding of both values to bf16 is
// one paired conversion.  Values outside the fast range of split_bf16, or whose a_1 residual
// is below 2^32 units of their last bit, take split_bf16.
template <int TERMS>
CLR_SPLIT_FN void split_bf16_pair(double x0, double x1, unsigned (&out)[TERMS]) {
  const unsigned long long u0 = bits_of(x0), u1 = bits_of(x1);
  const unsigned h[2] = {(unsigned)(u0 >> 32), (unsigned)(u1 >> 32)};
  const unsigned l[2] = {(unsigned)u0, (unsigned)u1};
  const unsigned E[2] = {(h[0] >> 20) & 0x7FFu, (h[1] >> 20) & 0x7FFu};
  if (E[0] - (1023u - 74u) <= 200u && E[1] - (1023u - 74u) <= 200u) {
    out[0] = cvt_bf16x2(ro24_of_double(h[1], l[1]), ro24_of_double(h[0], l[0]));
    if (TERMS == 1) return;
    // residuals in units of the last bit (as in split_bf16), from a_0's bits: the high word
    // of a_0 as an FP64 magnitude is (bf16 magnitude << 13) + (896 << 20)
    unsigned mh[2], ml[2], sg[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const unsigned b = e ? out[0] >> 16 : out[0];
      const int Rh = (int)((h[e] & 0x7FFFFFFFu) - ((b & 0x7FFFu) * 8192u + (896u << 20)));
      ml[e] = Rh < 0 ? 0u - l[e] : l[e];
      mh[e] = Rh < 0 ? (unsigned)(-Rh) - min_u32(l[e], 1u) : (unsigned)Rh;
      sg[e] = (h[e] ^ (unsigned)Rh) & 0x80000000u;  // sign of a_1: x's, flipped when Rh < 0
    }
    if (mh[0] != 0u && mh[1] != 0u) {
      unsigned f1[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        // normalise (leading bit to bit 31 of the top word), keep 24 bits and a sticky bit;
        // after >> 8 the leading bit lands on the exponent field's lowest bit, so the field
        // is written one less
        const int c = clz32(mh[e]);
        const unsigned t = funnel_left(ml[e], mh[e], c);
        const unsigned st = min_u32((t & 0xFFu) | (ml[e] << c), 1u);
        f1[e] = (sg[e] | st) | ((E[e] - 886u - (unsigned)c) * 8388608u + (t >> 8));
      }
      out[1] = cvt_bf16x2(f1[1], f1[0]);
      if (TERMS == 3) {
        // a_2: the residual after a_1 (whose magnitude has its leading bit at 2^32 or above)
        unsigned f2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const unsigned b = e ? out[1] >> 16 : out[1] & 0xFFFFu;
          const unsigned long long mag = ((unsigned long long)mh[e] << 32) | ml[e];
          const int s = (int)E[e] - 1075;
          const int p = (int)((b >> 7) & 0xFFu) - 127 - s;
          const unsigned long long mr = (unsigned long long)((b & 0x7Fu) | 0x80u) << (p - 7);
          const long long d = (long long)(mag - mr);
          f2[e] = d == 0 ? 0u
                         : ro24_pattern(d < 0 ? (unsigned long long)(-d) : (unsigned long long)d,
                                        190 + s, d < 0 ? sg[e] ^ 0x80000000u : sg[e]);
        }
        out[TERMS - 1] = cvt_bf16x2(f2[1], f2[0]);
      }
      return;
    }
  }
  unsigned short a[TERMS], b[TERMS];
  split_bf16<TERMS>(x0, a);
  split_bf16<TERMS>(x1, b);
#pragma unroll
  for (int t = 0; t < TERMS; ++t) out[t] = ((unsigned)b[t] << 16) | a[t];
}

}  // namespace split
}  // namespace clr
