// Device arithmetic of the simulation: Philox4x32-10 draws, exact uniforms,
// the fixed-point -log(u) of Eq. (sampling), and integer-pipe replacements for
// the IEEE conversions and comparisons the specification needs.
//
// On GB300 an FP64 instruction occupies its SM sub-partition's FP64 unit for 64
// cycles whatever the number of active lanes, so everything here that can be
// exact on the integer pipe is: conversions of integers to binary64 are built
// from bit fields, comparisons of non-negative finite doubles compare their bit
// patterns as integers, and the logarithm is 64-bit fixed point.
#pragma once
#include <cstdint>
#include "neglog_table.h"

namespace episim {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): per round two 32x32->64 products of
// words 0 and 2 by fixed odd multipliers; high halves are xored with the other
// words and the round key; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi_a = __umulhi(m0, c.x), lo_a = m0 * c.x;
    uint32_t hi_b = __umulhi(m1, c.z), lo_b = m1 * c.z;
    c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

constexpr uint32_t kEventTag = 0x40000000u;  // counter word 1 = day | tag for event draws

// ------------------------------------------------------- binary64 from bits
__device__ __forceinline__ double bits_to_double(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint64_t double_bits(double x) { return (uint64_t)__double_as_longlong(x); }

// Exact binary64 of a non-negative int32 (the I2F instruction runs on the FP64 pipe).
__device__ __forceinline__ double i2d_exact(int32_t n) {
  if (n <= 0) return 0.0;  // counts are never negative
  uint32_t u = (uint32_t)n;
  int top = 31 - __clz(u);                       // position of the leading one
  uint64_t mant = ((uint64_t)u << (52 - top)) & ((1ull << 52) - 1);
  return bits_to_double(((uint64_t)(1023 + top) << 52) | mant);
}

// u = (2j+1) 2^-53 for j = top 52 bits of a 64-bit word: exact, in (0, 1).
__device__ __forceinline__ double uniform_open(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  uint64_t x = ((w >> 12) << 1) | 1ull;          // odd, < 2^53
  int top = 63 - __clzll(x);
  uint64_t mant = (x << (52 - top)) & ((1ull << 52) - 1);
  return bits_to_double(((uint64_t)(1023 - 53 + top) << 52) | mant);
}

// Round-to-nearest-even binary64 of q * 2^-58 for 1 <= q < 2^64.
__device__ __forceinline__ double q58_to_double(uint64_t q) {
  int lz = __clzll(q);
  uint64_t m = q << lz;                          // leading one at bit 63
  uint64_t mant = m >> 11;
  uint64_t rest = m & 0x7FFull;
  mant += (rest > 0x400ull) | ((rest == 0x400ull) & (mant & 1ull));
  int e = (63 - lz) - 58 + 1023;
  if (mant >> 53) { mant >>= 1; ++e; }
  return bits_to_double(((uint64_t)e << 52) | (mant & ((1ull << 52) - 1)));
}

// floor(a * b / 2^62) for signed Q62 operands whose product fits.
__device__ __forceinline__ int64_t mul_q62(int64_t a, int64_t b) {
  int64_t hi = __mul64hi(a, b);
  uint64_t lo = (uint64_t)a * (uint64_t)b;
  return (int64_t)(((uint64_t)hi << 2) | (lo >> 62));
}

__device__ const int32_t kRecip[128] = {EPISIM_RECIP_TABLE};
__device__ const int64_t kLogR[128] = {EPISIM_LOGR_TABLE};

__host__ __device__ constexpr int64_t q62_over(int k) { return (int64_t)(((1ull << 62) + (uint64_t)(k / 2)) / (uint64_t)k); }

// E = -ln(u), u = (2j+1) 2^-53.  With x = 2j+1 = 2^n m, m in [1,2):
// E = (53 - n) ln2 - ln m, where ln m = ln(m R_i / 1024) + ln(1024 / R_i) for the
// table entry i of m's top seven fraction bits; ln(1 + z) for |z| < 2^-7.8 is
// Horner through z^7 in Q62.  The sum is formed in 128 bits, floored to Q58
// (at least one unit) and rounded once to binary64.
__device__ __forceinline__ double neglog_u(uint64_t j) {
  uint64_t x = (j << 1) | 1ull;
  int n = 63 - __clzll(x);
  uint64_t M = x << (52 - n);
  int i = (int)((M >> 45) & 127);
  int64_t R = __ldg(&kRecip[i]);
  int64_t z = (int64_t)(M * (uint64_t)R) - (int64_t)(1ull << 62);
  int64_t h = q62_over(7);
  h = q62_over(6) - mul_q62(z, h);
  h = q62_over(5) - mul_q62(z, h);
  h = q62_over(4) - mul_q62(z, h);
  h = q62_over(3) - mul_q62(z, h);
  h = q62_over(2) - mul_q62(z, h);
  h = q62_over(1) - mul_q62(z, h);
  int64_t lnm = mul_q62(z, h) + __ldg(&kLogR[i]);
  // (53 - n) * ln2 in 128 bits minus sign-extended lnm
  uint64_t k = (uint64_t)(53 - n);
  uint64_t p_lo = k * EPISIM_LN2_Q62;
  uint64_t p_hi = __umul64hi(k, EPISIM_LN2_Q62);
  uint64_t s_lo = p_lo - (uint64_t)lnm;
  uint64_t borrow = (p_lo < (uint64_t)lnm) ? 1ull : 0ull;
  uint64_t s_hi = p_hi - (lnm < 0 ? ~0ull : 0ull) - borrow;
  // floor(E62 / 16) clamped to >= 1
  uint64_t q = (s_hi << 60) | (s_lo >> 4);
  if ((int64_t)s_hi < 0 || (s_hi == 0 && (s_lo >> 4) == 0)) q = 1;
  return q58_to_double(q);
}

// a <= b for non-negative finite binary64 values (bit patterns order them).
__device__ __forceinline__ bool le_nonneg(double a, double b) { return double_bits(a) <= double_bits(b); }
__device__ __forceinline__ bool pos(double a) { return double_bits(a) != 0ull && !(double_bits(a) >> 63); }

// Uniform integer in [0, s), s >= 1 (Lemire 2019): multiply-shift with rejection.
// next() yields successive 32-bit words of the event's Philox stream.
template <class Next>
__device__ __forceinline__ uint32_t lemire(uint32_t s, Next&& next) {
  uint64_t m = (uint64_t)next() * s;
  uint32_t l = (uint32_t)m;
  if (l < s) {
    uint32_t t = (0u - s) % s;
    while (l < t) { m = (uint64_t)next() * s; l = (uint32_t)m; }
  }
  return (uint32_t)(m >> 32);
}

// Programmatic dependent launch (sm_90 and later): a kernel lets the next one in
// its stream be scheduled early, and that one waits for the previous grid's
// completion (and memory) only where it reads what the previous grid wrote.
// Both are no-ops for kernels launched without the programmatic attribute.
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int season_of(int day) {
  int dm = day % 365;
  return dm <= 91 ? 0 : dm <= 182 ? 1 : dm <= 273 ? 2 : 3;
}

}  // namespace episim
