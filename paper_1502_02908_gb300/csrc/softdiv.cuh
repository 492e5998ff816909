// IEEE-754 binary64 division x / y (round to nearest, ties to even) for positive
// normal operands, on the integer pipe.  On GB300 the FP64 divide takes 562
// cycles and ~7 FP64 issue slots; this takes ~45 integer instructions.
//
// Method (Moller & Granlund, "Improved division by invariant integers", IEEE
// Trans. Computers 60(2), 2011): the divisor's significand is normalised to a
// 64-bit d >= 2^63; its reciprocal v = floor((2^128 - 1) / d) - 2^64 comes from
// an 8-bit table and Newton steps (their Alg. 2); the 128-by-64 quotient of the
// dividend's significand is their 2-by-1 division with that reciprocal (Alg. 4),
// which also yields the exact remainder, so the rounding bit and sticky bit are
// exact.  Subnormal, zero, infinite or NaN operands, and quotients outside the
// normal range, take the hardware divide (never the case for the simulation's
// positive rates and times).  Results are bit-identical to IEEE division.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define EPI_HD __host__ __device__ __forceinline__
#else
#define EPI_HD inline
#endif

namespace episim {

EPI_HD uint64_t mulhi_u64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

EPI_HD double bits_as_f64(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

EPI_HD uint64_t f64_as_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}

EPI_HD double hw_div(double x, double y) {
#if defined(__CUDA_ARCH__)
  return __ddiv_rn(x, y);
#else
  return x / y;
#endif
}

// v0 of the reciprocal: floor((2^19 - 3 * 2^8) / d9) for d9 = 256..511.  On
// the device a table built at compile time from the same formula replaces the
// integer divide.
struct RecipSeedTable {
  uint16_t v[256];
};
constexpr RecipSeedTable make_recip_seed_table() {
  RecipSeedTable t{};
  for (int i = 0; i < 256; ++i) t.v[i] = (uint16_t)(((1u << 19) - 3u * (1u << 8)) / (256u + (unsigned)i));
  return t;
}
#if defined(__CUDACC__)
__device__ constexpr RecipSeedTable kRecipSeed = make_recip_seed_table();
#endif

EPI_HD uint64_t recip_seed(uint64_t d9) {
#if defined(__CUDA_ARCH__)
  return kRecipSeed.v[d9 - 256u];
#else
  return (uint64_t)((1u << 19) - 3u * (1u << 8)) / d9;
#endif
}

// v = floor((2^128 - 1) / d) - 2^64 for 2^63 <= d < 2^64.
EPI_HD uint64_t recip_u64(uint64_t d) {
  const uint64_t d0 = d & 1u;
  const uint64_t d9 = d >> 55;
  const uint64_t d40 = (d >> 24) + 1u;
  const uint64_t d63 = (d >> 1) + d0;
  const uint64_t v0 = recip_seed(d9);
  const uint64_t v1 = (v0 << 11) - ((v0 * v0 * d40) >> 40) - 1u;
  const uint64_t v2 = (v1 << 13) + ((v1 * ((1ull << 60) - v1 * d40)) >> 47);
  const uint64_t e = ((v2 >> 1) & (0u - d0)) - v2 * d63;      // 2^96 - v2 d63 + (v2/2) d0, mod 2^64
  const uint64_t v3 = (v2 << 31) + (mulhi_u64(v2, e) >> 1);
  // v4 = v3 - floor((v3 + 2^64 + 1) d / 2^64), mod 2^64
  const uint64_t lo = v3 * d;
  const uint64_t hi = mulhi_u64(v3, d);
  const uint64_t lo2 = lo + d;
  const uint64_t hi2 = hi + d + (lo2 < lo ? 1u : 0u);
  return v3 - hi2;
}

// Quotient and remainder of (u1 * 2^64 + u0) / d with u1 < d, d >= 2^63,
// v = recip_u64(d).
EPI_HD uint64_t div_2by1(uint64_t u1, uint64_t u0, uint64_t d, uint64_t v, uint64_t* rem) {
  uint64_t q0 = v * u1;
  uint64_t q1 = mulhi_u64(v, u1);
  const uint64_t s0 = q0 + u0;
  q1 += u1 + 1u + (s0 < q0 ? 1u : 0u);
  q0 = s0;
  uint64_t r = u0 - q1 * d;
  if (r > q0) { q1 -= 1u; r += d; }
  if (r >= d) { q1 += 1u; r -= d; }
  *rem = r;
  return q1;
}

// x / y, rounded to nearest even, for x, y > 0.
EPI_HD double div_pos(double x, double y) {
  const uint64_t bx = f64_as_bits(x), by = f64_as_bits(y);
  const int ex = (int)(bx >> 52), ey = (int)(by >> 52);
  if (ex == 0 || ey == 0 || ex >= 2047 || ey >= 2047) return hw_div(x, y);
  const uint64_t M = (1ull << 52) - 1u;
  uint64_t mx = (bx & M) | (1ull << 52);
  const uint64_t my = (by & M) | (1ull << 52);
  int e = ex - ey + 1023;
  if (mx < my) { mx <<= 1; e -= 1; }              // mx / my in [1, 2)
  if (e <= 0 || e >= 2047) return hw_div(x, y);   // subnormal or overflowing quotient
  // Q = floor(mx 2^53 / my) = floor(mx 2^64 / (my 2^11)), in [2^53, 2^54)
  const uint64_t d = my << 11;
  uint64_t rem;
  const uint64_t Q = div_2by1(mx, 0u, d, recip_u64(d), &rem);
  uint64_t mant = Q >> 1;                          // 53 bits
  const uint64_t guard = Q & 1u;
  if (guard && (rem != 0u || (mant & 1u))) mant += 1u;
  if (mant >> 53) { mant >>= 1; e += 1; if (e >= 2047) return hw_div(x, y); }
  return bits_as_f64(((uint64_t)e << 52) | (mant & M));
}

}  // namespace episim
