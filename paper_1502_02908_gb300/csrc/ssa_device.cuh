// Device code of the stochastic step (Eq. (numstep3); Sec. 3.3 Eqs. (sampling),
// (sampling2); the per-node loop of Alg. 1) with the fused phi update (Eq. (numstep5)):
// shared by the per-day kernels (ssa.cu) and the persistent batch kernel
// (batch.cu).  State other blocks may have written in the same launch is read
// with L2-coherent loads.
#pragma once
#include "internal.h"
#include "devmath.cuh"
#include "softdiv.cuh"

namespace episim {

template <int NA>
struct NodeState {
  int32_t x[2 * NA];
};

template <int NA>
__device__ __forceinline__ void load_counts(const SsaArgs& a, int r, int v, NodeState<NA>& s) {
  const int32_t* base = a.counts + (size_t)r * a.Nc * a.N + v;
#pragma unroll
  for (int c = 0; c < 2 * NA; ++c) s.x[c] = __ldcg(base + (size_t)c * a.N);
}

template <int NA>
__device__ __forceinline__ void store_counts(const SsaArgs& a, int r, int v, const NodeState<NA>& s) {
  int32_t* base = a.counts + (size_t)r * a.Nc * a.N + v;
#pragma unroll
  for (int c = 0; c < 2 * NA; ++c) base[(size_t)c * a.N] = s.x[c];
}

// phi_{d+1} = ((phi_d (1 - beta(d))) + (alpha I) / N) + eps; tangents d phi/d beta,
// d phi/d alpha carried alongside in score mode.
template <int NA, bool SCORE>
__device__ __forceinline__ double phi_step(const SsaArgs& a, const DevParams& p, int r, int v, int day,
                                           const NodeState<NA>& s, double phi) {
  int32_t I = 0, tot = 0;
#pragma unroll
  for (int j = 0; j < NA; ++j) { I += s.x[2 * j + 1]; tot += s.x[2 * j] + s.x[2 * j + 1]; }
  double omb = __dadd_rn(1.0, -p.beta[season_of(day)]);
  double q = 0.0;
  double dI = i2d_exact(I), dN = i2d_exact(tot);
  if (tot > 0) { const double aI = __dmul_rn(p.alpha, dI); q = pos(aI) ? div_pos(aI, dN) : 0.0; }
  double next = __dadd_rn(__dadd_rn(__dmul_rn(phi, omb), q), p.eps);
  if (SCORE && a.traj) {
    const double ion = (tot > 0 && I > 0) ? div_pos(dI, dN) : 0.0;
    a.traj[((size_t)2 * a.max_days + day) * a.R * a.N + (size_t)r * a.N + v] = ion;
  } else if (SCORE) {
    double* tb = a.tang + ((size_t)r * 2 + 0) * a.N + v;
    double* ta = a.tang + ((size_t)r * 2 + 1) * a.N + v;
    double ion = (tot > 0 && I > 0) ? div_pos(dI, dN) : 0.0;
    *tb = __dsub_rn(__dmul_rn(__ldcg(tb), omb), phi);
    *ta = __dadd_rn(__dmul_rn(__ldcg(ta), omb), ion);
  }
  return next;
}

// Sum over the warp's lanes; the total lands in lane 0.
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

struct DayTerms {
  double n_inf, n_rec, int_s, int_i, tlast;
};

// The direct method for one node-day; returns the number of transitions fired.
template <int NA, bool SCORE>
__device__ __forceinline__ uint32_t ssa_node_day(const DevParams& p, uint64_t seed, uint32_t rep, int v, int day,
                                                 double phi, NodeState<NA>& s, DayTerms (&T)[NA]) {
  double cinf[NA], ainf[NA], arec[NA], A[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    cinf[j] = __dmul_rn(p.ups[j], phi);
    ainf[j] = __dmul_rn(cinf[j], i2d_exact(s.x[2 * j]));
    arec[j] = __dmul_rn(p.gam[j], i2d_exact(s.x[2 * j + 1]));
    A[j] = __dadd_rn(ainf[j], arec[j]);
    if (SCORE) { T[j].n_inf = T[j].n_rec = T[j].int_s = T[j].int_i = 0.0; T[j].tlast = 0.0; }
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  double t = 0.0;
  uint32_t fired = 0;
  for (uint32_t k = 0;; ++k) {
    double P[NA];
    P[0] = A[0];
#pragma unroll
    for (int j = 1; j < NA; ++j) P[j] = __dadd_rn(P[j - 1], A[j]);
    const double a0 = P[NA - 1];
    if (!pos(a0)) break;
    uint4 w = philox10(make_uint4((uint32_t)v, (uint32_t)day, k, rep), k0, k1);
    double E = neglog_u(((((uint64_t)w.y) << 32) | w.x) >> 12);
    double u2 = uniform_open(w.z, w.w);
    double tn = __dadd_rn(t, div_pos(E, a0));
    if (le_nonneg(1.0, tn)) break;
    t = tn;
    double rr = __dmul_rn(a0, u2);
    // class: first with A_j > 0 and r <= P_j, else the last positive one
    int cls = -1, last = -1;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      if (cls < 0 && pos(A[j])) {
        last = j;
        if (le_nonneg(rr, P[j])) cls = j;
      }
    }
    if (cls < 0) cls = last;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      if (j != cls) continue;
      double thr = (j == 0) ? ainf[0] : __dadd_rn(P[j > 0 ? j - 1 : 0], ainf[j]);
      bool infect = pos(ainf[j]) && (le_nonneg(rr, thr) || !pos(arec[j]));
      if (SCORE) {
        double dt = __dsub_rn(t, T[j].tlast);
        T[j].int_s = __dadd_rn(T[j].int_s, __dmul_rn(i2d_exact(s.x[2 * j]), dt));
        T[j].int_i = __dadd_rn(T[j].int_i, __dmul_rn(i2d_exact(s.x[2 * j + 1]), dt));
        T[j].tlast = t;
        if (infect) T[j].n_inf = __dadd_rn(T[j].n_inf, 1.0); else T[j].n_rec = __dadd_rn(T[j].n_rec, 1.0);
      }
      if (infect) { s.x[2 * j] -= 1; s.x[2 * j + 1] += 1; }
      else        { s.x[2 * j + 1] -= 1; s.x[2 * j] += 1; }
      ainf[j] = __dmul_rn(cinf[j], i2d_exact(s.x[2 * j]));
      arec[j] = __dmul_rn(p.gam[j], i2d_exact(s.x[2 * j + 1]));
      A[j] = __dadd_rn(ainf[j], arec[j]);
    }
    ++fired;
  }
  if (SCORE) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      double dt = __dsub_rn(1.0, T[j].tlast);
      T[j].int_s = __dadd_rn(T[j].int_s, __dmul_rn(i2d_exact(s.x[2 * j]), dt));
      T[j].int_i = __dadd_rn(T[j].int_i, __dmul_rn(i2d_exact(s.x[2 * j + 1]), dt));
    }
  }
  return fired;
}

// ---------------------------------------------------------------------------
// binary32 helpers of the speculative methods below.

__device__ __forceinline__ float trunc_to_f32(double x) {
  // positive normal double within float range -> float with the top 23 fraction bits
  const uint64_t b = double_bits(x);
  const int e = (int)(b >> 52) - 1023 + 127;
  if (b == 0ull) return 0.0f;
  return __int_as_float((int)(((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7FFFFFull)));
}

__device__ __forceinline__ float small_int_to_f32(int32_t n) {  // exact for 0 <= n < 2^23
  return __fsub_rn(__int_as_float(0x4B000000 | n), 8388608.0f);
}

// -1: a < b decisively, +1: a > b decisively, 0: too close to call in FP32.
__device__ __forceinline__ int cmp_f32(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  if (ia < 0x00800000 || ib < 0x00800000) return 0;  // zero or subnormal: exact path
  const int d = ia - ib;
  return d <= -64 ? -1 : (d >= 64 ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Speculative binary32 clock.  The specification's clock is the binary64 chain
// t_{k+1} = fl(t_k + fl(E_k / a0_k)) and a day ends at the first k with
// t_{k+1} >= 1.  Here tau~_k = E~_k / a0~_k in binary32 (E~ the binary32 -log of
// the draw below, a0~ the binary32 propensity sum) is accumulated exactly in Q62
// fixed point.  With u = 2^-24: a0~ is within 6u of a0 (constants truncated to
// binary32: 2u, product u, three sums u each), E~ within 16u of E, and the
// division (__fdividef, 2 ulps) adds 4u, so tau~_k is within rho = 26u < 2^-19.2
// of tau_k.  At a decision the Q62 sum is below 2.5, hence within 2.5 rho
// (< 2^-17.9) plus k (2^-53 + 2^-62) of the binary64 chain for k < 2^24: a margin of 2^-17 makes
// "sum >= 1 + margin" a certain stop and "sum + margin < 1" a certain continue;
// anything between is handed to the exact binary64 method.  The stochastic
// choices are taken in binary32 only when decisive (below) and in binary64
// otherwise, so the result is the specification's, bit for bit.
constexpr uint64_t kQ62One = 1ull << 62;
constexpr uint64_t kClockMargin = kQ62One >> 17;   // largest allowed margin exponent: 17
constexpr uint32_t kSpecMaxSteps = 1u << 24;

// binary32 of m 2^-53 for 1 <= m < 2^53, rounded to nearest (ties away): within u.
__device__ __forceinline__ float f32_of_q53(uint64_t m) {
  const int lz = __clzll(m);
  const uint32_t top = ((uint32_t)((m << lz) >> 39) + 1u) >> 1;   // 24 bits, or 2^24 on carry
  const uint32_t e = (uint32_t)(137 - lz) + (top >> 24);
  return __uint_as_float((e << 23) | (top & 0x7FFFFFu));
}

// binary32 -log(u) for u = (2j+1) 2^-53, within 16u of -log(u).  Below 1/sqrt2,
// u = f 2^e with f in [1/sqrt2, sqrt2) and log u = e ln2 + 2 atanh((f-1)/(f+1));
// from 1/sqrt2 on, log u = log(1 - v) = 2 atanh(-v/(2-v)) with v = 1 - u taken
// exactly from the integers.  Either way |s| <= 0.1716 and atanh(s)/s is the
// series 1 + s^2/3 + s^4/5 + s^6/7 + s^8/9 (remainder below 2^-28).  Error
// budget: the argument's rounding (u, amplified at most 2x near the split),
// f + 1 or 2 - v (u), the quotient (__fdividef: 2 ulps), the series (2u), the
// product and the final sum (u each, the sum's cancellation amplifying the e ln2
// part at most 2x): below 14u.
__device__ __forceinline__ float neglog_f32(uint64_t j) {
  constexpr uint64_t kSplit = 3184525836262886ull;   // first j with (2j+1) 2^-53 >= 1/sqrt2
  const bool hi = j >= kSplit;
  const float x = f32_of_q53(hi ? ((((1ull << 52) - j) << 1) - 1ull) : ((j << 1) | 1ull));
  // low side: f = mantissa of x in [1/sqrt2, sqrt2), e = its exponent
  const uint32_t b = __float_as_uint(x);
  float f = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  int e = (int)(b >> 23) - 127;
  if (f >= 1.41421356f) { f = __fmul_rn(f, 0.5f); e += 1; }
  const float num = hi ? -x : __fsub_rn(f, 1.0f);
  const float den = hi ? __fsub_rn(2.0f, x) : __fadd_rn(f, 1.0f);
  const float sc = hi ? 0.0f : (float)e;
  const float sq = __fdividef(num, den);
  const float z = __fmul_rn(sq, sq);
  float poly = __fadd_rn(0.142857149f, __fmul_rn(z, 0.111111112f));
  poly = __fadd_rn(0.200000003f, __fmul_rn(z, poly));
  poly = __fadd_rn(0.333333343f, __fmul_rn(z, poly));
  poly = __fadd_rn(1.0f, __fmul_rn(z, poly));
  const float lg = __fadd_rn(__fmul_rn(__fmul_rn(2.0f, sq), poly), __fmul_rn(sc, 0.693147182f));
  return -lg;
}

// floor(f 2^62) for 0 <= f <= 1.5 (f normal or subnormal).
__device__ __forceinline__ uint64_t q62_of(float f) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)(b >> 23);
  const uint64_t m = e ? (uint64_t)((b & 0x7FFFFFu) | 0x800000u) : (uint64_t)(b & 0x7FFFFFu);
  const int sh = (e ? e : 1) - 127 - 23 + 62;
  return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
}

// binary32 copies of a node-day's rate constants; false when the binary32 bounds
// above do not hold (a constant outside [2^-100, 2^60] or a herd of 2^22 or more).
template <int NA>
__device__ __forceinline__ bool spec_constants(const DevParams& p, const double (&cinf)[NA], const int32_t (&x)[2 * NA],
                                               float (&cinff)[NA], float (&gamf)[NA]) {
  bool ok = true;
  int32_t herd = 0;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    for (int q = 0; q < 2; ++q) {
      const double c = q ? p.gam[j] : cinf[j];
      const int e = (int)(double_bits(c) >> 52) - 1023;
      if (pos(c) && (e < -100 || e > 60)) ok = false;
    }
    cinff[j] = trunc_to_f32(cinf[j]);
    gamf[j] = trunc_to_f32(p.gam[j]);
    herd += x[2 * j] + x[2 * j + 1];
  }
  return ok && herd < (1 << 22);
}

// State of a lane in the fixed-point iteration: the block's start x plus the
// transitions the lanes before it (within its group of SEG lanes) currently
// guess, counted with one ballot per transition kind (ch = 2*class + recovery;
// negative = none).
template <int NA, int SEG>
__device__ __forceinline__ void prefix_state(const int32_t (&x)[2 * NA], int ch, int lane, int32_t (&xs)[2 * NA]) {
  const uint32_t full = 0xffffffffu;
  const uint32_t below = ((1u << lane) - 1u) & (SEG == 32 ? full : ~((1u << (lane & ~(SEG - 1))) - 1u));
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    const int inf = __popc(__ballot_sync(full, ch == 2 * j) & below);
    const int rec = __popc(__ballot_sync(full, ch == 2 * j + 1) & below);
    xs[2 * j] = x[2 * j] - inf + rec;
    xs[2 * j + 1] = x[2 * j + 1] + inf - rec;
  }
}

// binary32 selection thresholds of state x, in the specification's order and
// rounding: a_inf,1, P_1, P_1 + a_inf,2, P_2, ...; a0~ = P_NA.  Returns whether
// any rate is positive (exact, from the counts and constants).
template <int NA>
__device__ __forceinline__ bool thresholds_f32(const bool (&cpos)[NA], const bool (&gpos)[NA],
                                               const float (&cinff)[NA], const float (&gamf)[NA],
                                               const int32_t (&x)[2 * NA], float (&T)[2 * NA - 1], float& a0f) {
  bool any = false;
  float P = 0.0f;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    any = any || (cpos[j] && x[2 * j] > 0) || (gpos[j] && x[2 * j + 1] > 0);
    const float aif = __fmul_rn(cinff[j], small_int_to_f32(x[2 * j]));
    const float A = __fadd_rn(aif, __fmul_rn(gamf[j], small_int_to_f32(x[2 * j + 1])));
    if (j == 0) { T[0] = aif; P = A; }
    else { T[2 * j] = __fadd_rn(P, aif); P = __fadd_rn(P, A); }
    if (2 * j + 1 < 2 * NA - 1) T[(2 * j + 1 < 2 * NA - 1) ? 2 * j + 1 : 0] = P;
  }
  a0f = P;
  return any;
}

// The transition the draw r = a0 u2 fires, from binary32 values: r falls in the
// k-th of the intervals cut by the thresholds (zero-width intervals, from zero
// rates, are never chosen), so k = 2*class + (1 if recovery) is the number of
// thresholds below r.  Decided only when every comparison is decisive (exactly
// zero thresholds always are); otherwise -1.
template <int NA>
__device__ __forceinline__ int choice_count_f32(const float (&T)[2 * NA - 1], float rf) {
  const int ir = __float_as_int(rf);
  bool amb = ir < 0x00800000;                      // r~ zero or subnormal: exact path
  int c = 0;
#pragma unroll
  for (int i = 0; i < 2 * NA - 1; ++i) {
    const int d = ir - __float_as_int(T[i]);       // thresholds are 0 or normal
    const bool zero = T[i] == 0.0f;
    amb = amb || (!zero && d > -64 && d < 64);
    c += (zero || d > 0) ? 1 : 0;
  }
  return amb ? -1 : c;
}

// Exact decision of the specification for the state x and uniform u2: returns
// 2*class + (1 if recovery else 0).
template <int NA>
__device__ __forceinline__ int exact_choice(const double (&cinf)[NA], const DevParams& p, const int32_t (&x)[2 * NA],
                                            double u2) {
  double ainf[NA], arec[NA], A[NA], P[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    ainf[j] = __dmul_rn(cinf[j], i2d_exact(x[2 * j]));
    arec[j] = __dmul_rn(p.gam[j], i2d_exact(x[2 * j + 1]));
    A[j] = __dadd_rn(ainf[j], arec[j]);
    P[j] = (j == 0) ? A[0] : __dadd_rn(P[j > 0 ? j - 1 : 0], A[j]);
  }
  const double rr = __dmul_rn(P[NA - 1], u2);
  int cls = -1, last = -1;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    if (cls < 0 && pos(A[j])) {
      last = j;
      if (le_nonneg(rr, P[j])) cls = j;
    }
  }
  if (cls < 0) cls = last;
  int out = 0;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    if (j != cls) continue;
    const double thr = (j == 0) ? ainf[0] : __dadd_rn(P[j > 0 ? j - 1 : 0], ainf[j]);
    const bool infect = pos(ainf[j]) && (le_nonneg(rr, thr) || !pos(arec[j]));
    out = 2 * j + (infect ? 0 : 1);
  }
  return out;
}

// The direct method for one node-day with the speculative clock (one thread):
// transitions fired, or -1 when a clock decision was too close to call (the
// caller then reruns the node-day with ssa_node_day from the same state).  One
// exit test per step; the draw of step k + 1 is computed during step k (it does
// not depend on the state), so its latency overlaps the state-dependent chain.
template <int NA>
__device__ __forceinline__ int32_t ssa_node_day_spec(const DevParams& p, uint64_t seed, uint32_t rep, int v, int day,
                                                     const double (&cinf)[NA], const float (&cinff)[NA],
                                                     const float (&gamf)[NA], uint64_t margin, NodeState<NA>& s) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  bool cpos[NA], gpos[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) { cpos[j] = pos(cinf[j]); gpos[j] = pos(p.gam[j]); }
  uint64_t tq = 0;
  uint4 wn = philox10(make_uint4((uint32_t)v, (uint32_t)day, 0u, rep), k0, k1);
  for (uint32_t k = 0;; ++k) {
    float T[2 * NA - 1], a0f;
    const bool any = thresholds_f32<NA>(cpos, gpos, cinff, gamf, s.x, T, a0f);
    const uint4 w = wn;
    wn = philox10(make_uint4((uint32_t)v, (uint32_t)day, k + 1u, rep), k0, k1);
    const float Ef = neglog_f32(((((uint64_t)w.y) << 32) | w.x) >> 12);
    const float u2f = f32_of_q53(((((((uint64_t)w.w) << 32) | w.z) >> 12) << 1) | 1ull);
    int choice = choice_count_f32<NA>(T, __fmul_rn(a0f, u2f));
    const uint64_t sq = tq + q62_of(fminf(__fdividef(Ef, a0f), 1.5f));
    if (!any || sq >= kQ62One + margin) return (int32_t)k;
    if (sq + margin >= kQ62One || k + 1u >= kSpecMaxSteps) return -1;
    if (choice < 0) choice = exact_choice<NA>(cinf, p, s.x, uniform_open(w.z, w.w));
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      if (2 * j == choice) { s.x[2 * j] -= 1; s.x[2 * j + 1] += 1; }
      if (2 * j + 1 == choice) { s.x[2 * j + 1] -= 1; s.x[2 * j] += 1; }
    }
    tq = sq;
  }
}

// Warp-cooperative direct method for one node-day (large herds), all 32 lanes
// together; phases per block of 32 draws:
//  1. lane l computes draw k0 + l: Philox, E = -log(u1), u2 (independent of the
//     state, so all 32 in parallel);
//  2. the embedded jump chain (which transition each draw fires): binary32
//     comparisons decide only when the operands are at least 64 float ulps apart
//     (relative gap >= 2^-18, beyond the <= 2^-20 error of the binary32 rates,
//     sums and product against the specification's binary64 values); otherwise
//     that draw is decided with the specification's binary64 arithmetic.  With
//     CLOCK > 0 all lanes decide at once by the fixed-point iteration below; with
//     CLOCK = 0 the lanes walk the chain in draw order;
//  3-4. the clock.  CLOCK = 2: lane l forms tau~_l from its draw's binary32
//     propensity sum; an inclusive warp scan of the Q62 values gives the clock
//     after every draw, and the first draw that is not a certain continue ends
//     the day (certain stop) or returns -1 (too close to call).  CLOCK = 1: the
//     same scan of the exact binary64 tau_l (a0 of the lane's state, the exact
//     -log), whose sum is within (k + 2) 2^-53 of the binary64 chain, so only a
//     decision within that of the day's end returns -1.  CLOCK = 0: the binary64
//     clock t + tau_l runs in draw order; the first draw reaching t >= 1 ends the
//     day in the state before that draw.
// Returns the transitions fired, or -1 (CLOCK > 0) for the caller to rerun the
// node-day with a smaller CLOCK from the same state.
// floor(x 2^62) for a non-negative binary64 x <= 1.5 (exact bits).
__device__ __forceinline__ uint64_t q62_of_f64(double x) {
  const uint64_t b = double_bits(x);
  const int e = (int)(b >> 52);
  const uint64_t m = e ? ((b & ((1ull << 52) - 1)) | (1ull << 52)) : (b & ((1ull << 52) - 1));
  const int sh = (e ? e : 1) - 1023 - 52 + 62;
  return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
}

// Rounds of the binary32 clock whose choices a warp logs, so that a day end too
// close to call resumes with the binary64 clock from that round instead of
// rerunning the node-day.
constexpr int kReplayRounds = 128;

// Returns the transitions fired, or -1.  kb0, tq0, fired0: resume at draw kb0
// (a multiple of 32) with the clock tq0 (Q62) and fired0 transitions behind.
template <int NA, int CLOCK>
__device__ __forceinline__ int32_t ssa_warp_node_day(const DevParams& p, uint64_t seed, uint32_t rep, int v, int day,
                                                     double phi, uint64_t margin, NodeState<NA>& s,
                                                     uint32_t kb0 = 0, uint64_t tq0 = 0, int32_t fired0 = 0) {
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  const uint32_t full = 0xffffffffu;
  double cinf[NA];
  float cinff[NA], gamf[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) cinf[j] = __dmul_rn(p.ups[j], phi);
  constexpr bool SPEC = CLOCK == 2;
  const bool spec_ok = spec_constants<NA>(p, cinf, s.x, cinff, gamf);
  if (SPEC && !spec_ok) return -1;
  bool cpos[NA], gpos[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) { cpos[j] = pos(cinf[j]); gpos[j] = pos(p.gam[j]); }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  double t = 0.0;
  uint64_t tq = tq0;
  int32_t fired = fired0;
  // binary32 clock: the day's start state and each continuing round's choice of
  // this lane, for a resume with the binary64 clock
  int32_t xday[NC];
  uint8_t chlog[CLOCK == 2 ? kReplayRounds : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) xday[c] = s.x[c];
  // more than two rounds a day expected at the start state (a0 > 64): the clock
  // once per round (below)
  bool dense = false;
  if (CLOCK == 2) {
    float T0[2 * NA - 1], a00;
    dense = thresholds_f32<NA>(cpos, gpos, cinff, gamf, s.x, T0, a00) && a00 > 64.0f;
  }
  for (uint32_t kb = kb0;; kb += 32) {
    if (CLOCK > 0 && kb >= kSpecMaxSteps) return -1;
    // 1. draws of this block
    const uint4 w = philox10(make_uint4((uint32_t)v, (uint32_t)day, kb + (uint32_t)lane, rep), k0, k1);
    const uint64_t j52 = ((((uint64_t)w.y) << 32) | w.x) >> 12;
    double E = 0.0;
    float Ef = 0.0f;
    if (CLOCK == 2) Ef = neglog_f32(j52);
    else E = neglog_u(j52);
    const double u2 = uniform_open(w.z, w.w);
    const float u2f = f32_of_q53(((((((uint64_t)w.w) << 32) | w.z) >> 12) << 1) | 1ull);
    // 2. embedded chain
    int32_t x[NC], xs[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { x[c] = s.x[c]; xs[c] = x[c]; }
    float a0l = 0.0f;
    int stop_at = 32;
    if (CLOCK == 2) {
      // The fixed-point iteration below with the binary32 clock in every round:
      // the clock after each draw comes from the lanes' current states, and the
      // first draw that is not a certain continue (a0 = 0, a certain stop, or too
      // close to call) is the day's end candidate e.  Once no choice of the draws
      // before e changes, those choices are the chain's, so are the states up to
      // e and the clock through e: the block is decided without waiting for the
      // draws after e, which cannot matter.
      int ch = -3;
      for (int it = 0; it <= 32; ++it) {
        prefix_state<NA, 32>(x, ch, lane, xs);
        float T[2 * NA - 1], a0f;
        int nc = -2;
        const bool valid = thresholds_f32<NA>(cpos, gpos, cinff, gamf, xs, T, a0f);
        if (valid) {
          nc = choice_count_f32<NA>(T, __fmul_rn(a0f, u2f));
          if (nc < 0) nc = exact_choice<NA>(cinf, p, xs, u2);
        }
        // a dense node-day (many rounds) almost never ends inside a round: settle
        // every lane's choice first and take the clock once
        if (dense && it < 32 && __ballot_sync(full, nc != ch)) {
          ch = nc;
          continue;
        }
        uint64_t sc = valid ? q62_of(fminf(__fdividef(Ef, a0f), 1.5f)) : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t y = __shfl_up_sync(full, sc, o);
          if (lane >= o) sc += y;
        }
        const uint64_t sl = tq + sc;
        const unsigned notcont = __ballot_sync(full, !(valid && sl + margin < kQ62One));
        const int e = notcont ? __ffs(notcont) - 1 : 32;
        const unsigned diff = __ballot_sync(full, nc != ch) & (e < 32 ? ((1u << e) - 1u) : full);
        ch = nc;
        if (diff != 0u) {
          if (it == 32) return -1;                  // cannot happen (33 rounds suffice)
          continue;
        }
        if (e < 32) {
          const unsigned ok = __ballot_sync(full, !valid || sl >= kQ62One + margin);
          if (!((ok >> e) & 1u)) {                  // too close to call
            const uint32_t rounds = kb >> 5;
            if (rounds > (uint32_t)kReplayRounds) return -1;
            // the binary64 clock's Q62 sum through the earlier rounds, from their
            // logged choices (every one a continue), then that clock from here on
            uint64_t tqx = 0;
            int32_t xr[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) xr[c] = xday[c];
            for (uint32_t r = 0; r < rounds; ++r) {
              const uint4 wr = philox10(make_uint4((uint32_t)v, (uint32_t)day, (r << 5) + (uint32_t)lane, rep), k0, k1);
              const double Er = neglog_u(((((uint64_t)wr.y) << 32) | wr.x) >> 12);
              const int chr = chlog[r];
              int32_t xsr[NC];
              prefix_state<NA, 32>(xr, chr, lane, xsr);
              double P = 0.0;
#pragma unroll
              for (int j = 0; j < NA; ++j) {
                const double ainf = __dmul_rn(cinf[j], i2d_exact(xsr[2 * j]));
                const double arec = __dmul_rn(p.gam[j], i2d_exact(xsr[2 * j + 1]));
                const double A = __dadd_rn(ainf, arec);
                P = (j == 0) ? A : __dadd_rn(P, A);
              }
              const double taur = div_pos(Er, P);
              tqx += __shfl_sync(full, warp_sum(q62_of_f64(le_nonneg(taur, 1.5) ? taur : 1.5)), 0);
              int32_t aft[NC];
#pragma unroll
              for (int j = 0; j < NA; ++j) {
                const int dj = ((chr >> 1) == j) ? ((chr & 1) ? -1 : 1) : 0;
                aft[2 * j] = xsr[2 * j] - dj;
                aft[2 * j + 1] = xsr[2 * j + 1] + dj;
              }
#pragma unroll
              for (int c = 0; c < NC; ++c) xr[c] = __shfl_sync(full, aft[c], 31);
            }
            return ssa_warp_node_day<NA, 1>(p, seed, rep, v, day, phi, 0, s, kb, tqx, fired);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) s.x[c] = __shfl_sync(full, xs[c], e);
          return fired + e;
        }
        tq = __shfl_sync(full, sl, 31);
        if ((kb >> 5) < (uint32_t)kReplayRounds) chlog[kb >> 5] = (uint8_t)ch;
        break;
      }
      // the whole block continues: the state after lane 31's draw
      int32_t after[NC];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int dj = (ch >= 0 && (ch >> 1) == j) ? ((ch & 1) ? -1 : 1) : 0;
        after[2 * j] = xs[2 * j] - dj;
        after[2 * j + 1] = xs[2 * j + 1] + dj;
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) s.x[c] = __shfl_sync(full, after[c], 31);
      fired += 32;
      continue;
    }
    if (CLOCK == 1) {
      // Fixed-point iteration over the lanes: every lane takes as its state the
      // block's start plus the transitions currently guessed for the lanes before
      // it and decides its own draw there.  A lane whose predecessors' guesses are
      // right decides right, so each round confirms at least one more leading lane
      // and the iteration stops, after at most 33 rounds, with every guess equal to
      // the sequential chain's choice.  The lanes' states come from ballots of the
      // guesses (prefix_state).
      int ch = -3;                                 // -3: no guess yet, -2: a0 = 0 here
      for (int it = 0; it <= 32; ++it) {
        prefix_state<NA, 32>(x, ch, lane, xs);
        float T[2 * NA - 1], a0f;
        int nc = -2;
        if (thresholds_f32<NA>(cpos, gpos, cinff, gamf, xs, T, a0f)) {
          a0l = a0f;
          nc = spec_ok ? choice_count_f32<NA>(T, __fmul_rn(a0f, u2f)) : -1;
          if (nc < 0) nc = exact_choice<NA>(cinf, p, xs, u2);
        }
        const unsigned diff = __ballot_sync(full, nc != ch);
        ch = nc;
        if (diff == 0u) break;
      }
      const unsigned stops = __ballot_sync(full, ch == -2);
      stop_at = stops ? __ffs(stops) - 1 : 32;
      // state after the block: the stopping lane's, or the last lane's after its draw
      const int src = stop_at < 32 ? stop_at : 31;
      int32_t after[NC];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int dj = (ch >= 0 && (ch >> 1) == j) ? ((ch & 1) ? -1 : 1) : 0;
        after[2 * j] = xs[2 * j] - (stop_at < 32 ? 0 : dj);
        after[2 * j + 1] = xs[2 * j + 1] + (stop_at < 32 ? 0 : dj);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = __shfl_sync(full, after[c], src);
    }
    for (int l = 0; l < (CLOCK > 0 ? 0 : 32); ++l) {
      if (l == lane) {
#pragma unroll
        for (int c = 0; c < NC; ++c) xs[c] = x[c];
      }
      float T[2 * NA - 1], a0f;
      const bool any = thresholds_f32<NA>(cpos, gpos, cinff, gamf, x, T, a0f);
      if (!any) { stop_at = l; break; }           // a0 = 0: nothing can fire
      if (l == lane) a0l = a0f;
      const float ul = __shfl_sync(full, u2f, l);
      int choice = spec_ok ? choice_count_f32<NA>(T, __fmul_rn(a0f, ul)) : -1;
      if (choice < 0) {                            // too close to call: exact arithmetic
        const double ud = __shfl_sync(full, u2, l);
        choice = exact_choice<NA>(cinf, p, x, ud);
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        if (2 * j == choice) { x[2 * j] -= 1; x[2 * j + 1] += 1; }
        if (2 * j + 1 == choice) { x[2 * j + 1] -= 1; x[2 * j] += 1; }
      }
    }
    int end_at = -1;
    double tau = 0.0;
    if (CLOCK < 2) {
      // 3. exact a0 and tau of each lane's draw
      double P = 0.0;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const double ainf = __dmul_rn(cinf[j], i2d_exact(xs[2 * j]));
        const double arec = __dmul_rn(p.gam[j], i2d_exact(xs[2 * j + 1]));
        const double A = __dadd_rn(ainf, arec);
        P = (j == 0) ? A : __dadd_rn(P, A);
      }
      tau = (lane < stop_at && pos(P)) ? div_pos(E, P) : 0.0;
    }
    if (CLOCK > 0) {
      // 4. Q62 scan of tau~ (binary32) or tau (binary64), certain decisions only
      const bool valid = lane < stop_at;
      uint64_t sc = 0ull, m = margin;
      sc = valid ? q62_of_f64(le_nonneg(tau, 1.5) ? tau : 1.5) : 0ull;
      m = ((uint64_t)kb + (uint64_t)lane + 2ull) << 10;   // (k + 2) 2^-52
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(full, sc, o);
        if (lane >= o) sc += y;
      }
      const uint64_t sl = tq + sc;
      const unsigned nc = __ballot_sync(full, valid && !(sl + m < kQ62One));
      if (nc != 0) {
        const int f = __ffs(nc) - 1;
        const unsigned st = __ballot_sync(full, valid && sl >= kQ62One + m);
        if (!((st >> f) & 1u)) return -1;         // too close to call
        end_at = f;
      } else {
        tq = __shfl_sync(full, sl, 31);
      }
    } else {
      // 4. clock in draw order
      for (int l = 0; l < stop_at; ++l) {
        const double tl = __shfl_sync(full, tau, l);
        const double tn = __dadd_rn(t, tl);
        if (le_nonneg(1.0, tn)) { end_at = l; break; }
        t = tn;
      }
    }
    if (end_at >= 0 || stop_at < 32) {
      const int at = end_at >= 0 ? end_at : stop_at;
      if (end_at >= 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) s.x[c] = __shfl_sync(full, xs[c], at);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) s.x[c] = x[c];
      }
      return fired + at;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) s.x[c] = x[c];
    fired += 32;
  }
}

// Group method: the warp's lanes form 32/SEG groups of SEG lanes, one node each
// (medium herds), with the binary32 clock: per round each group draws SEG steps
// at once and decides them by the fixed-point iteration of the warp method, with
// the clock inside every round (CLOCK = 2 above), all groups in lockstep (the
// warp iterates until every group is decided; a decided group's values stay put,
// as re-deciding a consistent guess gives the same values).  Every lane returns
// its group's result: the transitions fired, or -1 (binary32 bounds not met, or a
// clock decision too close to call) for the caller to rerun that node-day with
// the binary64 warp method.  Inactive groups (no node) return 0 at once.
template <int NA, int SEG>
__device__ __forceinline__ int32_t ssa_seg_node_day(const DevParams& p, uint64_t seed, uint32_t rep, int v, int day,
                                                    double phi, uint64_t margin, bool active, NodeState<NA>& s) {
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (SEG - 1);
  const int base = lane & ~(SEG - 1);
  const uint32_t full = 0xffffffffu;
  const uint32_t gfull = SEG == 32 ? full : ((1u << SEG) - 1u);
  double cinf[NA];
  float cinff[NA], gamf[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) cinf[j] = __dmul_rn(p.ups[j], phi);
  const bool spec_ok = spec_constants<NA>(p, cinf, s.x, cinff, gamf);
  bool cpos[NA], gpos[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) { cpos[j] = pos(cinf[j]); gpos[j] = pos(p.gam[j]); }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  int32_t result = 0, fired = 0;
  bool done = !active;
  if (active && !spec_ok) { result = -1; done = true; }
  uint64_t tq = 0;
  for (uint32_t kb = 0;; kb += SEG) {
    if (!done && kb >= kSpecMaxSteps) { result = -1; done = true; }
    if (__all_sync(full, done)) break;
    // 1. draws of this round
    const uint4 w = philox10(make_uint4((uint32_t)v, (uint32_t)day, kb + (uint32_t)gl, rep), k0, k1);
    const float Ef = neglog_f32(((((uint64_t)w.y) << 32) | w.x) >> 12);
    const float u2f = f32_of_q53(((((((uint64_t)w.w) << 32) | w.z) >> 12) << 1) | 1ull);
    // 2-4. fixed-point iteration with the clock in every round
    int32_t xs[NC];
    int ch = -3, e = SEG;
    uint64_t sl = 0;
    bool valid = false;
    unsigned okb = 0;
    for (int it = 0; it <= SEG; ++it) {
      prefix_state<NA, SEG>(s.x, ch, lane, xs);
      float T[2 * NA - 1], a0f;
      int nc = -2;
      valid = !done && thresholds_f32<NA>(cpos, gpos, cinff, gamf, xs, T, a0f);
      if (valid) {
        nc = choice_count_f32<NA>(T, __fmul_rn(a0f, u2f));
        if (nc < 0) nc = exact_choice<NA>(cinf, p, xs, uniform_open(w.z, w.w));
      }
      uint64_t sc = valid ? q62_of(fminf(__fdividef(Ef, a0f), 1.5f)) : 0ull;
#pragma unroll
      for (int o = 1; o < SEG; o <<= 1) {
        const uint64_t y = __shfl_up_sync(full, sc, o, SEG);
        if (gl >= o) sc += y;
      }
      sl = tq + sc;
      const unsigned notcont = (__ballot_sync(full, !(valid && sl + margin < kQ62One)) >> base) & gfull;
      e = notcont ? __ffs(notcont) - 1 : SEG;
      okb = (__ballot_sync(full, !valid || sl >= kQ62One + margin) >> base) & gfull;
      const unsigned diff = (__ballot_sync(full, nc != ch) >> base) & gfull & (e < SEG ? ((1u << e) - 1u) : gfull);
      ch = nc;
      if (__all_sync(full, done || diff == 0u)) break;
    }
    // outcome of the round, per group (every lane takes part in the shuffles)
    const int src = e < SEG ? e : SEG - 1;
    int32_t xe[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) xe[c] = __shfl_sync(full, xs[c], base + src);
    const int che = __shfl_sync(full, ch, base + src);
    const uint64_t sle = __shfl_sync(full, sl, base + src);
    if (!done) {
      if (e < SEG) {
        if ((okb >> e) & 1u) {
#pragma unroll
          for (int c = 0; c < NC; ++c) s.x[c] = xe[c];
          result = fired + e;
        } else {
          result = -1;                               // too close to call
        }
        done = true;
      } else {
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          const int dj = (che >= 0 && (che >> 1) == j) ? ((che & 1) ? -1 : 1) : 0;
          s.x[2 * j] = xe[2 * j] - dj;
          s.x[2 * j + 1] = xe[2 * j + 1] + dj;
        }
        tq = sle;
        fired += SEG;
      }
    }
  }
  return result;
}

// Adds one node-day's score terms to the node's accumulators (same op order as
// the oracle).
template <int NA>
__device__ __forceinline__ void accumulate_score(const SsaArgs& a, const DevParams& p, int r, int v,
                                                 double phi, const DayTerms (&T)[NA]) {
  double* sc = a.score + (size_t)r * kScoreTerms * a.N + v;
  double ups_int = 0.0;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    double gu = (pos(p.ups[j]) && pos(T[j].n_inf)) ? div_pos(T[j].n_inf, p.ups[j]) : 0.0;
    sc[(size_t)j * a.N] = __dadd_rn(__ldcg(sc + (size_t)j * a.N), __dsub_rn(gu, __dmul_rn(phi, T[j].int_s)));
    double gg = (pos(p.gam[j]) && pos(T[j].n_rec)) ? div_pos(T[j].n_rec, p.gam[j]) : 0.0;
    sc[(size_t)(3 + j) * a.N] = __dadd_rn(__ldcg(sc + (size_t)(3 + j) * a.N), __dsub_rn(gg, T[j].int_i));
    ups_int = __dadd_rn(ups_int, __dmul_rn(p.ups[j], T[j].int_s));
  }
  double ninf = 0.0;
#pragma unroll
  for (int j = 0; j < NA; ++j) ninf = __dadd_rn(ninf, T[j].n_inf);
  double cd = __dsub_rn((pos(phi) && pos(ninf)) ? div_pos(ninf, phi) : 0.0, ups_int);
  if (a.traj) {
    const size_t plane = (size_t)a.max_days * a.R * a.N, at = (size_t)a.day * a.R * a.N + (size_t)r * a.N + v;
    a.traj[at] = cd;
    a.traj[plane + at] = phi;
    return;
  }
  const double* tb = a.tang + ((size_t)r * 2 + 0) * a.N + v;
  const double* ta = a.tang + ((size_t)r * 2 + 1) * a.N + v;
  sc[(size_t)6 * a.N] = __dadd_rn(__ldcg(sc + (size_t)6 * a.N), __dmul_rn(cd, __ldcg(tb)));
  sc[(size_t)7 * a.N] = __dadd_rn(__ldcg(sc + (size_t)7 * a.N), __dmul_rn(cd, __ldcg(ta)));
}

// MODE 0: day a.day (prologue for a.day - 1 when a.prologue); MODE 1: finalize
// after the last day a.day (statistics of a.day; phi update in post-event mode).
constexpr int kRoleThread = 0;  // one node per thread
constexpr int kRoleWarp = 1;    // one node per warp (lane 0 stores and reports)
constexpr int kRoleGroup = 2;   // one node per group of kGroupLanes lanes (its first lane stores and reports)
constexpr int kGroupLanes = 8;

// One thread's part of node v of replicate r in the given role; then the warp's
// statistics and counters.
template <int NA, bool SCORE, int MODE>
__device__ __forceinline__ void node_day_work(const SsaArgs& a, int r, int v, bool active, int role) {
  const int lane = threadIdx.x & 31;
  const uint32_t full = 0xffffffffu;
  unsigned long long sI = 0, sN = 0, fired = 0;
  const bool do_prologue = (MODE == 1) || a.prologue;
  const int dprev = (MODE == 1) ? a.day : a.day - 1;
  const bool owner = role == kRoleThread || (role == kRoleWarp ? lane == 0 : (lane & (kGroupLanes - 1)) == 0);
  const DevParams& p = a.params[r];
  const uint32_t rep = (uint32_t)(a.rep_base + r);
  double* phip = a.phi + (size_t)r * a.N + v;
  NodeState<NA> s, s0;
  double phi = 0.0;
  int32_t f = 0;
  if (active) {
    load_counts<NA>(a, r, v, s);
    phi = __ldcg(phip);
    if (do_prologue) {
      if (owner) {
#pragma unroll
        for (int j = 0; j < NA; ++j) { sI += (unsigned)s.x[2 * j + 1]; sN += (unsigned)(s.x[2 * j] + s.x[2 * j + 1]); }
      }
      if (!a.pre_event) phi = phi_step<NA, SCORE>(a, p, r, v, dprev, s, phi);
    }
    s0 = s;
    if (MODE == 0 && role == kRoleThread) {
      f = -1;
      if (!SCORE && a.clock_margin) {
        double cinf[NA];
        float cinff[NA], gamf[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) cinf[j] = __dmul_rn(p.ups[j], phi);
        if (spec_constants<NA>(p, cinf, s.x, cinff, gamf)) {
          f = ssa_node_day_spec<NA>(p, a.seed, rep, v, a.day, cinf, cinff, gamf, a.clock_margin, s);
          if (f < 0) s = s0;
        }
      }
      if (SCORE) {
        DayTerms T[NA];
        f = (int32_t)ssa_node_day<NA, true>(p, a.seed, rep, v, a.day, phi, s, T);
        accumulate_score<NA>(a, p, r, v, phi, T);
      }
    }
  }
  if (MODE == 0 && !SCORE) {
    if (role == kRoleWarp) {
      if (active) {                                // warp-uniform
        f = -1;
        if (a.clock_margin) {
          f = ssa_warp_node_day<NA, 2>(p, a.seed, rep, v, a.day, phi, a.clock_margin, s);
          if (f < 0) s = s0;
        }
        if (f < 0) {
          f = ssa_warp_node_day<NA, 1>(p, a.seed, rep, v, a.day, phi, 0, s);
          if (f < 0) { s = s0; f = ssa_warp_node_day<NA, 0>(p, a.seed, rep, v, a.day, phi, 0, s); }
        }
      }
    } else {
      if (role == kRoleGroup) {                    // every lane of the warp takes part
        f = a.clock_margin ? ssa_seg_node_day<NA, kGroupLanes>(p, a.seed, rep, v, a.day, phi, a.clock_margin,
                                                               active, s)
                           : (active ? -1 : 0);
        if (f < 0) s = s0;
      }
      // nodes the binary32 clock could not decide (or could not take): the whole
      // warp runs the binary64 warp method for each of them in turn
      unsigned need = __ballot_sync(full, owner && active && f < 0);
      while (need) {
        const int l = __ffs(need) - 1;
        need &= need - 1;
        const int vl = __shfl_sync(full, v, l);
        const double phil = __shfl_sync(full, phi, l);
        NodeState<NA> t, t0;
#pragma unroll
        for (int c = 0; c < 2 * NA; ++c) t.x[c] = t0.x[c] = __shfl_sync(full, s0.x[c], l);
        int32_t g = ssa_warp_node_day<NA, 1>(p, a.seed, rep, vl, a.day, phil, 0, t);
        if (g < 0) { t = t0; g = ssa_warp_node_day<NA, 0>(p, a.seed, rep, vl, a.day, phil, 0, t); }
        const bool mine = role == kRoleGroup ? (lane & ~(kGroupLanes - 1)) == l : lane == l;
        if (mine) { s = t; f = g; }
      }
    }
  }
  if (active) {
    if (MODE == 0) {
      if (owner) fired = (unsigned long long)f;
      if (a.pre_event) phi = phi_step<NA, SCORE>(a, p, r, v, a.day, s, phi);
      if (owner) store_counts<NA>(a, r, v, s);
    }
    if (owner) *phip = phi;
  }
  if (!__any_sync(0xffffffffu, active)) return;
  fired = warp_sum(fired);
  sI = warp_sum(sI);
  sN = warp_sum(sN);
  if (lane == 0) {
    if (MODE == 0 && fired) atomicAdd(a.ctr + (size_t)r * 4 + 0, fired);
    if (do_prologue) {
      atomicAdd(a.prev_i + (size_t)r * a.max_days + dprev, sI);
      atomicAdd(a.prev_n + (size_t)r * a.max_days + dprev, sN);
    }
  }
}

// Block-contiguous mapping (the persistent batch kernel, score mode and the
// finalisation): with a node order (MODE 0), blocks [0, a.warp_blocks) give each
// warp one of the first a.n_big nodes of the order (warp-cooperative method);
// the other blocks give each thread one of the remaining nodes.
template <int NA, bool SCORE, int MODE>
__device__ __forceinline__ void node_day_block(const SsaArgs& a, int r, int bx) {
  const bool warp_role = (MODE == 0) && !SCORE && bx < a.warp_blocks;
  int v;
  bool active;
  if (warp_role) {
    const int wi = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    active = wi < a.n_big;
    v = active ? a.order[wi] : 0;
  } else {
    const int i = (bx - ((MODE == 0 && !SCORE) ? a.warp_blocks : 0)) * blockDim.x + threadIdx.x;
    if (MODE == 0 && !SCORE && a.order) {
      active = a.n_big + i < a.n_list;
      v = active ? a.order[a.n_big + i] : 0;
    } else {                                       // the handle's node range, in id order
      v = a.node_lo + i;
      active = v < a.node_hi;
      if (!active) v = 0;
    }
  }
  node_day_work<NA, SCORE, MODE>(a, r, v, active, warp_role ? kRoleWarp : kRoleThread);
}

// Dealt mapping of the per-day stochastic step: the work units are the
// warp-method nodes (largest first, a node's replicates together) and then groups
// of 32 consecutive per-thread nodes of the order (a.n_list of them; nodes marked
// in a.skip are left to another launch).  The grid is resident (at most
// one wave); warp w = slot * G + block takes units w, w + T, w + 2T, ... (T warps
// in all), so every block receives the same mix of heavy and light units, the
// heaviest ones first, and no SM carries the largest herds alone.
// In score mode every node is a per-thread node (a.n_big = a.n_mid = 0) and runs
// the binary64 method with its score terms; the dealing keeps herds of similar
// size in a warp, so its lanes finish close together.
template <int NA, bool SCORE>
__device__ __forceinline__ void node_day_dealt(const SsaArgs& a) {
  const int lane = threadIdx.x & 31;
  const int64_t T = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t R = a.R;
  const int64_t uw = R * a.n_big;                                    // one node per warp
  const int64_t ug = R * ((a.n_mid + 3) / 4);                        // four nodes per warp
  const int64_t ntu = (a.n_list - a.n_big - a.n_mid + 31) / 32;      // 32 nodes per warp
  const int64_t units = uw + ug + R * ntu;
  for (int64_t u = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; u < units; u += T) {
    int r = 0, v = 0, role = kRoleThread;
    bool active = false;
    if (u < uw) {
      r = (int)(u % R);
      v = a.order[u / R];
      active = true;
      role = kRoleWarp;
    } else if (u < uw + ug) {
      const int64_t ut = u - uw;
      r = (int)(ut % R);
      const int64_t i = a.n_big + (ut / R) * 4 + (lane / kGroupLanes);
      active = i < a.n_big + a.n_mid;
      v = active ? a.order[i] : 0;
      role = kRoleGroup;
    } else {
      const int64_t ut = u - uw - ug;
      r = (int)(ut % R);
      const int64_t i = a.n_big + a.n_mid + (ut / R) * 32 + lane;
      active = i < a.n_list;
      v = active ? a.order[i] : 0;
    }
    if (a.skip && active && ((__ldg(a.skip + (v >> 5)) >> (v & 31)) & 1u)) active = false;
    node_day_work<NA, SCORE, 0>(a, r, v, active, role);
  }
}

}  // namespace episim
