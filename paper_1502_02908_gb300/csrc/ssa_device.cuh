// Device code of the stochastic step (Eq. (numstep3); Sec. 3.3 Eqs. (sampling),
// (sampling2); Alg. 1 lines 3-10) with the fused phi update (Eq. (numstep5)):
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
// Warp-cooperative direct method for one node-day (large herds).  Identical
// results to ssa_node_day, bit for bit, in four phases per block of 32 draws:
//  1. lane l computes draw k0 + l: Philox, E = -log(u1), u2 (independent of the
//     state, so all 32 in parallel);
//  2. every lane runs the embedded jump chain (which transition each draw
//     fires) over the block in FP32.  Each FP32 comparison is decisive only when
//     the operands are at least 64 float ulps apart (relative gap >= 2^-18,
//     beyond the <= 2^-20 error of the FP32 rates, sums and product against the
//     specification's binary64 values); otherwise that draw is decided with the
//     specification's exact binary64 arithmetic;
//  3. lane l computes the exact binary64 propensity sum a0 of its draw's state
//     and tau_l = E_l / a0;
//  4. the binary64 clock t + tau_l runs in draw order; the first draw reaching
//     t >= 1 ends the day in the state before that draw.
// On GB300 the serial chain of the per-thread method costs ~8 FP64 instructions
// (64 cycles each) plus a divide per transition; here it is FP32 and integer.

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

template <int NA>
__device__ __forceinline__ uint32_t ssa_warp_node_day(const DevParams& p, uint64_t seed, uint32_t rep, int v,
                                                      int day, double phi, NodeState<NA>& s) {
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  const uint32_t full = 0xffffffffu;
  double cinf[NA];
  float cinff[NA], gamf[NA];
  bool spec_ok = true;
  int32_t herd = 0;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    cinf[j] = __dmul_rn(p.ups[j], phi);
    for (int q = 0; q < 2; ++q) {
      const double c = q ? p.gam[j] : cinf[j];
      const int e = (int)(double_bits(c) >> 52) - 1023;
      if (pos(c) && (e < -100 || e > 60)) spec_ok = false;
    }
    cinff[j] = trunc_to_f32(cinf[j]);
    gamf[j] = trunc_to_f32(p.gam[j]);
    herd += s.x[2 * j] + s.x[2 * j + 1];
  }
  if (herd >= (1 << 22)) spec_ok = false;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  double t = 0.0;
  uint32_t fired = 0;
  for (uint32_t kb = 0;; kb += 32) {
    // 1. draws of this block
    const uint4 w = philox10(make_uint4((uint32_t)v, (uint32_t)day, kb + (uint32_t)lane, rep), k0, k1);
    const double E = neglog_u(((((uint64_t)w.y) << 32) | w.x) >> 12);
    const double u2 = uniform_open(w.z, w.w);
    const float u2f = trunc_to_f32(u2);
    // 2. embedded chain
    int32_t x[NC], xs[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { x[c] = s.x[c]; xs[c] = x[c]; }
    int stop_at = 32;
    for (int l = 0; l < 32; ++l) {
      if (l == lane) {
#pragma unroll
        for (int c = 0; c < NC; ++c) xs[c] = x[c];
      }
      bool posA[NA], posI[NA];
      float aif[NA], Pf[NA];
      bool any = false;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        posI[j] = pos(cinf[j]) && x[2 * j] > 0;
        const bool posR = pos(p.gam[j]) && x[2 * j + 1] > 0;
        posA[j] = posI[j] || posR;
        any = any || posA[j];
        aif[j] = __fmul_rn(cinff[j], small_int_to_f32(x[2 * j]));
        const float arf = __fmul_rn(gamf[j], small_int_to_f32(x[2 * j + 1]));
        const float Af = __fadd_rn(aif[j], arf);
        Pf[j] = (j == 0) ? Af : __fadd_rn(Pf[j > 0 ? j - 1 : 0], Af);
      }
      if (!any) { stop_at = l; break; }           // a0 = 0: nothing can fire
      const float ul = __shfl_sync(full, u2f, l);
      int choice = -1;
      if (spec_ok) {
        const float rf = __fmul_rn(Pf[NA - 1], ul);
        int cls = -1, last = -1;
        bool amb = false;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          if (cls < 0 && !amb && posA[j]) {
            last = j;
            const int cmp = cmp_f32(rf, Pf[j]);
            if (cmp == 0) amb = true;
            else if (cmp < 0) cls = j;
          }
        }
        if (!amb) {
          if (cls < 0) cls = last;
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            if (j != cls) continue;
            const bool posR = pos(p.gam[j]) && x[2 * j + 1] > 0;
            if (!posI[j]) choice = 2 * j + 1;
            else if (!posR) choice = 2 * j;
            else {
              const float thrf = (j == 0) ? aif[0] : __fadd_rn(Pf[j > 0 ? j - 1 : 0], aif[j]);
              const int cmp = cmp_f32(rf, thrf);
              if (cmp != 0) choice = 2 * j + (cmp < 0 ? 0 : 1);
            }
          }
        }
      }
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
    // 3. exact a0 and tau of each lane's draw
    double P = 0.0;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const double ainf = __dmul_rn(cinf[j], i2d_exact(xs[2 * j]));
      const double arec = __dmul_rn(p.gam[j], i2d_exact(xs[2 * j + 1]));
      const double A = __dadd_rn(ainf, arec);
      P = (j == 0) ? A : __dadd_rn(P, A);
    }
    const double tau = (lane < stop_at && pos(P)) ? div_pos(E, P) : 0.0;
    // 4. clock in draw order
    int end_at = -1;
    for (int l = 0; l < stop_at; ++l) {
      const double tl = __shfl_sync(full, tau, l);
      const double tn = __dadd_rn(t, tl);
      if (le_nonneg(1.0, tn)) { end_at = l; break; }
      t = tn;
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
      return fired + (uint32_t)at;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) s.x[c] = x[c];
    fired += 32;
  }
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
// With a node order (MODE 0), blocks [0, a.warp_blocks) give each warp one of the
// first a.n_big nodes of the order (warp-cooperative method); the other blocks
// give each thread one of the remaining nodes.
template <int NA, bool SCORE, int MODE>
__device__ __forceinline__ void node_day_block(const SsaArgs& a, int r, int bx) {
  const int lane = threadIdx.x & 31;
  const bool warp_role = (MODE == 0) && !SCORE && bx < a.warp_blocks;
  int v;
  bool active;
  if (warp_role) {
    const int wi = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    active = wi < a.n_big;
    v = active ? a.order[wi] : 0;
  } else {
    const int i = (bx - ((MODE == 0 && !SCORE) ? a.warp_blocks : 0)) * blockDim.x + threadIdx.x;
    const int base = (MODE == 0 && !SCORE && a.order) ? a.n_big : 0;
    active = i + base < a.N;
    v = active ? (a.order && MODE == 0 && !SCORE ? a.order[base + i] : i + base) : 0;
  }
  unsigned long long sI = 0, sN = 0, fired = 0;
  const bool do_prologue = (MODE == 1) || a.prologue;
  const int dprev = (MODE == 1) ? a.day : a.day - 1;
  const bool owner = !warp_role || lane == 0;     // the thread that stores and reports
  if (active) {
    const DevParams& p = a.params[r];
    NodeState<NA> s;
    load_counts<NA>(a, r, v, s);
    double* phip = a.phi + (size_t)r * a.N + v;
    double phi = __ldcg(phip);
    if (do_prologue) {
      if (owner) {
#pragma unroll
        for (int j = 0; j < NA; ++j) { sI += (unsigned)s.x[2 * j + 1]; sN += (unsigned)(s.x[2 * j] + s.x[2 * j + 1]); }
      }
      if (!a.pre_event) phi = phi_step<NA, SCORE>(a, p, r, v, dprev, s, phi);
    }
    if (MODE == 0) {
      if (warp_role) {
        const uint32_t f = ssa_warp_node_day<NA>(p, a.seed, (uint32_t)(a.rep_base + r), v, a.day, phi, s);
        if (owner) fired = f;
      } else {
        DayTerms T[NA];
        fired = ssa_node_day<NA, SCORE>(p, a.seed, (uint32_t)(a.rep_base + r), v, a.day, phi, s, T);
        if (SCORE) accumulate_score<NA>(a, p, r, v, phi, T);
      }
      if (a.pre_event) phi = phi_step<NA, SCORE>(a, p, r, v, a.day, s, phi);
      if (owner) store_counts<NA>(a, r, v, s);
    }
    if (owner) *phip = phi;
  }
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

}  // namespace episim
