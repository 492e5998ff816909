// Kernels of the general compartment model (Secs. 2.1-2.2, 3.1-3.3): the
// stochastic step (direct method per node with a sparse dependency graph), the
// event step (one thread per component of the day's transfer graph) and the
// continuous update (Eqs. (numstep5) and (numstep2)).
//
// Arithmetic: rates, a0, thresholds, tau and the continuous update are binary64
// with the operation order of include/episim_general.h (no contraction; the
// build passes -fmad=false); -log(u) is the exact fixed-point logarithm of the
// SISe kernels; comparisons of non-negative doubles compare bit patterns.
#include "../../include/episim_general.h"
#include "devmath.cuh"
#include "general.h"
#include "softdiv.cuh"
#include "ssa_device.cuh"   // the binary32 helpers of the speculative clock

#include <algorithm>

namespace episim {

namespace {

__device__ __forceinline__ void copy16(void* dst, const void* src, int n16) {
  int4* d = reinterpret_cast<int4*>(dst);
  const int4* s = reinterpret_cast<const int4*>(src);
  for (int i = threadIdx.x; i < n16; i += blockDim.x) d[i] = __ldg(s + i);
}

// Exact binary64 of 0 <= n < 2^53 on the integer pipe.
__device__ __forceinline__ double u2d_exact(long long n) {
  if (n <= 0) return 0.0;
  const uint64_t u = (uint64_t)n;
  const int top = 63 - __clzll(u);
  const uint64_t mant = (u << (52 - top)) & ((1ull << 52) - 1);
  return bits_to_double(((uint64_t)(1023 + top) << 52) | mant);
}

__device__ __forceinline__ long long mask_sum(const int32_t* x, int stride, uint32_t mask, int nc) {
  long long s = 0;
  for (int c = 0; c < nc; ++c)
    if (mask >> c & 1u) s += x[c * stride];
  return s;
}

// a_j = k_j [* y_q] [* x_a] [* x_b] [/ P], left to right (IEEE products; the
// quotient by the integer-pipe division, bit-identical to IEEE).
__device__ __forceinline__ double gen_rate(const GenModelDev& m, const GenRepParams& p, const int32_t* x, int stride,
                                        const double* y, int j) {
  double a = p.rate[j];
  const int q = m.fy[j], fa = m.fa[j], fb = m.fb[j];
  const uint32_t pm = m.pop[j];
  if (q >= 0) a = __dmul_rn(a, y[q]);
  if (fa >= 0) a = __dmul_rn(a, i2d_exact(x[fa * stride]));
  if (fb >= 0) a = __dmul_rn(a, i2d_exact(x[fb * stride]));
  if (pm) {
    const long long P = mask_sum(x, stride, pm, m.nc);
    a = (P > 0 && pos(a)) ? div_pos(a, u2d_exact(P)) : 0.0;
  }
  return a;
}

__device__ __forceinline__ double gen_y_next(const GenModelDev& m, const GenRepParams& p, int q, int day,
                                             double y, double U, double D) {
  const double omb = __dsub_rn(1.0, p.beta[q][season_of(day)]);
  double mid;
  if (m.den[q] == 0u) mid = __dmul_rn(p.alpha[q], U);
  else mid = D > 0.0 ? __ddiv_rn(__dmul_rn(p.alpha[q], U), D) : 0.0;
  return __dadd_rn(__dadd_rn(__dmul_rn(y, omb), mid), p.eps[q]);
}

// Per-thread rate storage in shared memory: rate j of the thread at a[j * stride],
// its left-to-right partial sum at P[j * stride] (rolled loops keep the kernel
// small enough for the instruction cache).
struct RateRow {
  double* a;
  double* P;
  int stride;
};

// P_j = P_{j-1} + a_j for j >= j0 (P_0 = a_0, which equals 0 + a_0 for a_0 >= 0);
// returns a0 = P_{nt-1}.
__device__ __forceinline__ double prefix_from(const RateRow& R, int nt, int j0) {
  double run = j0 > 0 ? R.P[(j0 - 1) * R.stride] : 0.0;
  for (int j = j0; j < nt; ++j) {
    run = j == 0 ? R.a[0] : __dadd_rn(run, R.a[j * R.stride]);
    R.P[j * R.stride] = run;
  }
  return nt > 0 ? R.P[(nt - 1) * R.stride] : 0.0;
}

// Eq. (sampling2): the first j with a_j > 0 and r <= P_j, else the last j with a_j > 0.
__device__ __forceinline__ int select_transition(const RateRow& R, int nt, double r) {
  int last = -1;
  for (int j = 0; j < nt; ++j)
    if (pos(R.a[j * R.stride])) {
      last = j;
      if (le_nonneg(r, R.P[j * R.stride])) return j;
    }
  return last;
}

__device__ __forceinline__ void apply_changes(const GenModelDev& m, int32_t* x, int stride, int n, int times) {
  for (int q = m.chg_off[n]; q < m.chg_off[n + 1]; ++q) {
    const uint32_t c = m.chg[q];
    x[(c & 0xffu) * stride] += times * ((int32_t)c >> 8);
  }
}

// Direct method of one node-day by one thread (Eqs. (sampling), (sampling2));
// x is the node's counts in shared memory (stride = threads per block).  After a
// firing only the rates of its dependency graph are recomputed, and the partial
// sums from the first of them on.
__device__ __forceinline__ uint32_t gen_node_day(const GenModelDev& m, const GenRepParams& p, int32_t* x,
                                                 int stride, const RateRow& R, const double* y, uint32_t v,
                                                 uint32_t day, uint32_t rep, uint32_t k0, uint32_t k1) {
  const int nt = m.nt;
  for (int j = 0; j < nt; ++j) R.a[j * R.stride] = gen_rate(m, p, x, stride, y, j);
  double a0 = prefix_from(R, nt, 0);
  double t = 0.0;
  uint32_t fired = 0;
  for (uint32_t k = 0; pos(a0); ++k) {
    const uint4 w = philox10(make_uint4(v, day, k, rep), k0, k1);
    const double E = neglog_u((((uint64_t)w.y << 32) | w.x) >> 12);
    const double u2 = uniform_open(w.z, w.w);
    const double tn = __dadd_rn(t, div_pos(E, a0));
    if (le_nonneg(1.0, tn)) break;
    t = tn;
    const int chosen = select_transition(R, nt, __dmul_rn(a0, u2));
    apply_changes(m, x, stride, chosen, 1);
    uint32_t dm = m.dep[chosen];
    const int j0 = dm ? __ffs(dm) - 1 : nt;
    while (dm) {
      const int j = __ffs(dm) - 1;
      dm &= dm - 1u;
      R.a[j * R.stride] = gen_rate(m, p, x, stride, y, j);
    }
    a0 = prefix_from(R, nt, j0);
    ++fired;
  }
  return fired;
}

// Direct method of one node-day by a segment of SEG lanes (a whole warp, SEG =
// 32, or a quarter, SEG = 8, four nodes to a warp), SEG draws per round.  Lane l
// of the segment takes draw k + l.  Its state is the round's base state plus the
// transitions the segment's lanes before it choose; the choices are found by a
// fixed-point iteration (each lane chooses at the state the current choices of
// the lanes before it imply; lane 0's choice is final after one pass, and each
// pass fixes at least one more lane, so the choices settle within SEG passes).
// The clock then runs over the segment's lanes in draw order with the binary64
// sums of the sequential method, so the result is that method's.  Every lane of
// the warp takes part in its collectives; lanes of a segment without a node
// (live = false) only vote.  xl: this lane's counts (shared memory, stride as in
// the thread method); base: the segment's counts at the start of the round;
// ctau, cch: the segment's SEG clock increments and choices; sl, sb: the lane's
// index in its segment and the segment's first lane in the warp.
template <int SEG>
__device__ __forceinline__ uint32_t gen_seg_node_day(const GenModelDev& m, const GenRepParams& p, int32_t* xl,
                                                     int32_t* base, int stride, const RateRow& R, double* ctau,
                                                     int32_t* cch, const double* y, uint32_t v, uint32_t day,
                                                     uint32_t rep, uint32_t k0, uint32_t k1, int sl, int sb,
                                                     bool live) {
  const int nt = m.nt, nc = m.nc;
  const unsigned full = 0xffffffffu;
  const unsigned seg = SEG == 32 ? full : (((1u << SEG) - 1u) << sb);
  const unsigned below = ((1u << sl) - 1u) << sb;
  live = live && nt > 0;
  double t = 0.0;
  uint32_t fired = 0;
  for (uint32_t kb = 0; __any_sync(full, live); kb += SEG) {
    double E = 0.0, u2 = 0.0;
    if (live) {
      const uint4 w = philox10(make_uint4(v, day, kb + (uint32_t)sl, rep), k0, k1);
      E = neglog_u((((uint64_t)w.y << 32) | w.x) >> 12);
      u2 = uniform_open(w.z, w.w);
    }
    int choice = -1;
    double tau = 0.0;
    for (int pass = 0; pass <= SEG; ++pass) {
      if (live)
        for (int c = 0; c < nc; ++c) xl[c * stride] = base[c];
      for (int j = 0; j < nt; ++j) {
        const int cnt = __popc(__ballot_sync(full, live && choice == j) & below);
        if (cnt) apply_changes(m, xl, stride, j, cnt);
      }
      int next = -1;
      if (live) {
        for (int j = 0; j < nt; ++j) R.a[j * R.stride] = gen_rate(m, p, xl, stride, y, j);
        const double a0 = prefix_from(R, nt, 0);
        if (pos(a0)) {
          next = select_transition(R, nt, __dmul_rn(a0, u2));
          tau = div_pos(E, a0);
        }
      }
      const bool changed = __any_sync(full, live && next != choice);
      choice = next;
      if (!changed) break;
    }
    if (live) {
      ctau[sl] = tau;
      cch[sl] = choice;
    }
    __syncwarp();
    // clock over the segment's lanes in draw order (every lane of it runs the same sums)
    int stop = SEG;
    if (live)
      for (int l = 0; l < SEG; ++l) {
        if (cch[l] < 0) { stop = l; break; }
        const double tn = __dadd_rn(t, ctau[l]);
        if (le_nonneg(1.0, tn)) { stop = l; break; }
        t = tn;
      }
    const unsigned fired_lanes = stop == SEG ? seg : (((1u << stop) - 1u) << sb);
    for (int j = 0; j < nt; ++j) {
      const int cnt = __popc(__ballot_sync(full, live && choice == j) & fired_lanes);
      if (cnt && live && sl == 0) apply_changes(m, base, 1, j, cnt);
    }
    __syncwarp();
    if (live) {
      fired += (uint32_t)stop;
      if (stop < SEG) live = false;
    }
  }
  return fired;
}

constexpr int kGenSeg = 8;                          // lanes per node of the group method
constexpr int kGenWarps = kGenThreads / 32;
constexpr int kGenEventWarps = 8192;                // event step: a warp per component up to this many

// ---------------------------------------------------------------------------
// Speculative binary32 direct method of one node-day (one thread), the general
// form of the SISe kernels' certified clock.  With u = 2^-24, nt <= 32 and every
// rate constant and continuous variable 0 or within [2^-30, 2^30], counts below
// 2^21 (so every population below 2^23 is exact in binary32): a binary32 rate
// (constant and variable truncated to binary32, 2u each; at most three products
// and one IEEE quotient, u each) is within 8u of the binary64 rate, and never 0
// unless that rate is 0; a left-to-right partial sum P~_j of non-negative terms
// is within (nt + 8)u of P_j, r~ = a0~ u2~ within (nt + 10)u of r.  A selection
// is taken in binary32 only when r~ and every threshold it is compared with are
// at least 2 nt + 32 float ulps apart (their relative gap then exceeds the sum of
// the two bounds), else the exact binary64 rule decides that step.  The clock:
// tau~ = E~ / a0~ (E~ within 16u, the fast quotient 4u) is within (nt + 28)u <=
// 60u of tau; accumulated exactly in Q62 it stays, at a decision (sum < 2.5),
// within 150u plus k (2^-53 + 2^-62) of the binary64 chain, so a margin of 2^-16
// (256u) makes "sum >= 1 + margin" a certain stop and "sum + margin < 1" a
// certain continue; a decision in between hands the node-day back to the exact
// method.  The results are the specification's, bit for bit.
constexpr uint32_t kGenSpecMaxSteps = 1u << 21;

// binary32 of rate j, in gen_rate's order; exactly 0 when the binary64 rate is.
__device__ __forceinline__ float gen_rate_f32(const GenModelDev& m, const GenRepParams& p, const int32_t* x,
                                              int stride, const float* yf, int j) {
  float a = trunc_to_f32(p.rate[j]);
  const int q = m.fy[j], fa = m.fa[j], fb = m.fb[j];
  const uint32_t pm = m.pop[j];
  if (q >= 0) a = __fmul_rn(a, yf[q]);
  if (fa >= 0) a = __fmul_rn(a, small_int_to_f32(x[fa * stride]));
  if (fb >= 0) a = __fmul_rn(a, small_int_to_f32(x[fb * stride]));
  if (pm) {
    const long long P = mask_sum(x, stride, pm, m.nc);
    a = (P > 0 && a > 0.0f) ? __fdiv_rn(a, small_int_to_f32((int32_t)P)) : 0.0f;
  }
  return a;
}

// The exact rule of Eq. (sampling2) for state x and uniform u2, in two passes of
// binary64 rates (a0 first, then the running sums): the transition chosen.
__device__ __forceinline__ int gen_exact_choice(const GenModelDev& m, const GenRepParams& p, const int32_t* x,
                                                int stride, const double* y, double u2) {
  const int nt = m.nt;
  double a0 = 0.0;
  for (int j = 0; j < nt; ++j) {
    const double aj = gen_rate(m, p, x, stride, y, j);
    a0 = j == 0 ? aj : __dadd_rn(a0, aj);
  }
  const double r = __dmul_rn(a0, u2);
  double run = 0.0;
  int last = -1;
  for (int j = 0; j < nt; ++j) {
    const double aj = gen_rate(m, p, x, stride, y, j);
    run = j == 0 ? aj : __dadd_rn(run, aj);
    if (pos(aj)) {
      last = j;
      if (le_nonneg(r, run)) return j;
    }
  }
  return last;
}

// Transitions fired, -1 when a clock decision was too close to call (the caller
// reruns the node-day exactly from its start), -2 when the binary32 bounds do not
// hold for this node-day (the caller runs it exactly; x is untouched).  The
// binary32 rates af_j and partial sums Pf_j live in the thread's row of R.P,
// viewed as pairs of floats.
__device__ __forceinline__ int32_t gen_node_day_spec(const GenModelDev& m, const GenRepParams& p, int32_t* x,
                                                     int stride, const RateRow& R, const double* y, uint32_t v,
                                                     uint32_t day, uint32_t rep, uint32_t k0, uint32_t k1,
                                                     uint64_t margin) {
  const int nt = m.nt, nc = m.nc, ny = m.ny;
  if (nt == 0) return 0;                                      // no transitions: nothing fires
  bool ok = true;
  for (int j = 0; j < nt; ++j) {
    const double c = p.rate[j];
    const int e = (int)(double_bits(c) >> 52) - 1023;
    if (pos(c) && (e < -30 || e > 29)) ok = false;
  }
  float yf[kGenMaxCont];
  for (int q = 0; q < ny; ++q) {
    const double c = y[q];
    const int e = (int)(double_bits(c) >> 52) - 1023;
    if (pos(c) && (e < -30 || e > 29)) ok = false;
    if (!pos(c) && double_bits(c) != 0ull) ok = false;       // negative or -0: exact method
    yf[q] = pos(c) ? trunc_to_f32(c) : 0.0f;
  }
  long long tot = 0;
  for (int c = 0; c < nc; ++c) tot += x[c * stride];
  if (!ok || tot >= (1 << 21)) return -2;
  float* F = reinterpret_cast<float*>(R.P);
  const int S2 = 2 * R.stride;
  const int M = 2 * nt + 32;                                  // decisive gap in float ulps
  float run = 0.0f;
  for (int j = 0; j < nt; ++j) {
    const float aj = gen_rate_f32(m, p, x, stride, yf, j);
    run = j == 0 ? aj : __fadd_rn(run, aj);
    F[j * S2] = aj;
    F[j * S2 + 1] = run;
  }
  uint64_t tq = 0;
  uint4 wn = philox10(make_uint4(v, day, 0u, rep), k0, k1);
  for (uint32_t k = 0;; ++k) {
    const float a0f = F[(nt - 1) * S2 + 1];
    const uint4 w = wn;
    wn = philox10(make_uint4(v, day, k + 1u, rep), k0, k1);
    if (!(a0f > 0.0f)) return (int32_t)k;                     // every rate 0: the day ends
    const float Ef = neglog_f32(((((uint64_t)w.y) << 32) | w.x) >> 12);
    const float u2f = f32_of_q53(((((((uint64_t)w.w) << 32) | w.z) >> 12) << 1) | 1ull);
    const uint64_t sq = tq + q62_of(fminf(__fdividef(Ef, a0f), 1.5f));
    if (sq >= kQ62One + margin) return (int32_t)k;
    if (sq + margin >= kQ62One || k + 1u >= kGenSpecMaxSteps) return -1;
    // selection: the first j with a_j > 0 and r <= P_j, each comparison decisive
    const float rf = __fmul_rn(a0f, u2f);
    const int ir = __float_as_int(rf);
    int chosen = -1;
    bool amb = ir < 0x00800000;
    for (int j = 0; j < nt && !amb && chosen < 0; ++j) {
      if (!(F[j * S2] > 0.0f)) continue;
      const int d = ir - __float_as_int(F[j * S2 + 1]);
      if (d <= -M) chosen = j;
      else if (d < M) amb = true;
    }
    if (amb || chosen < 0) chosen = gen_exact_choice(m, p, x, stride, y, uniform_open(w.z, w.w));
    for (int q = m.chg_off[chosen]; q < m.chg_off[chosen + 1]; ++q) {
      const uint32_t c = m.chg[q];
      const int32_t dlt = (int32_t)c >> 8;
      x[(c & 0xffu) * stride] += dlt;
      tot += dlt;
    }
    if (tot >= (1 << 22)) return -1;                          // populations no longer exact in binary32
    uint32_t dm = m.dep[chosen];
    const int j0 = dm ? __ffs(dm) - 1 : nt;
    while (dm) {
      const int j = __ffs(dm) - 1;
      dm &= dm - 1u;
      F[j * S2] = gen_rate_f32(m, p, x, stride, yf, j);
    }
    float pr = j0 > 0 ? F[(j0 - 1) * S2 + 1] : 0.0f;
    for (int j = j0; j < nt; ++j) {
      pr = j == 0 ? F[0] : __fadd_rn(pr, F[j * S2]);
      F[j * S2 + 1] = pr;
    }
    tq = sq;
  }
}

// The segment method (gen_seg_node_day) with the binary32 arithmetic of
// gen_node_day_spec: each lane's draw gives E~ and u2~; the fixed-point iteration
// over the segment's lanes chooses with binary32 rates and partial sums, a choice
// taken in binary32 only when decisive (else gen_exact_choice at that lane's
// state), so the converged choices are the binary64 method's; each lane's tau~ =
// E~ / a0~ goes into an exact Q62 scan over the segment, and a lane is a certain
// continue when its clock plus the margin is below 1, a certain stop when its
// clock is at least 1 plus the margin (or it has no positive rate).  The day
// ends at the first lane that is not a certain continue; when that lane is not a
// certain stop, or a state it decides at leaves the bounds (a negative count, a
// population of 2^22 or more), the segment gives up.  Returns, for every lane,
// its segment's transitions fired; -1 when the segment gave up after changing
// `base` (the caller reloads the day's start state and reruns the node-day with
// gen_seg_node_day), -2 when the bounds fail at the day's start (nothing changed);
// 0 for lanes without a node.  Every lane of the warp takes part in the
// collectives.
template <int SEG>
__device__ __forceinline__ int32_t gen_seg_node_day_spec(const GenModelDev& m, const GenRepParams& p, int32_t* xl,
                                                         int32_t* base, int stride, const RateRow& R,
                                                         const double* y, uint32_t v, uint32_t day, uint32_t rep,
                                                         uint32_t k0, uint32_t k1, int sl, int sb, bool live,
                                                         uint64_t margin) {
  const int nt = m.nt, nc = m.nc, ny = m.ny;
  const unsigned full = 0xffffffffu;
  const unsigned seg = SEG == 32 ? full : (((1u << SEG) - 1u) << sb);
  const unsigned below = ((1u << sl) - 1u) << sb;
  float* F = reinterpret_cast<float*>(R.P);
  const int S2 = 2 * R.stride;
  const int M = 2 * nt + 32;                                  // decisive gap in float ulps
  int32_t status = 0;
  float yf[kGenMaxCont];
  bool act = live && nt > 0;
  if (act) {
    bool ok = true;
    for (int j = 0; j < nt; ++j) {
      const double c = p.rate[j];
      const int e = (int)(double_bits(c) >> 52) - 1023;
      if (pos(c) && (e < -30 || e > 29)) ok = false;
    }
    for (int q = 0; q < ny; ++q) {
      const double c = y[q];
      const int e = (int)(double_bits(c) >> 52) - 1023;
      if (pos(c) && (e < -30 || e > 29)) ok = false;
      if (!pos(c) && double_bits(c) != 0ull) ok = false;     // negative or -0: exact method
      yf[q] = pos(c) ? trunc_to_f32(c) : 0.0f;
    }
    long long tot = 0;
    for (int c = 0; c < nc; ++c) tot += base[c];
    if (!ok || tot >= (1 << 21)) { status = -2; act = false; }
  }
  uint64_t tq = 0;
  uint32_t fired = 0;
  for (uint32_t kb = 0; __any_sync(full, act); kb += SEG) {
    float Ef = 0.0f, u2f = 0.0f;
    uint32_t wz = 0, ww = 0;
    if (act) {
      const uint4 w = philox10(make_uint4(v, day, kb + (uint32_t)sl, rep), k0, k1);
      Ef = neglog_f32((((uint64_t)w.y << 32) | w.x) >> 12);
      u2f = f32_of_q53(((((((uint64_t)w.w) << 32) | w.z) >> 12) << 1) | 1ull);
      wz = w.z;
      ww = w.w;
    }
    int choice = -1;
    float a0f = 0.0f;
    bool bad = false;
    for (int pass = 0; pass <= SEG; ++pass) {
      if (act)
        for (int c = 0; c < nc; ++c) xl[c * stride] = base[c];
      for (int j = 0; j < nt; ++j) {
        const int cnt = __popc(__ballot_sync(full, act && choice == j) & below);
        if (cnt) apply_changes(m, xl, stride, j, cnt);
      }
      int next = -1;
      if (act) {
        long long tot = 0;
        bool neg = false;
        for (int c = 0; c < nc; ++c) {
          const int32_t xc = xl[c * stride];
          tot += xc;
          neg = neg || xc < 0;
        }
        bad = neg || tot >= (1 << 22);
        float run = 0.0f;
        for (int j = 0; j < nt; ++j) {
          const float aj = bad ? 0.0f : gen_rate_f32(m, p, xl, stride, yf, j);
          run = j == 0 ? aj : __fadd_rn(run, aj);
          F[j * S2] = aj;
          F[j * S2 + 1] = run;
        }
        a0f = run;
        if (!bad && a0f > 0.0f) {
          const float rf = __fmul_rn(a0f, u2f);
          const int ir = __float_as_int(rf);
          bool amb = ir < 0x00800000;
          for (int j = 0; j < nt && !amb && next < 0; ++j) {
            if (!(F[j * S2] > 0.0f)) continue;
            const int d = ir - __float_as_int(F[j * S2 + 1]);
            if (d <= -M) next = j;
            else if (d < M) amb = true;
          }
          if (amb || next < 0) next = gen_exact_choice(m, p, xl, stride, y, uniform_open(wz, ww));
        }
      }
      const bool changed = __any_sync(full, act && next != choice);
      choice = next;
      if (!changed) break;
    }
    // the segment's clock after each lane's draw, exactly in Q62
    uint64_t S = (act && !bad && choice >= 0) ? q62_of(fminf(__fdividef(Ef, a0f), 1.5f)) : 0ull;
    for (int d = 1; d < SEG; d <<= 1) {
      const uint64_t o = __shfl_up_sync(full, S, d, SEG);
      if (sl >= d) S += o;
    }
    S += tq;
    const bool cont = act && !bad && choice >= 0 && S + margin < kQ62One;
    const bool stop_ok = act && !bad && (choice < 0 || S >= kQ62One + margin);
    const unsigned notc = __ballot_sync(full, act && !cont) & seg;
    const unsigned sure = __ballot_sync(full, stop_ok) & seg;
    int stop = SEG;
    if (act && notc) {
      const int e = __ffs(notc) - 1;                           // absolute lane of the first non-continue
      if ((sure >> e) & 1u) stop = e - sb;
      else status = -1;
    }
    if (act && status == 0 && stop == SEG && kb + 2u * SEG >= kGenSpecMaxSteps) status = -1;
    const bool apply = act && status == 0;
    const unsigned fired_lanes = stop == SEG ? seg : (((1u << stop) - 1u) << sb);
    for (int j = 0; j < nt; ++j) {
      const int cnt = __popc(__ballot_sync(full, apply && choice == j) & fired_lanes);
      if (cnt && apply && sl == 0) apply_changes(m, base, 1, j, cnt);
    }
    __syncwarp();
    const uint64_t tq_end = __shfl_sync(full, S, sb + SEG - 1);
    if (act) {
      if (status < 0) act = false;
      else {
        fired += (uint32_t)stop;
        if (stop < SEG) act = false;
        else tq = tq_end;
      }
    }
  }
  if (!live) return 0;
  return status < 0 ? status : (int32_t)fired;
}

// At most 128 registers a thread (110 used): with __launch_bounds__ alone ptxas
// settled at 72 and spilled inside the binary32 segment method.
__global__ void __maxnreg__(128) k_gen_ssa(GenSsaArgs a) {
  extern __shared__ int4 smem4[];
  GenModelDev& m = *reinterpret_cast<GenModelDev*>(smem4);
  char* sp = reinterpret_cast<char*>(smem4) + sizeof(GenModelDev);
  GenRepParams& p = *reinterpret_cast<GenRepParams*>(sp);
  sp += sizeof(GenRepParams);
  double* ctau = reinterpret_cast<double*>(sp);                 // [threads]: per lane
  sp += kGenThreads * sizeof(double);
  const int r = blockIdx.y;
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  copy16(&p, a.params + r, (int)(sizeof(GenRepParams) / 16));
  __syncthreads();
  const int nc = m.nc, nt = m.nt, ny = m.ny, N = a.N;
  double* rates = reinterpret_cast<double*>(sp);                // [nt][threads], then partial sums
  sp += (size_t)2 * nt * kGenThreads * sizeof(double);
  int32_t* sbase = reinterpret_cast<int32_t*>(sp);              // [warps][4 segments][kGenMaxComp]
  sp += kGenWarps * (32 / kGenSeg) * kGenMaxComp * sizeof(int32_t);
  int32_t* cch = reinterpret_cast<int32_t*>(sp);                // [threads]: per lane
  sp += kGenThreads * sizeof(int32_t);
  int32_t* xs = reinterpret_cast<int32_t*>(sp);                 // [nc][threads]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int stride = blockDim.x;
  const int b = (int)blockIdx.x;
  // units: warp nodes (one per warp), group nodes (four per warp), thread nodes
  const int kind = b < a.warp_blocks ? 0 : (b < a.warp_blocks + a.group_blocks ? 1 : 2);
  const int sl = kind == 0 ? lane : (kind == 1 ? (lane & (kGenSeg - 1)) : 0);
  const int sb = kind == 1 ? (lane & ~(kGenSeg - 1)) : 0;
  int v = -1;
  if (kind == 0) {
    const int u = b * kGenWarps + warp;
    if (u < a.n_big) v = a.order[u];
  } else if (kind == 1) {
    const int g = ((b - a.warp_blocks) * kGenWarps + warp) * (32 / kGenSeg) + (lane / kGenSeg);
    if (g < a.n_mid) v = a.order[a.n_big + g];
  } else {
    const int i = a.n_big + a.n_mid + (b - a.warp_blocks - a.group_blocks) * kGenThreads + (int)threadIdx.x;
    if (i < N) v = a.order[i];
  }
  const bool coop = kind != 2;
  // a cooperative warp runs when any of its segments has a node; a thread when it has one
  const bool run = coop ? __any_sync(0xffffffffu, v >= 0) : v >= 0;
  uint32_t fired = 0;
  if (run) {
    const bool has = v >= 0;
    int32_t* x = xs + threadIdx.x;
    int32_t* base = sbase + (warp * (32 / kGenSeg) + (kind == 1 ? lane / kGenSeg : 0)) * kGenMaxComp;
    const RateRow R{rates + threadIdx.x, rates + (size_t)nt * kGenThreads + threadIdx.x, kGenThreads};
    int32_t* X = a.counts + (size_t)r * nc * N;
    if (coop) {
      if (has)
        for (int c = sl; c < nc; c += (kind == 0 ? 32 : kGenSeg)) base[c] = X[(size_t)c * N + v];
      __syncwarp();
    } else {
      for (int c = 0; c < nc; ++c) x[c * stride] = X[(size_t)c * N + v];
    }
    // the node's counts at the start of the day, as this lane sees them
    const int32_t* x0 = coop ? base : x;
    const int s0 = coop ? 1 : stride;
    double y[kGenMaxCont];
    double* Y = a.y + (size_t)r * ny * N;
    const bool writer = has && (!coop || sl == 0);
    if (has) {
      for (int q = 0; q < ny; ++q) y[q] = Y[(size_t)q * N + v];
      if (a.prologue) {
        // day - 1's continuous update from its post-event counts (and, for the
        // midpoint, the sums saved at its start), then frozen for this day
        for (int q = 0; q < ny; ++q) {
          double U = u2d_exact(mask_sum(x0, s0, m.num[q], nc));
          double D = u2d_exact(mask_sum(x0, s0, m.den[q], nc));
          if (m.y_source == kGenYMidpoint) {
            const double* M = a.mid + ((size_t)r * ny + q) * 2 * N;
            U = __dmul_rn(0.5, __dadd_rn(M[v], U));
            D = __dmul_rn(0.5, __dadd_rn(M[(size_t)N + v], D));
          }
          y[q] = gen_y_next(m, p, q, a.day - 1, y[q], U, D);
        }
      }
    }
    if (coop) __syncwarp();
    if (writer) {
      if (a.prologue)
        for (int q = 0; q < ny; ++q) Y[(size_t)q * N + v] = y[q];
      if (m.y_source == kGenYMidpoint)
        for (int q = 0; q < ny; ++q) {
          double* M = a.mid + ((size_t)r * ny + q) * 2 * N;
          M[v] = u2d_exact(mask_sum(x0, s0, m.num[q], nc));
          M[(size_t)N + v] = u2d_exact(mask_sum(x0, s0, m.den[q], nc));
        }
    }
    const uint32_t rep = (uint32_t)(a.rep_base + r), k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint32_t vv = (uint32_t)(has ? v : 0);
    if (coop) {
      // the binary32 segment method first; segments it hands back rerun with the
      // binary64 one from the day's start (the global counts are the day's start
      // until the writer stores below)
      int32_t f = -2;
      if (a.clock_margin)
        f = kind == 0 ? gen_seg_node_day_spec<32>(m, p, x, base, stride, R, y, vv, (uint32_t)a.day, rep, k0, k1,
                                                  sl, sb, has, a.clock_margin)
                      : gen_seg_node_day_spec<kGenSeg>(m, p, x, base, stride, R, y, vv, (uint32_t)a.day, rep, k0,
                                                       k1, sl, sb, has, a.clock_margin);
      const bool redo = has && f < 0;
      if (redo)
        for (int c = sl; c < nc; c += (kind == 0 ? 32 : kGenSeg)) base[c] = X[(size_t)c * N + v];
      __syncwarp();
      uint32_t g = 0;
      if (__any_sync(0xffffffffu, redo)) {
        if (kind == 0)
          g = gen_seg_node_day<32>(m, p, x, base, stride, R, ctau + warp * 32, cch + warp * 32, y, vv,
                                   (uint32_t)a.day, rep, k0, k1, sl, sb, redo);
        else
          g = gen_seg_node_day<kGenSeg>(m, p, x, base, stride, R, ctau + warp * 32 + sb, cch + warp * 32 + sb,
                                        y, vv, (uint32_t)a.day, rep, k0, k1, sl, sb, redo);
      }
      fired = redo ? g : (uint32_t)(f > 0 ? f : 0);
    } else {
      int32_t f = -2;
      if (a.clock_margin) {
        f = gen_node_day_spec(m, p, x, stride, R, y, (uint32_t)v, (uint32_t)a.day, rep, k0, k1, a.clock_margin);
        if (f == -1)                               // too close to call: rerun from the day's start
          for (int c = 0; c < nc; ++c) x[c * stride] = X[(size_t)c * N + v];
      }
      fired = f >= 0 ? (uint32_t)f : gen_node_day(m, p, x, stride, R, y, (uint32_t)v, (uint32_t)a.day, rep, k0, k1);
    }
    if (writer) {
      for (int c = 0; c < nc; ++c) X[(size_t)c * N + v] = x0[c * s0];
      if (m.y_source == kGenYPreEvent) {
        for (int q = 0; q < ny; ++q) {
          const double U = u2d_exact(mask_sum(x0, s0, m.num[q], nc));
          const double D = u2d_exact(mask_sum(x0, s0, m.den[q], nc));
          Y[(size_t)q * N + v] = gen_y_next(m, p, q, a.day, y[q], U, D);
        }
      }
    }
    if (coop && !writer) fired = 0;
  }
  const uint32_t tot = __reduce_add_sync(0xffffffffu, fired);
  if (lane == 0 && tot) atomicAdd(a.ctr + (size_t)r * 4, (unsigned long long)tot);
}

// One thread per component of the day's transfer graph: its events in input
// order (no other thread touches its nodes this day).  Components (largest first)
// are dealt lane-major over the grid's warps: component i runs on lane i / W of
// warp i mod W (W warps in all), so the largest W each have a warp to themselves
// and no warp serialises several long divergent chains.  The counts of the node an
// event samples from stay in a shared-memory row across consecutive events at
// that node; transfers add to the destination in global memory (a destination is
// never the node in the row, and the row is written back before another node is
// loaded).
__global__ void __launch_bounds__(kGenThreads) k_gen_events(GenEvArgs a) {
  __shared__ GenModelDev m;
  __shared__ int32_t cache[kGenMaxComp * kGenThreads];
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  __syncthreads();
  const int r = blockIdx.y, nc = m.nc, N = a.N;
  const int W = (int)gridDim.x * (int)(blockDim.x >> 5);
  const int ci = (int)(threadIdx.x & 31) * W + (int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
  int32_t* cc = cache + threadIdx.x;
  const int S = kGenThreads;
  uint32_t applied = 0, clamped = 0, skipped = 0;
  if (ci < a.ncomp) {
    int32_t* X = a.counts + (size_t)r * nc * N;
    const uint32_t rep = (uint32_t)(a.rep_base + r), k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    int cur = -1;
    const int p1 = a.comp_off[a.comp0 + ci + 1];
    int pi = a.comp_off[a.comp0 + ci];
    int e_next = 0;
    int4 rec_next = make_int4(0, 0, 0, 0);
    if (pi < p1) { e_next = __ldg(a.comp_ev + pi); rec_next = __ldg(a.rec + pi); }
    for (; pi < p1; ++pi) {
      const int e = e_next;
      const int4 rec = rec_next;
      if (pi + 1 < p1) { e_next = __ldg(a.comp_ev + pi + 1); rec_next = __ldg(a.rec + pi + 1); }
      const int node = rec.x, dest = rec.y, n = rec.z;
      const int kind = rec.w & 0xff, sel = (rec.w >> 8) & 0xff, sh = (rec.w >> 16) & 0xff;
      const uint32_t mask = m.select[sel];
      const int8_t* off = m.shift[sh];
      if (node != cur) {
        if (cur >= 0)
          for (int c = 0; c < nc; ++c) X[(size_t)c * N + cur] = cc[c * S];
        for (int c = 0; c < nc; ++c) cc[c * S] = X[(size_t)c * N + node];
        cur = node;
      }
      if (kind == SIM_ENTER) {
        const int c0 = __ffs(mask) - 1;
        cc[(c0 + off[c0]) * S] += n;
        ++applied;
        continue;
      }
      long long avail = 0;
      for (int c = 0; c < nc; ++c)
        if (mask >> c & 1u) avail += cc[c * S];
      int take = n;
      if ((long long)n > avail) {
        if (a.underflow_error) {
          ++skipped;
          atomicOr(a.err, 1);
          continue;
        }
        take = (int)avail;
        ++clamped;
      }
      uint4 buf = make_uint4(0, 0, 0, 0);
      uint32_t wq = 0;
      auto next = [&]() -> uint32_t {
        if ((wq & 3u) == 0u) buf = philox10(make_uint4((uint32_t)e, (uint32_t)a.day | kEventTag, wq >> 2, rep), k0, k1);
        const uint32_t s = wq & 3u;
        ++wq;
        return s == 0 ? buf.x : s == 1 ? buf.y : s == 2 ? buf.z : buf.w;
      };
      for (int t = 0; t < take; ++t) {
        uint32_t slot = lemire((uint32_t)(avail - t), next);
        int got = 0;
        for (int c = 0; c < nc; ++c) {
          if (!(mask >> c & 1u)) continue;
          const uint32_t have = (uint32_t)cc[c * S];
          if (slot < have) { got = c; break; }
          slot -= have;
        }
        cc[got * S] -= 1;
        if (kind == SIM_INTERNAL) cc[(got + off[got]) * S] += 1;
        else if (kind == SIM_EXTERNAL) X[(size_t)(got + off[got]) * N + dest] += 1;
      }
      ++applied;
    }
    if (cur >= 0)
      for (int c = 0; c < nc; ++c) X[(size_t)c * N + cur] = cc[c * S];
  }
  const uint32_t sa = __reduce_add_sync(0xffffffffu, applied);
  const uint32_t sc = __reduce_add_sync(0xffffffffu, clamped);
  const uint32_t ss = __reduce_add_sync(0xffffffffu, skipped);
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* C = a.ctr + (size_t)r * 4;
    if (sa) atomicAdd(C + 1, (unsigned long long)sa);
    if (sc) atomicAdd(C + 2, (unsigned long long)sc);
    if (ss) atomicAdd(C + 3, (unsigned long long)ss);
  }
}

// Continuous update of a run's last day from the post-event counts, or the
// midpoint with the sums the stochastic step saved (earlier days' updates run in
// the next day's stochastic-step prologue).
__global__ void __launch_bounds__(kGenThreads) k_gen_cont(GenContArgs a) {
  __shared__ GenModelDev m;
  __shared__ GenRepParams p;
  const int r = blockIdx.y;
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  copy16(&p, a.params + r, (int)(sizeof(GenRepParams) / 16));
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x, N = a.N, nc = m.nc, ny = m.ny;
  if (v >= N) return;
  const int32_t* X = a.counts + (size_t)r * nc * N + v;
  double* Y = a.y + (size_t)r * ny * N + v;
  for (int q = 0; q < ny; ++q) {
    double U = u2d_exact(mask_sum(X, N, m.num[q], nc));
    double D = u2d_exact(mask_sum(X, N, m.den[q], nc));
    if (m.y_source == kGenYMidpoint) {
      const double* M = a.mid + ((size_t)r * ny + q) * 2 * N + v;
      U = __dmul_rn(0.5, __dadd_rn(M[0], U));
      D = __dmul_rn(0.5, __dadd_rn(M[N], D));
    }
    Y[(size_t)q * N] = gen_y_next(m, p, q, a.day, Y[(size_t)q * N], U, D);
  }
}

}  // namespace

size_t gen_ssa_smem_bytes(int nc, int nt) {
  return sizeof(GenModelDev) + sizeof(GenRepParams) + kGenThreads * sizeof(double) +
         (size_t)2 * nt * kGenThreads * sizeof(double) +
         (size_t)(kGenThreads / 32) * (32 / 8) * kGenMaxComp * sizeof(int32_t) + kGenThreads * sizeof(int32_t) +
         (size_t)nc * kGenThreads * sizeof(int32_t);
}

cudaError_t launch_gen_ssa(GenSsaArgs a, int nt, int nc, cudaStream_t st) {
  a.warp_blocks = (a.n_big + kGenWarps - 1) / kGenWarps;
  const int per_block = kGenWarps * (32 / kGenSeg);
  a.group_blocks = (a.n_mid + per_block - 1) / per_block;
  const int rest = a.N - a.n_big - a.n_mid;
  const dim3 grid((unsigned)(a.warp_blocks + a.group_blocks + (rest + kGenThreads - 1) / kGenThreads), (unsigned)a.R);
  const size_t smem = gen_ssa_smem_bytes(nc, nt);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_gen_ssa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gen_ssa<<<grid, kGenThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gen_events(const GenEvArgs& a, cudaStream_t st) {
  if (a.ncomp <= 0) return cudaSuccess;
  // a warp per component up to kGenEventWarps warps, then up to 32 per warp
  const int warps = std::max((a.ncomp + 31) / 32, std::min(a.ncomp, kGenEventWarps));
  const dim3 grid((unsigned)((warps + kGenWarps - 1) / kGenWarps), (unsigned)a.R);
  k_gen_events<<<grid, kGenThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gen_cont(const GenContArgs& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + kGenThreads - 1) / kGenThreads), (unsigned)a.R);
  k_gen_cont<<<grid, kGenThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace episim
