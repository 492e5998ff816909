// Dataflow day loop (SIM_LAUNCH_FLOW): one persistent kernel runs a whole call's
// days with no per-day barrier.
//
// The stochastic step and the phi update of a herd (Eqs. (numstep3), (numstep5))
// read only that herd, and only the day's events couple herds, within a connected
// component of the day's transfer graph (Sec. 3.4: the paper's own parallel
// algorithm also runs a node's stochastic steps as soon as its inputs are ready,
// as tasks; Alg. 2).  So a herd the day's events leave untouched can start its
// next day as soon as its own day is done, and a component's events can run as
// soon as its herds' stochastic steps are.  Work items, fetched by warps from one
// counter in a fixed order: for each day, the stochastic-step units of the dealt
// mapping (one warp-path herd, four group-path herds or 32 thread-path herds of
// one replicate; heaviest first), then the transfer-graph components of at least
// kFlowLong events (one per warp, longest first: the lanes compute the events'
// random words in parallel, one lane applies them in input order), then groups
// of 32 shorter components of one replicate (one per lane).  Each stochastic-step
// unit (its herds are the same every day) has a completion counter per replicate,
// incremented once by the unit's stochastic step of each day and once by each
// component that touches its herds.  The unit's step of day d waits until the
// counter shows its own earlier days and every earlier component on its herds
// (the host's cumulative per-unit table K gives that count); a component of day d
// waits until each of its units shows its day-d step, applies its events in input
// order (the result of the sequential list, since no other event of the day
// touches those herds) and increments them.  One lane polls one word per unit,
// which keeps the polling traffic far below the memory traffic of the work.  Every wait
// points to an earlier item and a warp fetches an item only while it runs, so the
// earliest unfinished item can always proceed: no co-residency is assumed.  Waits
// are bounded; running out sets the event-wait error bit and an abort flag that
// every warp checks, and the kernel returns.  The results are those of the
// per-day kernels bit for bit (counter-based random numbers keyed by node, day and
// event position; integer statistics).
#include <algorithm>

#include "events_device.cuh"
#include "ssa_device.cuh"

namespace episim {

namespace {

__device__ __forceinline__ int flow_ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned flow_ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *p >= target; false when the wait ran out or the run was aborted.
// Polls with relaxed loads, backing off from 32 to 256 ns, and makes one acquire
// fence once the value is seen.
__device__ bool flow_wait(const unsigned* p, unsigned target, const FlowArgs& f) {
  if (flow_ld_relaxed_u32(p) >= target) {
    __threadfence();
    return true;
  }
  unsigned ns = 32;
  for (long long it = 0; it < f.spin_limit; ++it) {
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
    if (flow_ld_relaxed_u32(p) >= target) {
      __threadfence();
      return true;
    }
    if ((it & 15) == 0 && flow_ld_relaxed(f.abort)) return false;
  }
  atomicOr(f.a.err_word, kEventWaitTimeout);
  atomicExch(f.abort, 1);
  return false;
}

// Completions unit u1 of replicate r must show before its stochastic step of day d
// (after = 0) may start, or before the events of day d on its herds (after = 1):
// one per earlier day of the call for its own stochastic step, one per earlier
// component that touched its herds, and (after = 1) its day-d stochastic step.
__device__ __forceinline__ unsigned flow_target(const FlowArgs& f, int d, int u1, int after) {
  return (unsigned)(d - f.d0 + after) + (unsigned)(__ldg(f.K + (size_t)d * f.U1 + u1) - __ldg(f.K + (size_t)f.d0 * f.U1 + u1));
}

// The stochastic step of unit u of day d (the dealt decomposition of one day).
template <int NA>
__device__ __forceinline__ bool flow_ssa_unit(const FlowArgs& f, int d, int64_t u) {
  const SsaArgs& a0 = f.a.ssa;
  const int lane = threadIdx.x & 31;
  const int64_t R = a0.R;
  const int64_t uw = R * a0.n_big;
  const int64_t ug = R * ((a0.n_mid + 3) / 4);
  int r = 0, v = 0, role = kRoleThread, u1 = 0;
  bool active = false;
  if (u < uw) {
    r = (int)(u % R);
    u1 = (int)(u / R);
    v = a0.order[u1];
    active = true;
    role = kRoleWarp;
  } else if (u < uw + ug) {
    const int64_t ut = u - uw;
    r = (int)(ut % R);
    u1 = a0.n_big + (int)(ut / R);
    const int64_t i = a0.n_big + (ut / R) * 4 + (lane / kGroupLanes);
    active = i < a0.n_big + a0.n_mid;
    v = active ? a0.order[i] : 0;
    role = kRoleGroup;
  } else {
    const int64_t ut = u - uw - ug;
    r = (int)(ut % R);
    u1 = a0.n_big + (a0.n_mid + 3) / 4 + (int)(ut / R);
    const int64_t i = a0.n_big + a0.n_mid + (ut / R) * 32 + lane;
    active = i < a0.n_list;
    v = active ? a0.order[i] : 0;
  }
  unsigned* cnt = f.unit_cnt + (size_t)r * f.U1 + u1;
  bool ok = true;
  if (lane == 0)
    ok = flow_wait(cnt, flow_target(f, d, u1, 0) + ((r == 0 && u1 == 0 && d == f.d0) ? f.stall_extra : 0u), f);
  if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
  __syncwarp();
  SsaArgs a = a0;
  a.day = d;
  a.prologue = d > f.d0;
  node_day_work<NA, false, 0>(a, r, v, active, role);
  __threadfence();
  __syncwarp();
  if (lane == 0) atomicAdd(cnt, 1u);
  return true;
}

// Waits, with the calling lanes spread over the component's units, until its
// herds' stochastic steps of day d are done.
__device__ __forceinline__ bool flow_wait_units(const FlowArgs& f, int d, int r, int c, int j0, int step) {
  const int u0 = f.cuoff[c], u1e = f.cuoff[c + 1];
  bool ok = true;
  for (int j = u0 + j0; j < u1e && ok; j += step) {
    const int u = f.cunit[j];
    ok = flow_wait(f.unit_cnt + (size_t)r * f.U1 + u, flow_target(f, d, u, 1), f);
  }
  return ok;
}

__device__ __forceinline__ void flow_release_units(const FlowArgs& f, int r, int c, int j0, int step) {
  for (int j = f.cuoff[c] + j0; j < f.cuoff[c + 1]; j += step) atomicAdd(f.unit_cnt + (size_t)r * f.U1 + f.cunit[j], 1u);
}

// A long component c of day d for replicate r, on a whole warp: its herds are
// staged in the warp's shared-memory slots (the 32 lanes' regions are contiguous:
// up to 32 x kFlowSlots herds); the lanes compute the Philox blocks of 32 events
// at a time and lane 0 applies the events in input order with each event's words
// shuffled to it.
template <int NA>
__device__ __forceinline__ bool flow_long_component(const FlowArgs& f, int d, int r, int c, int32_t* cnt0) {
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  const EvArgs& ev = f.a.ev;
  const int n0 = f.cnoff[c], n1 = f.cnoff[c + 1];
  const int k = n1 - n0;
  if (!__all_sync(0xffffffffu, flow_wait_units(f, d, r, c, lane, 32))) return false;
  __syncwarp();
  int32_t* X = ev.counts + (size_t)r * NC * ev.N;
  const uint32_t rep = (uint32_t)(ev.rep_base + r);
  const uint32_t k0 = (uint32_t)ev.seed, k1 = (uint32_t)(ev.seed >> 32);
  const int q0 = f.cev[c], q1 = f.cev[c + 1];
  unsigned applied = 0, clamped = 0, skipped = 0;
  if (k <= 32 * kFlowSlots) {
    for (int sl = lane; sl < k; sl += 32) {
      const int v = f.cnode[n0 + sl];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) cnt0[sl * NC + cc] = __ldcg(X + (size_t)cc * ev.N + v);
    }
    __syncwarp();
    for (int qb = q0; qb < q1; qb += 32) {
      const int q = qb + lane;
      int4 rc = make_int4(0, 0, 0, 0);
      Words8 wd;
      wd.a = make_uint4(0u, 0u, 0u, 0u);
      wd.b = wd.a;
      if (q < q1) {
        rc = f.rec[q];
        if ((rc.w & 3) != 1) {
          wd.a = philox10(make_uint4((uint32_t)rc.z, (uint32_t)d | kEventTag, 0u, rep), k0, k1);
          wd.b = philox10(make_uint4((uint32_t)rc.z, (uint32_t)d | kEventTag, 1u, rep), k0, k1);
        }
      }
      const int m = min(32, q1 - qb);
      for (int j = 0; j < m; ++j) {
        int4 r4;
        Words8 w8;
        r4.x = __shfl_sync(0xffffffffu, rc.x, j); r4.y = __shfl_sync(0xffffffffu, rc.y, j);
        r4.z = __shfl_sync(0xffffffffu, rc.z, j); r4.w = __shfl_sync(0xffffffffu, rc.w, j);
        w8.a.x = __shfl_sync(0xffffffffu, wd.a.x, j); w8.a.y = __shfl_sync(0xffffffffu, wd.a.y, j);
        w8.a.z = __shfl_sync(0xffffffffu, wd.a.z, j); w8.a.w = __shfl_sync(0xffffffffu, wd.a.w, j);
        w8.b.x = __shfl_sync(0xffffffffu, wd.b.x, j); w8.b.y = __shfl_sync(0xffffffffu, wd.b.y, j);
        w8.b.z = __shfl_sync(0xffffffffu, wd.b.z, j); w8.b.w = __shfl_sync(0xffffffffu, wd.b.w, j);
        if (lane == 0)
          apply_event_smem<NA, false>(ev.underflow_error, ev.err, d, ev.seed, cnt0, rep, r4, w8, applied, clamped,
                                      skipped);
      }
    }
    __syncwarp();
    for (int sl = lane; sl < k; sl += 32) {
      const int v = f.cnode[n0 + sl];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) X[(size_t)cc * ev.N + v] = cnt0[sl * NC + cc];
    }
  } else if (lane == 0) {
    // more herds than the warp's slots: the events straight on the global counts
    EvArgs e = ev;
    e.day = d;
    for (int q = q0; q < q1; ++q) {
      int4 rc = f.rec[q];
      rc.x = f.cnode[n0 + rc.x];
      if ((rc.w & 3) == 3) rc.y = f.cnode[n0 + rc.y];
      apply_event<NA>(e, X, r, rc, applied, clamped, skipped);
    }
  }
  __threadfence();
  __syncwarp();
  flow_release_units(f, r, c, lane, 32);
  if (lane == 0) {
    unsigned long long* ct = ev.ctr + (size_t)r * 4;
    if (applied) atomicAdd(ct + 1, (unsigned long long)applied);
    if (clamped) atomicAdd(ct + 2, (unsigned long long)clamped);
    if (skipped) atomicAdd(ct + 3, (unsigned long long)skipped);
  }
  return true;
}

// Group g (of 32 short components, one per lane) of day d for replicate r.
template <int NA>
__device__ __forceinline__ bool flow_components(const FlowArgs& f, int d, int r, int g, int32_t* cnt) {
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  const EvArgs& ev = f.a.ev;
  const int c0 = f.day_comp[d] + f.day_long[d], c1 = f.day_comp[d + 1];
  const int c = c0 + g * 32 + lane;
  unsigned applied = 0, clamped = 0, skipped = 0;
  bool ok = true;
  if (c < c1) {
    ok = flow_wait_units(f, d, r, c, 0, 1);
    if (ok) {
      const int n0 = f.cnoff[c], n1 = f.cnoff[c + 1];
      int32_t* X = ev.counts + (size_t)r * NC * ev.N;
      const uint32_t rep = (uint32_t)(ev.rep_base + r);
      const uint32_t k0 = (uint32_t)ev.seed, k1 = (uint32_t)(ev.seed >> 32);
      const int q0 = f.cev[c], q1 = f.cev[c + 1];
      const int k = n1 - n0;
      if (k <= kFlowSlots) {
        // the component's herds staged in this lane's slots; no other thread
        // touches them until this lane releases them
        for (int s = 0; s < k; ++s) {
          const int v = f.cnode[n0 + s];
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) cnt[s * NC + cc] = __ldcg(X + (size_t)cc * ev.N + v);
        }
        int4 rc = f.rec[q0];
        Words8 wd;
        wd.a = philox10(make_uint4((uint32_t)rc.z, (uint32_t)d | kEventTag, 0u, rep), k0, k1);
        wd.b = philox10(make_uint4((uint32_t)rc.z, (uint32_t)d | kEventTag, 1u, rep), k0, k1);
        for (int q = q0; q < q1; ++q) {
          // the next record and its first Philox blocks in flight while this one is applied
          int4 nrc = rc;
          Words8 nwd = wd;
          if (q + 1 < q1) {
            nrc = f.rec[q + 1];
            nwd.a = philox10(make_uint4((uint32_t)nrc.z, (uint32_t)d | kEventTag, 0u, rep), k0, k1);
            nwd.b = philox10(make_uint4((uint32_t)nrc.z, (uint32_t)d | kEventTag, 1u, rep), k0, k1);
          }
          apply_event_smem<NA, false>(ev.underflow_error, ev.err, d, ev.seed, cnt, rep, rc, wd, applied, clamped,
                                      skipped);
          rc = nrc;
          wd = nwd;
        }
        for (int s = 0; s < k; ++s) {
          const int v = f.cnode[n0 + s];
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) X[(size_t)cc * ev.N + v] = cnt[s * NC + cc];
        }
      } else {
        // a large component: its events straight on the global counts
        EvArgs e = ev;
        e.day = d;
        for (int q = q0; q < q1; ++q) {
          int4 rc = f.rec[q];
          rc.x = f.cnode[n0 + rc.x];
          if ((rc.w & 3) == 3) rc.y = f.cnode[n0 + rc.y];
          apply_event<NA>(e, X, r, rc, applied, clamped, skipped);
        }
      }
      __threadfence();
      flow_release_units(f, r, c, 0, 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    applied += __shfl_down_sync(0xffffffffu, applied, o);
    clamped += __shfl_down_sync(0xffffffffu, clamped, o);
    skipped += __shfl_down_sync(0xffffffffu, skipped, o);
  }
  if (lane == 0) {
    unsigned long long* ct = ev.ctr + (size_t)r * 4;
    if (applied) atomicAdd(ct + 1, (unsigned long long)applied);
    if (clamped) atomicAdd(ct + 2, (unsigned long long)clamped);
    if (skipped) atomicAdd(ct + 3, (unsigned long long)skipped);
  }
  return __all_sync(0xffffffffu, ok);
}

template <int NA>
__global__ void __launch_bounds__(kFlowThreads, 2) k_flow(FlowArgs f) {
  extern __shared__ __align__(16) int32_t flow_smem[];
  constexpr int NC = 2 * NA;
  const int lane = threadIdx.x & 31;
  int32_t* cnt = flow_smem + (size_t)threadIdx.x * kFlowSlots * NC;
  int32_t* cnt0 = flow_smem + (size_t)(threadIdx.x & ~31) * kFlowSlots * NC;   // lane 0's slots
  const long long total = f.item_off[f.ndays];
  for (;;) {
    unsigned long long it = 0;
    int stop = 0;
    if (lane == 0) {
      it = atomicAdd(f.next, 1ull);
      stop = (long long)it >= total || flow_ld_relaxed(f.abort);
    }
    it = __shfl_sync(0xffffffffu, it, 0);
    if (__shfl_sync(0xffffffffu, stop, 0)) break;
    // the item's day: the largest k with item_off[k] <= it
    int lo = 0, hi = f.ndays - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (f.item_off[mid] <= (long long)it) lo = mid; else hi = mid - 1;
    }
    const int d = f.d0 + lo;
    const long long local = (long long)it - f.item_off[lo];
    bool ok;
    if (local < f.units) {
      ok = flow_ssa_unit<NA>(f, d, local);
    } else {
      const int nlong = f.day_long[d];
      const long long cl = local - f.units;
      const long long R = f.a.ssa.R;
      if (cl < R * nlong) {
        ok = flow_long_component<NA>(f, d, (int)(cl / nlong), f.day_comp[d] + (int)(cl % nlong), cnt0);
      } else {
        const long long cs = cl - R * nlong;
        const int groups = (f.day_comp[d + 1] - f.day_comp[d] - nlong + 31) / 32;
        ok = flow_components<NA>(f, d, (int)(cs / groups), (int)(cs % groups), cnt);
      }
    }
    if (!ok) break;
  }
}

template <int NA>
cudaError_t launch_flow_impl(const FlowArgs& f, int sms, cudaStream_t st) {
  const size_t smem = (size_t)kFlowThreads * kFlowSlots * 2 * NA * sizeof(int32_t);
  static bool attr = false;
  static int per_sm = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_flow<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flow<NA>, kFlowThreads, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  k_flow<NA><<<grid, kFlowThreads, smem, st>>>(f);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flow(const FlowArgs& f, int n_age, int sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(f.unit_cnt, 0, (size_t)f.a.ssa.R * f.U1 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.next, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.abort, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return n_age == 1 ? launch_flow_impl<1>(f, sms, st) : launch_flow_impl<3>(f, sms, st);
}

}  // namespace episim
