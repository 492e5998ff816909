// Persistent work-stealing kernel (template) for batched and uneven runs: several
// simulations (handles, each with its model, nodes, replicates, horizon, events
// and parameters) advance together in one launch.
//
// Work items, in a fixed global order that every block fetches from one atomic
// counter: for each step s (day day0 + s of every instance still running), first
// the stochastic-step chunks of every (instance, replicate) -- a chunk is
// kBatchSubs blocks' worth of nodes with one thread each, or one large herd per
// warp -- then the event item of every (instance, replicate); after the last
// step, finalisation chunks (phi update and statistics of each instance's last
// day).  A chunk of day d waits until the events of day d-1 of its replicate are
// applied; an event item waits until every chunk of its day is done.
// Dependencies always point to earlier items, and a block fetches an item only
// while it runs, so the earliest unfinished item can always proceed: no
// co-residency assumption is needed.  The items a block fetches only increase,
// so a block decodes each by a galloping search of the step and instance tables
// from its previous item's position.  Waits spin on acquire loads with a bounded
// count (about two seconds); running out sets an error and an abort flag that
// every block checks, and the kernel returns instead of hanging.  State written
// by other blocks is read with L2-coherent loads (see ssa_device.cuh,
// events_device.cuh).
#pragma once
#include "batch.h"
#include "events_device.cuh"
#include "ssa_device.cuh"

namespace episim {

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *p >= target.  Returns false when the wait ran out or the run was aborted.
__device__ bool wait_at_least(const unsigned* p, unsigned target, const BatchCtl& c) {
  if (ld_acquire(p) >= target) return true;
  for (long long it = 0; it < c.spin_limit; ++it) {
    __nanosleep(128);
    if (ld_acquire(p) >= target) return true;
    if (ld_relaxed_int(c.abort)) return false;
  }
  atomicOr(c.err, kBatchTimeout);
  atomicExch(c.abort, 1);
  return false;
}

// Largest k in [lo, n) with cum[k] <= x, for non-decreasing cum and cum[lo] <= x:
// steps of 1, 2, 4, ... from lo, then a binary search within the last step.
__device__ __forceinline__ int upper_index_from(const long long* cum, int n, int lo, long long x) {
  int step = 1;
  while (lo + step < n && cum[lo + step] <= x) {
    lo += step;
    step <<= 1;
  }
  int hi = min(lo + step, n) - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cum[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int upper_index(const long long* cum, int n, long long x) {
  // largest k in [0, n) with cum[k] <= x (cum non-decreasing, cum[0] = 0)
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cum[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int NA, bool SCORE, int MODE>
__device__ __forceinline__ void run_chunk(const BatchInst& I, int r, int chunk, int day, int prologue) {
  SsaArgs a = I.ssa;
  a.day = day;
  a.prologue = prologue;
  const int wb = (MODE == 0 && !SCORE) ? a.warp_blocks : 0;
  if (MODE == 1 || chunk < wb) { node_day_block<NA, SCORE, MODE>(a, r, chunk); return; }
  // A per-thread chunk is I.subs blocks' worth of nodes, run one after another with
  // no barrier between them: a warp's time is then a sum over I.subs nodes a lane,
  // and the block's closing barrier waits on sums that differ less than single
  // node-days do.
  const int q0 = (chunk - wb) * I.subs;
  for (int j = 0; j < I.subs; ++j) {
    if ((q0 + j) * (int)blockDim.x >= I.n_thread) break;
    node_day_block<NA, SCORE, MODE>(a, r, wb + q0 + j);
  }
}

template <bool SCORE_ANY>
__device__ __forceinline__ void dispatch_chunk(const BatchInst& I, int r, int chunk, int day, int prologue, int mode) {
  if (I.na == 1) {
    if (SCORE_ANY && I.score) { if (mode == 0) run_chunk<1, SCORE_ANY, 0>(I, r, chunk, day, prologue); else run_chunk<1, SCORE_ANY, 1>(I, r, chunk, day, prologue); }
    else { if (mode == 0) run_chunk<1, false, 0>(I, r, chunk, day, prologue); else run_chunk<1, false, 1>(I, r, chunk, day, prologue); }
  } else {
    if (SCORE_ANY && I.score) { if (mode == 0) run_chunk<3, SCORE_ANY, 0>(I, r, chunk, day, prologue); else run_chunk<3, SCORE_ANY, 1>(I, r, chunk, day, prologue); }
    else { if (mode == 0) run_chunk<3, false, 0>(I, r, chunk, day, prologue); else run_chunk<3, false, 1>(I, r, chunk, day, prologue); }
  }
}

__device__ __forceinline__ void dispatch_events(const BatchInst& I, int r, int day, unsigned char* smem, int smem_cap) {
  if (!I.has_events) return;
  const int dl0 = __ldg(I.evg.day_lvl + day), dl1 = __ldg(I.evg.day_lvl + day + 1);
  if (dl1 <= dl0) return;
  const int need = __ldg(I.day_smem + day);
  if (need > 0 && need <= smem_cap) {
    EvSmemArgs a = I.evs;
    a.day = day;
    a.smem_bytes = need;
    if (I.na == 1) events_block_smem<1>(a, r, smem); else events_block_smem<3>(a, r, smem);
  } else {
    EvArgs a = I.evg;
    a.day = day;
    if (I.na == 1) events_block_global<1>(a, r); else events_block_global<3>(a, r);
  }
}

// THREADS threads a block, MINB blocks an SM (the register budget), and whether
// any instance computes the score (its stochastic step is compiled in only then).
template <int THREADS, int MINB, bool SCORE_ANY>
__global__ void __launch_bounds__(THREADS, MINB) k_batch(BatchCtl c) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_go;   // written by thread 0 only before the loop-top barrier
  __shared__ int s_ok;   // the item's dependency wait succeeded (its own flag: s_go
                         // may still be being read when the wait's result lands)
  __shared__ int s_hs, s_hk, s_hkind;   // the previous item's step, instance and kind (0 chunk, 1 events)
  if (threadIdx.x == 0) { s_hs = 0; s_hk = 0; s_hkind = -1; }   // read after the loop's first barrier
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)atomicAdd(c.next, 1ull);
      s_go = (s_item < c.total) && !ld_relaxed_int(c.abort);
    }
    __syncthreads();
    const long long t = s_item;
    if (!s_go) break;
    if (t < c.total_main) {
      const int hs = s_hs, hk = s_hk, hkind = s_hkind;
      const int s = upper_index_from(c.step_off, c.n_steps, hs, t);
      const long long local = t - c.step_off[s];
      const int act = c.active[s];
      const long long nA = c.cumA[act];
      int k, r, chunk = 0;
      const bool is_ssa = local < nA;
      if (is_ssa) {
        k = upper_index_from(c.cumA, act, (hs == s && hkind == 0) ? hk : 0, local);
        const long long w = local - c.cumA[k];
        const BatchInst& I0 = c.inst[k];
        r = (int)(w / I0.bpr);
        chunk = (int)(w - (long long)r * I0.bpr);
      } else {
        k = upper_index_from(c.cumB, act, (hs == s && hkind == 1) ? hk : 0, local - nA);
        r = (int)(local - nA - c.cumB[k]);
      }
      const BatchInst& I = c.inst[k];
      const int day = I.day0 + s;
      if (threadIdx.x == 0) s_ok = is_ssa ? wait_at_least(I.ev_done + r, (unsigned)day, c)
                                          : wait_at_least(I.ssa_done + r, (unsigned)((s + 1) * I.bpr), c);
      __syncthreads();
      if (s_ok) {
        if (is_ssa) dispatch_chunk<SCORE_ANY>(I, r, chunk, day, s > 0, 0);
        else dispatch_events(I, r, day, smem, c.smem_cap);
      }
      __syncthreads();
      if (threadIdx.x == 0) { s_hs = s; s_hk = k; s_hkind = is_ssa ? 0 : 1; }   // read after the next barrier
      if (threadIdx.x == 0 && s_ok) {
        __threadfence();
        if (is_ssa) atomicAdd(I.ssa_done + r, 1u);
        else atomicMax(I.ev_done + r, (unsigned)(day + 1));
      }
    } else {
      const long long local = t - c.total_main;
      const int k = upper_index(c.cumF, c.n_inst, local);
      const BatchInst& I = c.inst[k];
      const long long w = local - c.cumF[k];
      const int r = (int)(w / I.tbpr), chunk = (int)(w - (long long)r * I.tbpr);
      const int last = I.day0 + I.ndays - 1;
      if (threadIdx.x == 0) s_ok = wait_at_least(I.ev_done + r, (unsigned)(last + 1), c);
      __syncthreads();
      if (s_ok) dispatch_chunk<SCORE_ANY>(I, r, chunk, last, 1, 1);
    }
    __syncthreads();
  }
}

}  // namespace

// The kernel of one block shape, with or without the score step compiled in; each
// shape is instantiated in a translation unit of its own (batch_shape_*.cu).
template <int THREADS, int MINB>
BatchKernel batch_kernel_of(bool score_any) {
  return score_any ? (BatchKernel)k_batch<THREADS, MINB, true> : (BatchKernel)k_batch<THREADS, MINB, false>;
}

}  // namespace episim
