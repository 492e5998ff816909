// Deterministic step (Eq. (numstep4); Sec. 3.3 "read and incorporate"; Alg. 1
// line 13): the day's scheduled events (Sec. 3.2, Eq. (event)) applied level by
// level.  The host assigns levels so that, within a level, no two events sample
// the same node and no node is both sampled and added to; adds that share a node
// commute and use integer atomics.  The result equals applying the events one
// by one in their input order (scheduling rule 2(b) of Sec. 3.6 applied per node).
//
// One block per replicate; its threads take a level's events in parallel, with a
// block barrier between levels.  Removed animals are drawn without replacement,
// uniformly over the selected compartments, one at a time (Lemire's bounded
// integers on the event's own Philox word stream).
#include "internal.h"
#include "devmath.cuh"

namespace episim {

namespace {

struct WordStream {
  uint4 ctr;
  uint32_t k0, k1;
  uint4 buf;
  uint32_t q;
  __device__ uint32_t operator()() {
    if ((q & 3u) == 0u) { ctr.z = q >> 2; buf = philox10(ctr, k0, k1); }
    uint32_t sel = q & 3u;
    ++q;
    return sel == 0 ? buf.x : sel == 1 ? buf.y : sel == 2 ? buf.z : buf.w;
  }
};

template <int NA>
__device__ __forceinline__ void apply_event(const EvArgs& a, int32_t* X, int r, int4 rec,
                                            unsigned& applied, unsigned& clamped, unsigned& skipped) {
  const int N = a.N;
  const int node = rec.x, dest = rec.y, e = rec.z;
  const int kind = rec.w & 3;
  const int cls = ((rec.w >> 2) & 3) - 1;
  const int32_t n = (int32_t)((uint32_t)rec.w >> 4);
  if (kind == 1) {  // enter: susceptible animals of class cls (class 0 for -1)
    const int j = cls < 0 ? 0 : cls;
    atomicAdd(&X[(size_t)(2 * j) * N + node], n);
    ++applied;
    return;
  }
  // selected compartments: both states of class cls, or every compartment
  const int c_lo = cls < 0 ? 0 : 2 * cls;
  const int c_hi = cls < 0 ? 2 * NA : 2 * cls + 2;
  int32_t have[2 * NA];
  int32_t took[2 * NA];
  int64_t avail = 0;
#pragma unroll
  for (int c = 0; c < 2 * NA; ++c) {
    have[c] = (c >= c_lo && c < c_hi) ? X[(size_t)c * N + node] : 0;
    took[c] = 0;
    avail += have[c];
  }
  int32_t take = n;
  if ((int64_t)n > avail) {
    if (a.underflow_error) {
      ++skipped;
      atomicOr(a.err, 1);
      return;
    }
    take = (int32_t)avail;
    ++clamped;
  }
  WordStream ws;
  ws.ctr = make_uint4((uint32_t)e, (uint32_t)a.day | kEventTag, 0u, (uint32_t)r);
  ws.k0 = (uint32_t)a.seed;
  ws.k1 = (uint32_t)(a.seed >> 32);
  ws.q = 0;
  for (int32_t t = 0; t < take; ++t) {
    uint32_t slot = lemire((uint32_t)(avail - t), ws);
    bool done = false;
#pragma unroll
    for (int c = 0; c < 2 * NA; ++c) {
      if (!done) {
        if (slot < (uint32_t)have[c]) { have[c] -= 1; took[c] += 1; done = true; }
        else slot -= (uint32_t)have[c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2 * NA; ++c) {
    if (c >= c_lo && c < c_hi) X[(size_t)c * N + node] = have[c];
  }
  if (kind == 2) {  // aging: same state, next class of the same node
#pragma unroll
    for (int c = 0; c + 2 < 2 * NA; ++c)
      if (took[c]) X[(size_t)(c + 2) * N + node] += took[c];
  } else if (kind == 3) {  // external transfer to dest
#pragma unroll
    for (int c = 0; c < 2 * NA; ++c)
      if (took[c]) atomicAdd(&X[(size_t)c * N + dest], took[c]);
  }
  ++applied;
}

template <int NA>
__global__ void __launch_bounds__(512) k_events_day(EvArgs a) {
  const int r = blockIdx.x;
  int32_t* X = a.counts + (size_t)r * a.Nc * a.N;
  const int l0 = a.day_lvl[a.day], l1 = a.day_lvl[a.day + 1];
  unsigned applied = 0, clamped = 0, skipped = 0;
  for (int l = l0; l < l1; ++l) {
    const int b = a.lvl_start[l], end = a.lvl_start[l + 1];
    for (int q = b + (int)threadIdx.x; q < end; q += blockDim.x)
      apply_event<NA>(a, X, r, a.rec[q], applied, clamped, skipped);
    __syncthreads();
  }
  // counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    applied += __shfl_down_sync(0xffffffffu, applied, o);
    clamped += __shfl_down_sync(0xffffffffu, clamped, o);
    skipped += __shfl_down_sync(0xffffffffu, skipped, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* c = a.ctr + (size_t)r * 4;
    if (applied) atomicAdd(c + 1, (unsigned long long)applied);
    if (clamped) atomicAdd(c + 2, (unsigned long long)clamped);
    if (skipped) atomicAdd(c + 3, (unsigned long long)skipped);
  }
}

}  // namespace

cudaError_t launch_events_day(const EvArgs& a, int n_age, cudaStream_t st) {
  if (n_age == 1) k_events_day<1><<<a.R, 512, 0, st>>>(a);
  else k_events_day<3><<<a.R, 512, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace episim
