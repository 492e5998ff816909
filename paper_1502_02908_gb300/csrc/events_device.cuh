// Device code of the deterministic step (Eq. (numstep4); Sec. 3.3; the event
// step of Alg. 1): the day's scheduled events (Sec. 3.2, Eq. (event)) applied in dependency
// levels.  Shared by the per-day kernels (events.cu) and the persistent batch
// kernel (batch.cu).  The host assigns levels so that, within a level, no two
// events sample the same node and no node is both sampled and added to; adds
// that share a node commute and use integer atomics.  The result equals applying
// the events one by one in their input order (scheduling rule 2(b) of Sec. 3.6
// applied per node).  Removed animals are drawn without replacement, uniformly
// over the selected compartments, one at a time (Lemire's bounded integers on the
// event's own Philox word stream).  Counts other blocks may have written in the
// same launch are read with L2-coherent loads.
#pragma once
#include "internal.h"
#include "devmath.cuh"

namespace episim {

// ---- global-memory variant: one block per replicate, counts in global memory
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
    have[c] = (c >= c_lo && c < c_hi) ? __ldcg(X + (size_t)c * N + node) : 0;
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
  ws.ctr = make_uint4((uint32_t)e, (uint32_t)a.day | kEventTag, 0u, (uint32_t)(a.rep_base + r));
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
      if (took[c]) X[(size_t)(c + 2) * N + node] = __ldcg(X + (size_t)(c + 2) * N + node) + took[c];
  } else if (kind == 3) {  // external transfer to dest
#pragma unroll
    for (int c = 0; c < 2 * NA; ++c)
      if (took[c]) atomicAdd(&X[(size_t)c * N + dest], took[c]);
  }
  ++applied;
}

template <int NA>
__device__ __forceinline__ void events_block_global(const EvArgs& a, int r) {
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


// ---- staged variant.  Per replicate block: the day's records, the first two
// Philox blocks of every event, the level offsets and the counts of every node
// the day touches are loaded into shared memory; levels wider than a warp are
// processed by the whole block with a block barrier after each, narrower levels
// by warp 0 alone with a warp barrier (the deep tail of a hub node's chain);
// counts are written back at the end.  Same results as the global variant.
struct Words8 {
  uint4 a, b;
};

// Word stream of one event: the two precomputed Philox blocks, then further
// blocks computed on demand (events of more than 8 animals or with rejections).
struct EventWords {
  Words8 w;
  uint4 extra;
  uint32_t q, e, day, rep, k0, k1;
  __device__ __forceinline__ uint32_t operator()() {
    const uint32_t i = q++;
    if (i < 4u) return i == 0 ? w.a.x : i == 1 ? w.a.y : i == 2 ? w.a.z : w.a.w;
    if (i < 8u) return i == 4 ? w.b.x : i == 5 ? w.b.y : i == 6 ? w.b.z : w.b.w;
    if ((i & 3u) == 0u) extra = philox10(make_uint4(e, day | kEventTag, i >> 2, rep), k0, k1);
    const uint32_t sel = i & 3u;
    return sel == 0 ? extra.x : sel == 1 ? extra.y : sel == 2 ? extra.z : extra.w;
  }
};

template <bool ATOMIC>
__device__ __forceinline__ void add_count(int32_t* p, int32_t v) {
  if (ATOMIC) atomicAdd(p, v); else *p += v;
}

// The k-th 32-bit word of an event's stream when no draw before k was rejected.
__device__ __forceinline__ uint32_t word_k(const Words8& w, int k) {
  const uint4 v = k < 4 ? w.a : w.b;
  const int j = k & 3;
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Draw slots one at a time.  Draw k uses word k and range avail - k while no
// earlier draw was rejected (one word per draw, so the stream position is k);
// the first draw that Lemire's method might reject (low product word below the
// range) and every draw after it go through the exact word stream from position
// k on, rejections included.  Same slots as the sequential definition.
struct DrawState {
  EventWords ws;
  bool exact;
};

__device__ __forceinline__ uint32_t draw_slot(DrawState& st, int k, uint32_t range) {
  if (!st.exact && k < 8) {
    const uint64_t m = (uint64_t)word_k(st.ws.w, k) * range;
    if ((uint32_t)m >= range) return (uint32_t)(m >> 32);
    st.exact = true;
    st.ws.q = (uint32_t)k;
  } else if (!st.exact) {
    st.exact = true;
    st.ws.q = (uint32_t)k;
  }
  return lemire(range, st.ws);
}

template <int NA, bool ATOMIC>
__device__ __forceinline__ void apply_event_smem(int underflow_error, int32_t* err, int day, uint64_t seed,
                                                 int32_t* cnt, uint32_t rep, int4 rec, const Words8& w8,
                                                 unsigned& applied, unsigned& clamped, unsigned& skipped) {
  constexpr int NC = 2 * NA;
  const int src = rec.x, dst = rec.y;
  const int kind = rec.w & 3;
  const int cls = ((rec.w >> 2) & 3) - 1;
  const int32_t n = (int32_t)((uint32_t)rec.w >> 4);
  int32_t* cs = cnt + src * NC;
  if (kind == 1) {                                   // enter: susceptibles of the class
    add_count<ATOMIC>(&cs[2 * (cls < 0 ? 0 : cls)], n);
    ++applied;
    return;
  }
  DrawState st;
  st.ws.w = w8; st.ws.q = 0; st.ws.e = (uint32_t)rec.z; st.ws.day = (uint32_t)day; st.ws.rep = rep;
  st.ws.k0 = (uint32_t)seed; st.ws.k1 = (uint32_t)(seed >> 32);
  st.exact = false;
  if (cls >= 0) {
    // one class: draws pick S or I
    const int32_t s0 = cs[2 * cls], s1 = cs[2 * cls + 1];
    const int32_t avail = s0 + s1;
    int32_t take = n;
    if (n > avail) {
      if (underflow_error) { ++skipped; atomicOr(err, 1); return; }
      take = avail;
      ++clamped;
    }
    int32_t t0, t1;
    if (take == avail) { t0 = s0; t1 = s1; }
    else if (s0 == 0) { t0 = 0; t1 = take; }
    else if (s1 == 0) { t0 = take; t1 = 0; }
    else {
      t0 = 0;
      for (int32_t k = 0; k < take; ++k) {
        const uint32_t sl = draw_slot(st, k, (uint32_t)(avail - k));
        t0 += (sl < (uint32_t)(s0 - t0)) ? 1 : 0;
      }
      t1 = take - t0;
    }
    cs[2 * cls] = s0 - t0;
    cs[2 * cls + 1] = s1 - t1;
    if (kind == 2) {                                 // aging: same state, next class
      cs[2 * cls + 2] += t0;
      cs[2 * cls + 3] += t1;
    } else if (kind == 3) {
      int32_t* cd = cnt + dst * NC;
      if (t0) add_count<ATOMIC>(&cd[2 * cls], t0);
      if (t1) add_count<ATOMIC>(&cd[2 * cls + 1], t1);
    }
    ++applied;
    return;
  }
  // every class: draws over all compartments in order
  int32_t have[NC];
  int32_t avail = 0, nonempty = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    have[c] = cs[c];
    avail += have[c];
    nonempty += have[c] > 0 ? 1 : 0;
  }
  int32_t take = n;
  if (n > avail) {
    if (underflow_error) { ++skipped; atomicOr(err, 1); return; }
    take = avail;
    ++clamped;
  }
  int32_t took[NC];
  if (take == avail || nonempty <= 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      took[c] = (take == avail) ? have[c] : (have[c] > 0 ? take : 0);
      cs[c] = have[c] - took[c];
    }
  } else {
    int32_t cum[NC];
    int32_t acc = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) { acc += have[c]; cum[c] = acc; took[c] = 0; }
    for (int32_t k = 0; k < take; ++k) {
      const uint32_t sl = draw_slot(st, k, (uint32_t)(avail - k));
      bool below[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) below[c] = sl < (uint32_t)cum[c];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        took[c] += (below[c] && (c == 0 || !below[c > 0 ? c - 1 : 0])) ? 1 : 0;
        cum[c] -= below[c] ? 1 : 0;
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) cs[c] = have[c] - took[c];
  }
  if (kind == 3) {
    int32_t* cd = cnt + dst * NC;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (took[c]) add_count<ATOMIC>(&cd[c], took[c]);
  }
  ++applied;
}

template <int NA>
__device__ __forceinline__ void events_block_smem(const EvSmemArgs& a, int r, unsigned char* smem) {
  constexpr int NC = 2 * NA;
  const uint32_t rep = (uint32_t)(a.rep_base + r);
  int32_t* X = a.counts + (size_t)r * NC * a.N;
  const int l0 = a.day_lvl[a.day], l1 = a.day_lvl[a.day + 1];
  const int e0 = a.lvl_start[l0], e1 = a.lvl_start[l1];
  const int nev = e1 - e0, nlev = l1 - l0;
  const int t0 = a.day_touch[a.day], t1 = a.day_touch[a.day + 1];
  const int nt = t1 - t0;
  int4* srec = reinterpret_cast<int4*>(smem);
  Words8* swords = reinterpret_cast<Words8*>(smem + (size_t)nev * 16);
  int32_t* scnt = reinterpret_cast<int32_t*>(smem + (size_t)nev * 48);
  int32_t* slvl = scnt + (size_t)nt * NC;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  // counts of the touched nodes: one node per thread, its compartments in flight together
  for (int i0 = threadIdx.x; i0 < nt; i0 += 4 * blockDim.x) {
    int v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < nt ? a.touched[t0 + i] : -1;
    }
    int32_t x[4][NC];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NC; ++c) x[u][c] = v[u] >= 0 ? __ldcg(X + (size_t)c * a.N + v[u]) : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < nt) {
#pragma unroll
        for (int c = 0; c < NC; ++c) scnt[i * NC + c] = x[u][c];
      }
    }
  }
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    const int4 rc = a.rec[e0 + i];
    srec[i] = rc;
    const uint4 c0 = make_uint4((uint32_t)rc.z, (uint32_t)a.day | kEventTag, 0u, rep);
    Words8 w;
    w.a = philox10(c0, k0, k1);
    w.b = philox10(make_uint4(c0.x, c0.y, 1u, rep), k0, k1);
    swords[i] = w;
  }
  for (int i = threadIdx.x; i <= nlev; i += blockDim.x) slvl[i] = a.lvl_start[l0 + i] - e0;
  __syncthreads();
  unsigned applied = 0, clamped = 0, skipped = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int l = 0;
  while (l < nlev) {
    const int b = slvl[l], end = slvl[l + 1];
    if (end - b > 32) {
      for (int q = b + (int)threadIdx.x; q < end; q += blockDim.x)
        apply_event_smem<NA, true>(a.underflow_error, a.err, a.day, a.seed, scnt, rep, srec[q], swords[q], applied, clamped, skipped);
      __syncthreads();
      ++l;
      continue;
    }
    // a run of narrow levels: warp 0 alone (lane i takes the level's i-th event),
    // the other warps wait at the barrier after the run
    int lr = l;
    while (lr < nlev && slvl[lr + 1] - slvl[lr] <= 32) ++lr;
    if (warp == 0) {
      int bb = b, ee = end;
      int4 rc = (bb + lane < ee) ? srec[bb + lane] : make_int4(0, 0, 0, 0);
      Words8 wd;
      if (bb + lane < ee) wd = swords[bb + lane];
      for (int k = l; k < lr; ++k) {
        // prefetch the next level's record while this one is applied
        const int nb = ee, ne = (k + 1 < lr) ? slvl[k + 2] : ee;
        int4 nrc = make_int4(0, 0, 0, 0);
        Words8 nwd;
        if (nb + lane < ne) { nrc = srec[nb + lane]; nwd = swords[nb + lane]; }
        if (bb + lane < ee) apply_event_smem<NA, true>(a.underflow_error, a.err, a.day, a.seed, scnt, rep, rc, wd, applied, clamped, skipped);
        __syncwarp();
        bb = nb; ee = ne; rc = nrc; wd = nwd;
      }
    }
    __syncthreads();
    l = lr;
  }
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const int v = a.touched[t0 + i];
    int32_t x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = scnt[i * NC + c];
#pragma unroll
    for (int c = 0; c < NC; ++c) X[(size_t)c * a.N + v] = x[c];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    applied += __shfl_down_sync(0xffffffffu, applied, o);
    clamped += __shfl_down_sync(0xffffffffu, clamped, o);
    skipped += __shfl_down_sync(0xffffffffu, skipped, o);
  }
  if (lane == 0) {
    unsigned long long* c = a.ctr + (size_t)r * 4;
    if (applied) atomicAdd(c + 1, (unsigned long long)applied);
    if (clamped) atomicAdd(c + 2, (unsigned long long)clamped);
    if (skipped) atomicAdd(c + 3, (unsigned long long)skipped);
  }
}


// One event on a node whose counts live in the owner's registers (x).  Same
// semantics and draws as apply_event_smem; transfer destinations are added in
// shared memory.  Each class case is straight-line code with compile-time
// register indices (a lone thread pays the latency of every instruction).
template <int NA, int J>
__device__ __forceinline__ void one_class_reg(int kind, int32_t n, int underflow_error, int32_t* err,
                                              DrawState& st, int32_t* cd, int32_t (&x)[2 * NA],
                                              unsigned& applied, unsigned& clamped, unsigned& skipped) {
  const int32_t s0 = x[2 * J], s1 = x[2 * J + 1];
  const int32_t avail = s0 + s1;
  int32_t take = n;
  if (n > avail) {
    if (underflow_error) { ++skipped; atomicOr(err, 1); return; }
    take = avail;
    ++clamped;
  }
  int32_t t0, t1;
  if (take == avail) { t0 = s0; t1 = s1; }
  else if (s0 == 0) { t0 = 0; t1 = take; }
  else if (s1 == 0) { t0 = take; t1 = 0; }
  else {
    t0 = 0;
    for (int32_t k = 0; k < take; ++k) {
      const uint32_t sl = draw_slot(st, k, (uint32_t)(avail - k));
      t0 += (sl < (uint32_t)(s0 - t0)) ? 1 : 0;
    }
    t1 = take - t0;
  }
  x[2 * J] = s0 - t0;
  x[2 * J + 1] = s1 - t1;
  if (kind == 2) {
    if (2 * J + 3 < 2 * NA) { x[2 * J + 2 < 2 * NA ? 2 * J + 2 : 0] += t0; x[2 * J + 3 < 2 * NA ? 2 * J + 3 : 0] += t1; }
  } else if (kind == 3) {
    if (t0) atomicAdd(&cd[2 * J], t0);
    if (t1) atomicAdd(&cd[2 * J + 1], t1);
  }
  ++applied;
}

template <int NA>
__device__ __forceinline__ void all_classes_reg(int kind, int32_t n, int underflow_error, int32_t* err,
                                                DrawState& st, int32_t* cd, int32_t (&x)[2 * NA],
                                                unsigned& applied, unsigned& clamped, unsigned& skipped) {
  constexpr int NC = 2 * NA;
  int32_t avail = x[0] + x[1];
  if (NA == 3) avail += (x[2 < NC ? 2 : 0] + x[3 < NC ? 3 : 0]) + (x[4 < NC ? 4 : 0] + x[5 < NC ? 5 : 0]);
  int32_t take = n;
  if (n > avail) {
    if (underflow_error) { ++skipped; atomicOr(err, 1); return; }
    take = avail;
    ++clamped;
  }
  if (take == 0) { ++applied; return; }
  int32_t took[NC];
  if (take == avail) {
#pragma unroll
    for (int c = 0; c < NC; ++c) { took[c] = x[c]; x[c] = 0; }
  } else {
    int nonempty = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) nonempty += x[c] > 0 ? 1 : 0;
    if (nonempty <= 1) {
#pragma unroll
      for (int c = 0; c < NC; ++c) { took[c] = x[c] > 0 ? take : 0; x[c] -= took[c]; }
    } else {
      int32_t cum[NC];
      int32_t acc = 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) { acc += x[c]; cum[c] = acc; took[c] = 0; }
      for (int32_t k = 0; k < take; ++k) {
        const uint32_t sl = draw_slot(st, k, (uint32_t)(avail - k));
        bool below[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) below[c] = sl < (uint32_t)cum[c];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          took[c] += (below[c] && (c == 0 || !below[c > 0 ? c - 1 : 0])) ? 1 : 0;
          cum[c] -= below[c] ? 1 : 0;
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] -= took[c];
    }
  }
  if (kind == 3) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (took[c]) atomicAdd(&cd[c], took[c]);
  }
  ++applied;
}

template <int NA>
__device__ __forceinline__ void apply_event_reg(int underflow_error, int32_t* err, int day, uint64_t seed,
                                                int32_t* cnt, uint32_t rep, int4 rec, const Words8& w8,
                                                int32_t (&x)[2 * NA], unsigned& applied, unsigned& clamped,
                                                unsigned& skipped) {
  const int kind = rec.w & 3;
  const int cls = ((rec.w >> 2) & 3) - 1;
  const int32_t n = (int32_t)((uint32_t)rec.w >> 4);
  if (kind == 1) {
    if (cls <= 0) x[0] += n;
    else if (NA == 3 && cls == 1) x[2 < 2 * NA ? 2 : 0] += n;
    else if (NA == 3) x[4 < 2 * NA ? 4 : 0] += n;
    ++applied;
    return;
  }
  DrawState st;
  st.ws.w = w8; st.ws.q = 0; st.ws.e = (uint32_t)rec.z; st.ws.day = (uint32_t)day; st.ws.rep = rep;
  st.ws.k0 = (uint32_t)seed; st.ws.k1 = (uint32_t)(seed >> 32);
  st.exact = false;
  int32_t* cd = cnt + rec.y * 2 * NA;
  if (cls < 0) all_classes_reg<NA>(kind, n, underflow_error, err, st, cd, x, applied, clamped, skipped);
  else if (cls == 0) one_class_reg<NA, 0>(kind, n, underflow_error, err, st, cd, x, applied, clamped, skipped);
  else if (NA == 3 && cls == 1) one_class_reg<NA, (NA == 3 ? 1 : 0)>(kind, n, underflow_error, err, st, cd, x, applied, clamped, skipped);
  else if (NA == 3) one_class_reg<NA, (NA == 3 ? 2 : 0)>(kind, n, underflow_error, err, st, cd, x, applied, clamped, skipped);
}

// ---- owner-computes variant (no levels): the day's touched nodes come in
// independent blocks (unions of connected components of the day's transfer
// graph; no event of one block touches a node of another).  In block b, thread t
// applies, in input order, the events of the nodes it owns.  A sampling of node v first waits until every
// transfer into v that precedes it in input order has been added (v's add
// counter); a transfer into w first waits until every sampling of w that precedes
// it is done (w's sampling counter).  Waits point only to earlier positions and
// each thread follows input order, so the earliest pending event is always
// runnable.  Waits are bounded: running out sets an error bit and an abort flag.
template <int NA>
__device__ __forceinline__ void events_block_dataflow(const EvDfArgs& a, int r, int b, unsigned char* smem) {
  constexpr int NC = 2 * NA;
  grid_dependents_launch();
  const uint32_t rep = (uint32_t)(a.rep_base + r);
  int32_t* X = a.counts + (size_t)r * NC * a.N;
  const int4 m0 = a.blk_meta[a.blk0 + b], m1 = a.blk_meta[a.blk0 + b + 1];
  const int e0 = m0.x, nev = m1.x - m0.x;
  const int t0 = m0.y, nt = m1.y - m0.y;
  const int h0 = m0.z, nslot = m1.z - m0.z - 1;
  int4* srec = reinterpret_cast<int4*>(smem);
  Words8* swords = reinterpret_cast<Words8*>(smem + (size_t)nev * 16);
  int4* swait = reinterpret_cast<int4*>(smem + (size_t)nev * 48);
  int32_t* scnt = reinterpret_cast<int32_t*>(smem + (size_t)nev * 64);
  int32_t* sadd = scnt + (size_t)nt * NC;
  int32_t* ssmp = sadd + nt;
  int32_t* sbeg = ssmp + nt;                       // per thread: its events [sbeg, send)
  int32_t* send = sbeg + kDfThreads;
  int32_t* sabort = send + kDfThreads;
  for (int i = threadIdx.x; i < kDfThreads; i += blockDim.x) { sbeg[i] = 0; send[i] = 0; }
  __syncthreads();
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  // setup, first what does not depend on the previous kernel (records, waits,
  // Philox blocks, the thread table), then, after the grid dependency is
  // resolved, the scattered count loads of up to 4 nodes per thread
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    const int4 rc = a.rec[e0 + i];
    const int4 wv = a.wait[e0 + i];
    const uint4 c0 = make_uint4((uint32_t)rc.z, (uint32_t)a.day | kEventTag, 0u, rep);
    Words8 w;
    w.a = philox10(c0, k0, k1);
    w.b = philox10(make_uint4(c0.x, c0.y, 1u, rep), k0, k1);
    swords[i] = w;
    srec[i] = rc;
    swait[i] = wv;
  }
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) {
    const int t = a.thr_id[h0 + i];
    sbeg[t] = a.thr_off[h0 + i];
    send[t] = a.thr_off[h0 + i + 1];
  }
  grid_dependency_wait();
  for (int i0 = threadIdx.x; i0 < nt; i0 += 4 * blockDim.x) {
    int v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < nt ? a.touched[t0 + i] : -1;
    }
    int32_t x[4][NC];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NC; ++c) x[u][c] = v[u] >= 0 ? __ldcg(X + (size_t)c * a.N + v[u]) : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < nt) {
#pragma unroll
        for (int c = 0; c < NC; ++c) scnt[i * NC + c] = x[u][c];
        sadd[i] = 0;
        ssmp[i] = 0;
      }
    }
  }
  if (threadIdx.x == 0) *sabort = 0;
  __syncthreads();
  unsigned applied = 0, clamped = 0, skipped = 0;
  const int q0 = sbeg[threadIdx.x], q1 = send[threadIdx.x];
  // a thread owning one heavy node (lane 0 of one of the block's first heavy warps)
  // keeps the node's counts in registers; the node's shared-memory counts then
  // act as an inbox for transfers from other threads, drained after each wait
  const bool whole = (m0.w >> 16) != 0;
  const bool heavy = !whole && (threadIdx.x & 31) == 0 && (int)(threadIdx.x >> 5) < (m0.w & 0xFFFF) && q0 < q1;
  int32_t hx[NC];
  int hslot = -1;
  if (whole) {
    // every thread owns whole components: no other thread touches its nodes, so
    // the counts of the node its events currently sample stay in registers
    // (written back when the sampled node changes); adds to other nodes go to
    // shared memory, where a later switch reads them
    int4 rcw = make_int4(0, 0, 0, 0);
    Words8 wdw;
    if (q0 < q1) { rcw = srec[q0]; wdw = swords[q0]; }
    for (int q = q0; q < q1; ++q) {
      int4 nrc = rcw;
      Words8 nwd = wdw;
      if (q + 1 < q1) { nrc = srec[q + 1]; nwd = swords[q + 1]; }
      if (rcw.x != hslot) {
        if (hslot >= 0) {
#pragma unroll
          for (int c = 0; c < NC; ++c) scnt[hslot * NC + c] = hx[c];
        }
        hslot = rcw.x;
#pragma unroll
        for (int c = 0; c < NC; ++c) hx[c] = scnt[hslot * NC + c];
      }
      apply_event_reg<NA>(a.underflow_error, a.err, a.day, a.seed, scnt, rep, rcw, wdw, hx, applied, clamped, skipped);
      rcw = nrc; wdw = nwd;
    }
    if (hslot >= 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) scnt[hslot * NC + c] = hx[c];
    }
  }
  if (heavy) {
    hslot = srec[q0].x;
#pragma unroll
    for (int c = 0; c < NC; ++c) { hx[c] = scnt[hslot * NC + c]; scnt[hslot * NC + c] = 0; }
  }
  int4 rc = make_int4(0, 0, 0, 0), wt = make_int4(0, 0, 0, 0);
  Words8 wd;
  if (q0 < q1) { rc = srec[q0]; wt = swait[q0]; wd = swords[q0]; }
  for (int q = (whole ? q1 : q0); q < q1; ++q) {
    // next record in flight while this one is applied
    int4 nrc = rc, nwt = wt;
    Words8 nwd = wd;
    if (q + 1 < q1) { nrc = srec[q + 1]; nwt = swait[q + 1]; nwd = swords[q + 1]; }
    const int kind = rc.w & 3;
    if (wt.z & kDfAcquire) {
      bool ok = true;
      if (wt.x > 0) {                                  // transfers into src before this sampling
        volatile int32_t* p = sadd + rc.x;
        for (int it = 0; *p < wt.x; ++it)
          if (it >= a.spin_limit || *(volatile int32_t*)sabort) { ok = false; break; }
      }
      if (ok && wt.y > 0) {                            // samplings of dst before this transfer
        volatile int32_t* p = ssmp + rc.y;
        for (int it = 0; *p < wt.y; ++it)
          if (it >= a.spin_limit || *(volatile int32_t*)sabort) { ok = false; break; }
      }
      if (!ok) {
        if (!*(volatile int32_t*)sabort) atomicOr(a.err, kEventWaitTimeout);
        *(volatile int32_t*)sabort = 1;
        break;
      }
      __threadfence_block();
      if (heavy && wt.x > 0) {                        // drain the transfers received so far
#pragma unroll
        for (int c = 0; c < NC; ++c) hx[c] += atomicExch(&scnt[hslot * NC + c], 0);
      }
    }
    if (heavy) apply_event_reg<NA>(a.underflow_error, a.err, a.day, a.seed, scnt, rep, rc, wd, hx, applied, clamped,
                                   skipped);
    else apply_event_smem<NA, true>(a.underflow_error, a.err, a.day, a.seed, scnt, rep, rc, wd, applied, clamped,
                                    skipped);
    if (wt.z & (kDfPublishSampling | kDfPublishAdd)) {
      __threadfence_block();
      if (wt.z & kDfPublishSampling) *(volatile int32_t*)(ssmp + rc.x) = *(volatile int32_t*)(ssmp + rc.x) + 1;
      if (wt.z & kDfPublishAdd) atomicAdd(sadd + rc.y, 1);
    }
    (void)kind;
    rc = nrc; wt = nwt; wd = nwd;
  }
  if (heavy) {
#pragma unroll
    for (int c = 0; c < NC; ++c) atomicAdd(&scnt[hslot * NC + c], hx[c]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const int v = a.touched[t0 + i];
    int32_t x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = scnt[i * NC + c];
#pragma unroll
    for (int c = 0; c < NC; ++c) X[(size_t)c * a.N + v] = x[c];
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    applied += __shfl_down_sync(0xffffffffu, applied, o);
    clamped += __shfl_down_sync(0xffffffffu, clamped, o);
    skipped += __shfl_down_sync(0xffffffffu, skipped, o);
  }
  if (lane == 0) {
    unsigned long long* c = a.ctr + (size_t)r * 4;
    if (applied) atomicAdd(c + 1, (unsigned long long)applied);
    if (clamped) atomicAdd(c + 2, (unsigned long long)clamped);
    if (skipped) atomicAdd(c + 3, (unsigned long long)skipped);
  }
}

}  // namespace episim
