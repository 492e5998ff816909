// Host side of libepisim: the C ABI of include/episim.h, the event preprocessing
// (stable sort by day, per-day dependency levels; Sec. 3.4 rearrangement and
// the ordering rule 2(b) of Sec. 3.6, applied per node), device memory, and the
// per-day launch sequence (Alg. 1: stochastic step, events, phi update).
#include "../../include/episim.h"
#include "batch.h"
#include "internal.h"
#include "softdiv.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

using namespace episim;

struct sim_handle {
  sim_config cfg{};
  bool owns_state = true;           // false: counts and phi are the caller's device buffers (sim_create_on)
  int n_age = 1, nc = 2;
  std::vector<int32_t> u0;          // [Nc][N]
  std::vector<double> phi0;         // [N]
  std::vector<DevParams> params;    // [R]
  // device state
  int32_t* d_counts = nullptr;
  double* d_phi = nullptr;
  DevParams* d_params = nullptr;
  unsigned long long* d_prev_i = nullptr;
  unsigned long long* d_prev_n = nullptr;
  unsigned long long* d_ctr = nullptr;
  int32_t* d_err = nullptr;
  double* d_score = nullptr;
  double* d_tang = nullptr;
  double* d_traj = nullptr;         // reverse-mode score trajectory [3][max_days][R][N]
  int32_t score_day0 = 0;           // day since which score terms accumulate
  double* d_per_rep = nullptr;      // [R][8]
  double* d_moments = nullptr;      // scratch for sim_gradient_moments
  int32_t* d_days = nullptr;
  int32_t moments_cap = 0;
  int32_t* d_u0 = nullptr;          // [Nc][N] master copy for resets
  int32_t* d_order = nullptr;       // node order of the stochastic step
  int32_t n_order = 0;              // nodes in it: the handle's node range
  int32_t node_lo = 0, node_hi = 0; // nodes whose stochastic step and phi update this handle runs
                                    // (sim_shard; default every node); events apply to all nodes
  int32_t phase = 0;                // 1: the current day's stochastic step ran alone
                                    // (sim_run_day_stochastic), its event step is due
  int32_t* d_pack_touched = nullptr;// scratch of sim_unpack_touched: rank bounds
  int32_t pack_bounds_cap = 0;
  // dataflow day loop (SIM_LAUNCH_FLOW)
  std::vector<int4> ev_host;          // events of days < max_days in day-stable order:
                                      // {node, dest (-1 unless a transfer), position, packed}
  std::vector<int64_t> ev_first;      // [max_days + 1]
  bool flow_built = false;
  std::vector<int32_t> flow_day_comp; // [max_days + 1] first component of each day
  int4* d_fl_rec = nullptr;
  int32_t* d_fl_cev = nullptr;
  int32_t* d_fl_cnode = nullptr;
  int32_t* d_fl_cnoff = nullptr;
  int32_t* d_fl_day_comp = nullptr;
  int32_t* d_fl_day_long = nullptr;
  std::vector<int32_t> flow_day_long; // [max_days] components of >= kFlowLong events
  int32_t* d_fl_cunit = nullptr;      // per component: its herds' distinct units
  int32_t* d_fl_cuoff = nullptr;
  int32_t* d_fl_K = nullptr;          // [max_days + 1][U1] cumulative components per unit
  int32_t flow_U1 = 0;
  std::vector<int32_t> order_host;    // the node order of the stochastic step (host copy)
  unsigned* d_rdy = nullptr;          // [R][U1] unit completion counters
  unsigned long long* d_flow_next = nullptr;
  int32_t* d_flow_abort = nullptr;
  long long* d_item_off = nullptr;
  int32_t item_cap = 0;
  long long flow_spin_limit = 1ll << 22;  // ~2 s of polling per wait
  int32_t n_big = 0;                // leading nodes of the order simulated one per warp
  int32_t warp_threshold = -1;      // herd size from which a node gets a warp (-1: automatic)
  int32_t group_threshold = -1;     // herd size from which a node gets an 8-lane group (-1: automatic)
  int32_t n_mid = 0;                // nodes after the warp-path ones simulated one per 8-lane group
  int32_t clock_margin_log2 = 17;   // speculative clock margin 2^-k (0: exact clock only)
  int32_t sm_count = 1;             // SMs of the handle's device
  int32_t overlap = 1;              // programmatic dependent launch between the day's kernels
  int32_t split = 0;                // next day's untouched herds alongside the event step
  int32_t eff_threshold = 1 << 30;  // herd size of the warp path in effect
  int32_t eff_group_threshold = 1 << 30;  // herd size of the group path in effect
  std::vector<int32_t> tlist_nmid;     // per day: group-path herds after them
  std::vector<int32_t> touched_host;   // per day, the herds the day's events touch
  std::vector<int32_t> day_touch_host; // [max_days + 1]
  std::vector<int32_t> tlist_nbig;     // per day: warp-path herds at the head of the day's touched list
  uint32_t* d_skip = nullptr;          // [max_days][ceil(N/32)] touched-herd bitmaps
  int32_t* d_tlist = nullptr;          // per day: touched herds, warp-path ones first, largest first
  cudaStream_t side = nullptr;         // stream of the untouched herds' step
  // region statistics of the fitting goal
  int32_t n_regions = 0;
  int32_t* d_reg_nodes = nullptr;      // nodes sorted by region
  int32_t* d_reg_off = nullptr;        // [J + 1]
  unsigned long long* d_s1 = nullptr;  // [max_days][J][Nc]
  unsigned long long* d_s2 = nullptr;
  long long* d_ref = nullptr;          // scratch for sim_goal
  double* d_goal = nullptr;
  size_t ref_cap = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* d_phi0 = nullptr;
  // event schedule
  bool events_loaded = false;
  int4* d_rec = nullptr;
  int4* d_rec_slot = nullptr;
  int32_t* d_lvl_start = nullptr;
  int32_t* d_day_lvl = nullptr;
  int32_t* d_touched = nullptr;
  int32_t* d_day_touch = nullptr;
  std::vector<int32_t> day_smem;     // shared-memory bytes of the staged event step per day (0: global variant)
  std::vector<int32_t> day_df;       // shared-memory bytes of the owner-computes step per day (0: not used)
  std::vector<int32_t> day_nblk;     // owner-computes blocks per replicate per day
  int4* d_rec_df = nullptr;
  int4* d_wait_df = nullptr;
  int32_t* d_thr_off = nullptr;
  int32_t* d_touched_df = nullptr;
  std::vector<int32_t> day_blk0;     // first block of each day
  int4* d_blk_meta = nullptr;
  int32_t* d_thr_id = nullptr;
  int32_t event_variant = 0;         // 0 auto, 1 global only, 2 levels (no owner-computes)
  int32_t* d_day_smem = nullptr;     // device copy for the persistent batch kernel
  std::vector<int64_t> sched_order;  // position in the day-stable order, execution order
  std::vector<int32_t> sched_level;
  std::vector<int32_t> day_lvl;      // [max_days + 1]
  int32_t day = 0;
  std::string err;
  // launch mode of sim_run_days: 0 stream, 1 CUDA graph, 2 persistent batch kernel
  int32_t launch_mode = 0;
  cudaGraphExec_t graph_exec = nullptr;
  int32_t graph_d0 = -1, graph_nd = -1;
  // tracing
  bool profiling = false;
  bool force_global_events = false;  // test switch: always use the global-memory event step
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;        // kind of each recorded pair
  size_t ev_used = 0;
};

namespace {

thread_local std::string g_create_error;

sim_status fail(sim_handle* h, sim_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_create_error = buf;
  return s;
}

sim_status cuda_fail(sim_handle* h, cudaError_t e, const char* what) {
  sim_status s = (e == cudaErrorMemoryAllocation) ? SIM_E_OOM : SIM_E_CUDA;
  return fail(h, s, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call, what)                              \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}

void free_split(sim_handle* h) {
  cudaFree(h->d_skip); cudaFree(h->d_tlist);
  h->d_skip = nullptr; h->d_tlist = nullptr;
  h->tlist_nbig.clear();
}

void free_flow(sim_handle* h) {
  cudaFree(h->d_fl_rec); cudaFree(h->d_fl_cev); cudaFree(h->d_fl_cnode); cudaFree(h->d_fl_cnoff);
  cudaFree(h->d_fl_day_comp); cudaFree(h->d_fl_day_long);
  cudaFree(h->d_fl_cunit); cudaFree(h->d_fl_cuoff); cudaFree(h->d_fl_K);
  cudaFree(h->d_rdy);
  h->d_rdy = nullptr;
  h->d_fl_cunit = nullptr; h->d_fl_cuoff = nullptr; h->d_fl_K = nullptr;
  h->flow_U1 = 0;
  h->d_fl_day_long = nullptr;
  h->flow_day_long.clear();
  h->d_fl_rec = nullptr; h->d_fl_cev = nullptr; h->d_fl_cnode = nullptr; h->d_fl_cnoff = nullptr;
  h->d_fl_day_comp = nullptr;
  h->flow_day_comp.clear();
  h->flow_built = false;
}

void free_events(sim_handle* h) {
  free_flow(h);
  h->ev_host.clear();
  h->ev_host.shrink_to_fit();
  h->ev_first.clear();
  cudaFree(h->d_rec); cudaFree(h->d_lvl_start); cudaFree(h->d_day_lvl);
  cudaFree(h->d_rec_slot); cudaFree(h->d_touched); cudaFree(h->d_day_touch); cudaFree(h->d_day_smem);
  cudaFree(h->d_rec_df); cudaFree(h->d_wait_df); cudaFree(h->d_thr_off); cudaFree(h->d_touched_df);
  cudaFree(h->d_blk_meta); cudaFree(h->d_thr_id);
  h->d_rec_df = nullptr; h->d_wait_df = nullptr; h->d_thr_off = nullptr; h->d_touched_df = nullptr;
  h->d_blk_meta = nullptr; h->d_thr_id = nullptr;
  h->day_blk0.clear();
  h->day_df.clear();
  h->day_nblk.clear();
  h->d_day_smem = nullptr;
  h->d_rec = nullptr; h->d_lvl_start = nullptr; h->d_day_lvl = nullptr;
  h->d_rec_slot = nullptr; h->d_touched = nullptr; h->d_day_touch = nullptr;
  h->sched_order.clear(); h->sched_level.clear(); h->day_lvl.clear(); h->day_smem.clear();
  h->touched_host.clear(); h->day_touch_host.clear();
  free_split(h);
  h->events_loaded = false;
}

void free_profile(sim_handle* h) {
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear(); h->ev_kind.clear(); h->ev_used = 0;
}

void free_graph(sim_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
  h->graph_d0 = h->graph_nd = -1;
}

void free_regions(sim_handle* h) {
  cudaFree(h->d_reg_nodes); cudaFree(h->d_reg_off); cudaFree(h->d_s1); cudaFree(h->d_s2);
  cudaFree(h->d_ref); cudaFree(h->d_goal);
  h->d_reg_nodes = h->d_reg_off = nullptr; h->d_s1 = h->d_s2 = nullptr; h->d_ref = nullptr; h->d_goal = nullptr;
  h->n_regions = 0; h->ref_cap = 0;
}

void free_all(sim_handle* h) {
  free_graph(h);
  free_regions(h);
  free_split(h);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->side = nullptr; h->ev_fork = h->ev_join = nullptr;
  free_profile(h);
  free_events(h);
  if (h->owns_state) { cudaFree(h->d_counts); cudaFree(h->d_phi); }
  cudaFree(h->d_params); cudaFree(h->d_prev_i);
  cudaFree(h->d_prev_n); cudaFree(h->d_ctr); cudaFree(h->d_err); cudaFree(h->d_score);
  cudaFree(h->d_tang); cudaFree(h->d_u0); cudaFree(h->d_phi0); cudaFree(h->d_order);
  cudaFree(h->d_traj); cudaFree(h->d_per_rep); cudaFree(h->d_moments); cudaFree(h->d_days);
  cudaFree(h->d_pack_touched);
  h->d_pack_touched = nullptr;
  h->pack_bounds_cap = 0;
  free_flow(h);
  cudaFree(h->d_flow_next); cudaFree(h->d_flow_abort); cudaFree(h->d_item_off);
  h->d_flow_next = nullptr; h->d_flow_abort = nullptr; h->d_item_off = nullptr;
  h->item_cap = 0;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

size_t n_counts(const sim_handle* h) { return (size_t)h->cfg.n_replicates * h->nc * h->cfg.n_nodes; }
size_t n_phi(const sim_handle* h) { return (size_t)h->cfg.n_replicates * h->cfg.n_nodes; }

// Initial state for every replicate and cleared accumulators (synchronous).
// Per-replicate constants from the public struct, validated (finite, >= 0,
// beta <= 1); errors are reported on handle eh (NULL: the creation error).
sim_status fill_params(const sim_handle* h, sim_handle* eh, const sim_params* p, std::vector<DevParams>& out) {
  const int R = h->cfg.n_replicates;
  if (!p->upsilon || !p->gamma || !p->alpha || !p->beta || !p->epsilon)
    return fail(eh, SIM_E_INVALID_ARG, "null parameter array");
  for (int r = 0; r < R; ++r) {
    DevParams& d = out[(size_t)r];
    std::memset(&d, 0, sizeof d);
    for (int j = 0; j < 3; ++j) {
      d.ups[j] = p->upsilon[(size_t)r * 3 + j];
      d.gam[j] = p->gamma[(size_t)r * 3 + j];
    }
    d.alpha = p->alpha[r];
    for (int s2 = 0; s2 < 4; ++s2) d.beta[s2] = p->beta[(size_t)r * 4 + s2];
    d.eps = p->epsilon[r];
    bool ok = finite_nonneg(d.alpha) && finite_nonneg(d.eps);
    for (int j = 0; j < 3; ++j) ok = ok && finite_nonneg(d.ups[j]) && finite_nonneg(d.gam[j]);
    for (int s2 = 0; s2 < 4; ++s2) ok = ok && finite_nonneg(d.beta[s2]) && d.beta[s2] <= 1.0;
    if (!ok)
      return fail(eh, SIM_E_INVALID_ARG, "replicate %d: parameters must be finite, >= 0, and beta <= 1", r);
  }
  return SIM_OK;
}

sim_status reset_state(sim_handle* h) {
  const size_t cbytes = (size_t)h->nc * h->cfg.n_nodes * sizeof(int32_t);
  const size_t pbytes = (size_t)h->cfg.n_nodes * sizeof(double);
  CK(h, launch_broadcast(h->d_counts, h->d_u0, cbytes, h->cfg.n_replicates, 0), "initial counts");
  CK(h, launch_broadcast(h->d_phi, h->d_phi0, pbytes, h->cfg.n_replicates, 0), "initial phi");
  const size_t stats = (size_t)h->cfg.n_replicates * (h->cfg.max_days > 0 ? h->cfg.max_days : 1);
  CK(h, cudaMemset(h->d_prev_i, 0, stats * 8), "clear stats");
  CK(h, cudaMemset(h->d_prev_n, 0, stats * 8), "clear stats");
  CK(h, cudaMemset(h->d_ctr, 0, (size_t)h->cfg.n_replicates * 4 * 8), "clear counters");
  CK(h, cudaMemset(h->d_err, 0, sizeof(int32_t)), "clear error");
  if (h->n_regions > 0) {
    const size_t rows = (size_t)std::max(1, h->cfg.max_days) * h->n_regions * h->nc;
    CK(h, cudaMemset(h->d_s1, 0, rows * 8), "clear region statistics");
    CK(h, cudaMemset(h->d_s2, 0, rows * 8), "clear region statistics");
  }
  if (h->d_score) {
    CK(h, cudaMemset(h->d_score, 0, n_phi(h) * kScoreTerms * sizeof(double)), "clear score");
    CK(h, cudaMemset(h->d_tang, 0, n_phi(h) * 2 * sizeof(double)), "clear tangents");
  }
  CK(h, cudaDeviceSynchronize(), "reset");
  h->day = 0;
  h->score_day0 = 0;
  return SIM_OK;
}

sim_status check_latched(sim_handle* h) {
  int32_t e = 0;
  CK(h, cudaMemcpy(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost), "read device error word");
  if (e) {
    CK(h, cudaMemset(h->d_err, 0, sizeof(int32_t)), "clear device error word");
    if (e & kEventWaitTimeout) return fail(h, SIM_E_TIMEOUT, "an event-step dependency wait ran out");
    return fail(h, SIM_E_UNDERFLOW, "an event asked for more animals than present (ERROR policy)");
  }
  return SIM_OK;
}

SsaArgs ssa_args(sim_handle* h) {
  SsaArgs a{};
  a.counts = h->d_counts; a.phi = h->d_phi; a.params = h->d_params;
  a.prev_i = h->d_prev_i; a.prev_n = h->d_prev_n; a.ctr = h->d_ctr;
  a.score = h->d_score; a.tang = h->d_tang; a.seed = h->cfg.seed; a.rep_base = h->cfg.replicate_base;
  a.N = h->cfg.n_nodes; a.R = h->cfg.n_replicates; a.Nc = h->nc; a.max_days = h->cfg.max_days;
  a.pre_event = (h->cfg.flags & SIM_FLAG_PHI_PRE_EVENT) ? 1 : 0;
  a.traj = h->d_traj;
  a.order = h->d_order;
  a.n_big = h->n_big;
  a.n_mid = h->n_mid;
  a.warp_blocks = (h->n_big + 7) / 8;
  a.clock_margin = h->clock_margin_log2 > 0 ? (1ull << (62 - h->clock_margin_log2)) : 0ull;
  a.sm_count = h->sm_count;
  a.overlap = h->overlap;
  a.n_list = h->n_order;
  a.node_lo = h->node_lo;
  a.node_hi = h->node_hi;
  a.skip = nullptr;
  return a;
}

// Node order of the stochastic step: nodes with at least `threshold` animals
// (initial herd) first, one warp each, largest first; then the others, largest
// first, one thread each (similar work per warp).  threshold < 0: automatic --
// warps only while the per-thread work leaves the GPU under-occupied (fewer than
// 152 x 1024 node-replicates), for herds of 400 animals or more.
// Tables of the split day step: the stochastic step of day d + 1 runs as two
// launches, the herds that day d's events leave untouched (alongside the event
// step of day d, on a second stream) and the touched ones (after it).  Per day:
// a bitmap of the touched herds and their list, warp-path herds first, each part
// largest first.
sim_status build_split(sim_handle* h) {
  free_split(h);
  if (!h->events_loaded || (h->cfg.flags & SIM_FLAG_SCORE) || h->day_touch_host.empty()) return SIM_OK;
  const int N = h->cfg.n_nodes;
  const int32_t T = h->cfg.max_days;
  const size_t words = ((size_t)N + 31) / 32;
  std::vector<int64_t> herd(N, 0);
  for (int c = 0; c < h->nc; ++c)
    for (int v = 0; v < N; ++v) herd[v] += h->u0[(size_t)c * N + v];
  std::vector<uint32_t> skip;
  std::vector<int32_t> tl(h->touched_host.size());
  try { skip.assign((size_t)T * words, 0u); } catch (...) { return fail(h, SIM_E_OOM, "host allocation"); }
  h->tlist_nbig.assign((size_t)T, 0);
  h->tlist_nmid.assign((size_t)T, 0);
  for (int32_t d = 0; d < T; ++d) {
    const int32_t b = h->day_touch_host[(size_t)d], e = h->day_touch_host[(size_t)d + 1];
    for (int32_t i = b; i < e; ++i) {
      const int v = h->touched_host[(size_t)i];
      skip[(size_t)d * words + (size_t)(v >> 5)] |= 1u << (v & 31);
      tl[(size_t)i] = v;
    }
    std::stable_sort(tl.begin() + b, tl.begin() + e, [&](int32_t x, int32_t y) { return herd[x] > herd[y]; });
    int32_t nb = 0, nm = 0;
    while (b + nb < e && herd[tl[(size_t)(b + nb)]] >= h->eff_threshold) ++nb;
    while (b + nb + nm < e && herd[tl[(size_t)(b + nb + nm)]] >= h->eff_group_threshold) ++nm;
    h->tlist_nbig[(size_t)d] = nb;
    h->tlist_nmid[(size_t)d] = nm;
  }
  cudaError_t err = dalloc(&h->d_skip, skip.size());
  if (err == cudaSuccess) err = dalloc(&h->d_tlist, tl.size());
  if (err == cudaSuccess && !skip.empty()) err = cudaMemcpy(h->d_skip, skip.data(), skip.size() * 4, cudaMemcpyHostToDevice);
  if (err == cudaSuccess && !tl.empty()) err = cudaMemcpy(h->d_tlist, tl.data(), tl.size() * 4, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) { free_split(h); return cuda_fail(h, err, "split tables"); }
  return SIM_OK;
}

sim_status set_order(sim_handle* h, int32_t threshold) {
  const int N = h->cfg.n_nodes;
  std::vector<int64_t> herd(N, 0);
  for (int c = 0; c < h->nc; ++c)
    for (int v = 0; v < N; ++v) herd[v] += h->u0[(size_t)c * N + v];
  const int n_own = h->node_hi - h->node_lo;
  std::vector<int32_t> order(n_own);
  for (int i = 0; i < n_own; ++i) order[i] = h->node_lo + i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return herd[a] > herd[b]; });
  int32_t thr = threshold;
  if (thr < 0) {
    const int64_t work = (int64_t)N * h->cfg.n_replicates;
    thr = (work < 152 * 1024) ? 400 : (1 << 30);
  }
  int32_t gthr = h->group_threshold;
  if (gthr < 0) {
    const int64_t work = (int64_t)N * h->cfg.n_replicates;
    gthr = (work < 152 * 1024) ? 200 : (1 << 30);
  }
  int32_t nb = 0, nm = 0;
  if (!(h->cfg.flags & SIM_FLAG_SCORE)) {
    while (nb < n_own && herd[order[nb]] >= thr) ++nb;
    while (nb + nm < n_own && herd[order[nb + nm]] >= gthr) ++nm;
  }
  if (!h->d_order) CK(h, dalloc(&h->d_order, (size_t)N), "node order allocation");
  if (n_own > 0)
    CK(h, cudaMemcpy(h->d_order, order.data(), (size_t)n_own * 4, cudaMemcpyHostToDevice), "node order upload");
  h->n_order = n_own;
  h->order_host.swap(order);
  free_flow(h);
  h->n_big = nb;
  h->n_mid = nm;
  h->eff_group_threshold = (h->cfg.flags & SIM_FLAG_SCORE) ? (1 << 30) : gthr;
  h->warp_threshold = threshold;
  h->eff_threshold = (h->cfg.flags & SIM_FLAG_SCORE) ? (1 << 30) : thr;
  free_graph(h);
  return build_split(h);
}


struct Schedule {
  std::vector<int4> rec;          // execution order
  std::vector<int4> rec_slot;     // same, with node slots of the day's touched list
  // owner-computes form: per day, the touched nodes split into independent blocks
  // (unions of connected components of the day's transfer graph); per block,
  // events grouped by owner thread, input order within
  std::vector<int4> rec_df;       // {block slot of src, block slot of dst, position, packed}
  std::vector<int4> wait_df;      // {transfer-adds into src before it, samplings of dst before it, flags, 0}
  std::vector<int32_t> touched_df;// node ids per block slot, blocks in order
  std::vector<int32_t> thr_off;   // per block: event offsets of its owner threads in use (block-relative), + end
  std::vector<int32_t> thr_id;    // per block, aligned with thr_off: those threads' indices, then -1
  std::vector<int32_t> day_blk;   // [max_days + 1] first block of each day
  std::vector<int4> blk_meta;     // [blocks + 1] first record, first node, first thr_off entry, heavy units
  std::vector<int32_t> touched;   // node ids per day slot
  std::vector<int32_t> day_touch; // [max_days + 1]
  std::vector<int32_t> lvl_start; // [levels + 1]
  std::vector<int32_t> day_lvl;   // [max_days + 1]
  std::vector<int64_t> order;     // day-stable position of each record
  std::vector<int32_t> level;
};

// Scratch of build_owner_form, kept across the days one thread schedules (its
// vectors are re-filled each day, so the day loop allocates only while they grow).
struct OwnerScratch {
  std::vector<int32_t> par, comp_of, comp_ev, id, evcount, blk_of_comp, cs, blk_nt, local, blk_t0, adds, samps,
      blk_n, comp_depth, comp_nodes, owner, comp_owner;
  std::vector<int64_t> last_into, last_samp;
  std::vector<std::pair<int64_t, int>> heapv;
  std::vector<int4> rec, wt;
  // per block, in CSR form: its nodes, components and events (ascending)
  std::vector<int32_t> bn_off, bn, bc_off, bc, be_off, be, fillb;
  // per block while it is built
  std::vector<int32_t> units, ord, uowner, slot_of_thr, thr_ids, off, fill;
  std::vector<int64_t> uev, load;
  std::vector<std::pair<int64_t, int>> thr_heap;
  std::vector<char> single;
};

// CSR of items 0..n-1 grouped by key_of(item) in [0, G), ascending items inside
// a group (the order push_back in item order gives).
template <class K>
void group_csr(int n, int G, K key_of, std::vector<int32_t>& off, std::vector<int32_t>& items,
               std::vector<int32_t>& fill) {
  off.assign((size_t)G + 1, 0);
  for (int i = 0; i < n; ++i) off[(size_t)key_of(i) + 1]++;
  for (int g = 0; g < G; ++g) off[(size_t)g + 1] += off[(size_t)g];
  items.resize((size_t)n);
  fill.assign(off.begin(), off.end() - 1);
  for (int i = 0; i < n; ++i) items[(size_t)fill[(size_t)key_of(i)]++] = i;
}

// Owner-computes form of one day (events at day-stable positions [s0, s1)).
// The day's touched nodes fall into connected components of its transfer graph;
// events of different components never touch a common node, so the components
// are packed longest-first onto at most max_blocks blocks that run without any
// exchange between them.  Within a block every node is owned by one thread, which
// applies the node's events (enter, exit, aging, transfer out) in input order.  A
// sampling event waits until every transfer into its node that precedes it has
// been added; a transfer waits until every sampling of its destination that
// precedes it is done.  Waits only ever point to earlier input positions, so
// threads that each follow input order always make progress.  Nodes with many
// events get a warp of their own (lane 0), so that their chain is not serialised
// behind other lanes; the others are packed longest-first onto the least-loaded
// threads.
void build_owner_form(Schedule& S, int64_t s0, int64_t s1, int32_t touch0,
                      const std::vector<int64_t>& by_pos, const int32_t* kind, const int32_t* node,
                      const int32_t* dest, const int32_t* count, const int32_t* cls,
                      const std::vector<int32_t>& slot_of, const std::vector<int32_t>& lvl_of, int max_blocks,
                      OwnerScratch& W) {
  const int nt = (int)S.touched.size() - touch0;
  const int64_t n = s1 - s0;
  S.day_blk.push_back((int32_t)S.blk_meta.size());
  if (n == 0) return;
  // components (union-find over the day slots)
  auto& par = W.par;
  par.resize((size_t)nt);
  for (int i = 0; i < nt; ++i) par[(size_t)i] = i;
  auto find = [&](int x) {
    while (par[(size_t)x] != x) { par[(size_t)x] = par[(size_t)par[(size_t)x]]; x = par[(size_t)x]; }
    return x;
  };
  for (int64_t s = s0; s < s1; ++s) {
    const int64_t e = by_pos[(size_t)s];
    if (kind[e] != SIM_EXTERNAL) continue;
    const int a = find(slot_of[node[e]]), b = find(slot_of[dest[e]]);
    if (a != b) par[(size_t)(a < b ? b : a)] = a < b ? a : b;
  }
  auto& comp_of = W.comp_of;
  auto& comp_ev = W.comp_ev;
  comp_of.resize((size_t)nt);
  comp_ev.clear();
  W.id.assign((size_t)nt, -1);
  for (int i = 0; i < nt; ++i) {
    const int r = find(i);
    if (W.id[(size_t)r] < 0) { W.id[(size_t)r] = (int32_t)comp_ev.size(); comp_ev.push_back(0); }
    comp_of[(size_t)i] = W.id[(size_t)r];
  }
  auto& evcount = W.evcount;
  evcount.assign((size_t)nt, 0);
  for (int64_t s = s0; s < s1; ++s) {
    const int a = slot_of[node[by_pos[(size_t)s]]];
    evcount[(size_t)a]++;
    comp_ev[(size_t)comp_of[(size_t)a]]++;
  }
  const int ncomp = (int)comp_ev.size();
  const int G = std::max(1, std::min(max_blocks, ncomp));
  // components longest-first onto the least-loaded block
  auto& blk_of_comp = W.blk_of_comp;
  blk_of_comp.resize((size_t)ncomp);
  {
    auto& cs = W.cs;
    cs.resize((size_t)ncomp);
    for (int c = 0; c < ncomp; ++c) cs[(size_t)c] = c;
    std::stable_sort(cs.begin(), cs.end(), [&](int a, int b) { return comp_ev[(size_t)a] > comp_ev[(size_t)b]; });
    auto& heapv = W.heapv;
    heapv.clear();
    for (int b = 0; b < G; ++b) heapv.push_back({0, b});
    auto cmp = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
      return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    std::make_heap(heapv.begin(), heapv.end(), cmp);
    for (int c : cs) {
      std::pop_heap(heapv.begin(), heapv.end(), cmp);
      heapv.back().first += comp_ev[(size_t)c];
      blk_of_comp[(size_t)c] = heapv.back().second;
      std::push_heap(heapv.begin(), heapv.end(), cmp);
    }
  }
  // block-local slots, blocks in order, day slot order within a block
  auto& blk_nt = W.blk_nt;
  auto& local = W.local;
  blk_nt.assign((size_t)G, 0);
  local.resize((size_t)nt);
  for (int i = 0; i < nt; ++i) {
    const int b = blk_of_comp[(size_t)comp_of[(size_t)i]];
    local[(size_t)i] = blk_nt[(size_t)b]++;
  }
  auto& blk_t0 = W.blk_t0;
  blk_t0.assign((size_t)G + 1, 0);
  for (int b = 0; b < G; ++b) blk_t0[(size_t)b + 1] = blk_t0[(size_t)b] + blk_nt[(size_t)b];
  const size_t tbase = S.touched_df.size();
  S.touched_df.resize(tbase + (size_t)nt);
  for (int i = 0; i < nt; ++i) {
    const int b = blk_of_comp[(size_t)comp_of[(size_t)i]];
    S.touched_df[tbase + (size_t)(blk_t0[(size_t)b] + local[(size_t)i])] = S.touched[(size_t)touch0 + (size_t)i];
  }
  // wait counts in input order, and which events must publish: a sampling of v
  // when a transfer into v follows it, a transfer into w when a sampling of w
  // follows it (only those counters are ever waited on)
  auto& adds = W.adds;
  auto& samps = W.samps;
  adds.assign((size_t)nt, 0);
  samps.assign((size_t)nt, 0);
  auto& last_into = W.last_into;
  auto& last_samp = W.last_samp;
  last_into.assign((size_t)nt, -1);
  last_samp.assign((size_t)nt, -1);
  for (int64_t s = s0; s < s1; ++s) {
    const int64_t e = by_pos[(size_t)s];
    const int k = kind[e];
    if (k != SIM_ENTER) last_samp[(size_t)slot_of[node[e]]] = s;
    if (k == SIM_EXTERNAL) last_into[(size_t)slot_of[dest[e]]] = s;
  }
  auto& rec = W.rec;
  auto& wt = W.wt;
  rec.resize((size_t)n);
  wt.resize((size_t)n);
  auto& blk_n = W.blk_n;
  blk_n.assign((size_t)G, 0);
  for (int64_t s = s0; s < s1; ++s) {
    const int64_t e = by_pos[(size_t)s];
    const int k = kind[e];
    const int a = slot_of[node[e]];
    const int b = (k == SIM_EXTERNAL) ? slot_of[dest[e]] : -1;
    const uint32_t packed = (uint32_t)k | ((uint32_t)(cls[e] + 1) << 2) | ((uint32_t)count[e] << 4);
    rec[(size_t)(s - s0)] = make_int4(local[(size_t)a], b >= 0 ? local[(size_t)b] : -1, (int32_t)s, (int32_t)packed);
    int4 w = make_int4(0, 0, 0, 0);
    if (k != SIM_ENTER) {
      w.x = adds[(size_t)a]; samps[(size_t)a]++;
      if (s < last_into[(size_t)a]) w.z |= kDfPublishSampling;
    }
    if (k == SIM_EXTERNAL) {
      w.y = samps[(size_t)b]; adds[(size_t)b]++;
      if (s < last_samp[(size_t)b]) w.z |= kDfPublishAdd;
    }
    if (w.x > 0 || w.y > 0) w.z |= kDfAcquire;
    wt[(size_t)(s - s0)] = w;
    blk_n[(size_t)blk_of_comp[(size_t)comp_of[(size_t)a]]]++;
  }
  // per block: owner threads, events grouped by owner in input order.  A
  // component whose events are about as many as its dependency depth (a chain,
  // as register-shaped days mostly give) is owned whole by one thread: its events
  // then need no wait and no publication at all.  A block holding a component
  // with much more parallelism inside gives each of its nodes a thread instead.
  auto& comp_depth = W.comp_depth;
  auto& comp_nodes = W.comp_nodes;
  comp_depth.assign((size_t)ncomp, 0);
  comp_nodes.assign((size_t)ncomp, 0);
  for (int64_t s = s0; s < s1; ++s) {
    const int c = comp_of[(size_t)slot_of[node[by_pos[(size_t)s]]]];
    comp_depth[(size_t)c] = std::max(comp_depth[(size_t)c], lvl_of[(size_t)s]);
  }
  for (int i = 0; i < nt; ++i) comp_nodes[(size_t)comp_of[(size_t)i]]++;
  group_csr(nt, G, [&](int i) { return blk_of_comp[(size_t)comp_of[(size_t)i]]; }, W.bn_off, W.bn, W.fillb);
  group_csr(ncomp, G, [&](int c) { return blk_of_comp[(size_t)c]; }, W.bc_off, W.bc, W.fillb);
  group_csr((int)n, G, [&](int i) { return blk_of_comp[(size_t)comp_of[(size_t)slot_of[node[by_pos[(size_t)(s0 + i)]]]]]; },
            W.be_off, W.be, W.fillb);
  auto& owner = W.owner;
  auto& comp_owner = W.comp_owner;
  owner.assign((size_t)nt, -1);
  comp_owner.assign((size_t)ncomp, -1);
  const int warps = kDfThreads / 32;
  for (int b = 0; b < G; ++b) {
    const int32_t* bnodes = W.bn.data() + W.bn_off[(size_t)b];
    const int nbn = W.bn_off[(size_t)b + 1] - W.bn_off[(size_t)b];
    const int32_t* bcomps = W.bc.data() + W.bc_off[(size_t)b];
    const int nbc = W.bc_off[(size_t)b + 1] - W.bc_off[(size_t)b];
    const int32_t* bevs = W.be.data() + W.be_off[(size_t)b];
    const int nbe = W.be_off[(size_t)b + 1] - W.be_off[(size_t)b];
    bool whole = true;
    for (int q = 0; q < nbc; ++q) {
      const int c = bcomps[q];
      if (comp_ev[(size_t)c] > 4 * comp_depth[(size_t)c] + 32) whole = false;
    }
    // owner units: components (whole) or nodes, with their event counts and
    // whether all their events sample one node (register-resident chains)
    auto& units = W.units;
    auto& uev = W.uev;
    auto& single = W.single;
    units.clear(); uev.clear(); single.clear();
    if (whole) {
      for (int q = 0; q < nbc; ++q) {
        const int c = bcomps[q];
        units.push_back(c); uev.push_back(comp_ev[(size_t)c]); single.push_back(comp_nodes[(size_t)c] == 1);
      }
    } else {
      for (int q = 0; q < nbn; ++q) {
        const int i = bnodes[q];
        if (evcount[(size_t)i] > 0) { units.push_back(i); uev.push_back(evcount[(size_t)i]); single.push_back(1); }
      }
    }
    auto& ord = W.ord;
    ord.resize(units.size());
    for (size_t k = 0; k < ord.size(); ++k) ord[k] = (int32_t)k;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return uev[(size_t)x] > uev[(size_t)y]; });
    auto& uowner = W.uowner;
    uowner.assign(units.size(), -1);
    const int64_t nb = blk_n[(size_t)b];
    int heavy = 0;
    const int64_t heavy_min = std::max<int64_t>(32, nb / 64);
    while (heavy < (int)ord.size() && heavy < warps / 2 && uev[(size_t)ord[(size_t)heavy]] >= heavy_min &&
           single[(size_t)ord[(size_t)heavy]]) {
      uowner[(size_t)ord[(size_t)heavy]] = heavy * 32;            // lane 0 of its own warp
      ++heavy;
    }
    // the others dealt lane-major over the remaining warps (a warp per unit while
    // they last, heaviest first, so that units share no warp: their event kinds
    // would diverge); past 32 per warp, least-loaded threads
    const int wfree = warps - heavy;
    auto& load = W.load;
    load.assign((size_t)kDfThreads, 0);
    for (int h = 0; h < heavy; ++h) load[(size_t)h * 32] = uev[(size_t)ord[(size_t)h]];
    // (least loaded: smallest (load, thread), kept in a min-heap once reached)
    auto& tq = W.thr_heap;
    auto tq_cmp = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
      return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    for (size_t k = (size_t)heavy; k < ord.size(); ++k) {
      const int64_t kk = (int64_t)k - heavy;
      int t;
      if (kk < (int64_t)wfree * 32) {
        t = (heavy + (int)(kk % wfree)) * 32 + (int)(kk / wfree);
      } else {
        if (kk == (int64_t)wfree * 32) {
          tq.clear();
          for (int q = heavy * 32; q < kDfThreads; ++q) tq.push_back({load[(size_t)q], q});
          std::make_heap(tq.begin(), tq.end(), tq_cmp);
        }
        std::pop_heap(tq.begin(), tq.end(), tq_cmp);
        t = tq.back().second;
        tq.back().first += uev[(size_t)ord[k]];
        std::push_heap(tq.begin(), tq.end(), tq_cmp);
      }
      uowner[(size_t)ord[k]] = t;
      load[(size_t)t] += uev[(size_t)ord[k]];
    }
    if (whole) {
      for (size_t k = 0; k < units.size(); ++k) comp_owner[(size_t)units[k]] = uowner[k];
      for (int q = 0; q < nbn; ++q) owner[(size_t)bnodes[q]] = comp_owner[(size_t)comp_of[(size_t)bnodes[q]]];
    } else {
      for (size_t k = 0; k < units.size(); ++k) owner[(size_t)units[k]] = uowner[k];
    }
    if (whole)                                       // one thread per component: no waits
      for (int q = 0; q < nbe; ++q) wt[(size_t)bevs[q]] = make_int4(0, 0, 0, 0);
    // owner threads in use, ascending; events grouped by them, input order within
    auto& slot_of_thr = W.slot_of_thr;
    auto& thr_ids = W.thr_ids;
    slot_of_thr.assign((size_t)kDfThreads, -1);
    thr_ids.clear();
    for (int t = 0; t < kDfThreads; ++t)
      if (load[(size_t)t] > 0) { slot_of_thr[(size_t)t] = (int32_t)thr_ids.size(); thr_ids.push_back(t); }
    const int nslot = (int)thr_ids.size();
    auto& off = W.off;
    off.assign((size_t)nslot + 1, 0);
    auto slot_of_ev = [&](int32_t i) {
      return slot_of_thr[(size_t)owner[(size_t)slot_of[node[by_pos[(size_t)(s0 + i)]]]]];
    };
    for (int q = 0; q < nbe; ++q) off[(size_t)slot_of_ev(bevs[q]) + 1]++;
    for (int q = 0; q < nslot; ++q) off[(size_t)q + 1] += off[(size_t)q];
    auto& fill = W.fill;
    fill.assign(off.begin(), off.end() - 1);
    const size_t base = S.rec_df.size();
    S.blk_meta.push_back(make_int4((int32_t)base, (int32_t)(tbase + (size_t)blk_t0[(size_t)b]),
                                   (int32_t)S.thr_off.size(), heavy | (whole ? (1 << 16) : 0)));
    S.rec_df.resize(base + (size_t)nb);
    S.wait_df.resize(base + (size_t)nb);
    for (int q = 0; q < nbe; ++q) {
      const int32_t i = bevs[q];
      const int32_t at = fill[(size_t)slot_of_ev(i)]++;
      S.rec_df[base + (size_t)at] = rec[(size_t)i];
      S.wait_df[base + (size_t)at] = wt[(size_t)i];
    }
    S.thr_off.insert(S.thr_off.end(), off.begin(), off.end());
    S.thr_id.insert(S.thr_id.end(), thr_ids.begin(), thr_ids.end());
    S.thr_id.push_back(-1);                          // aligned with thr_off
  }
}

// Runs fn(0) .. fn(n - 1), fn(0) on the calling thread and the others on threads of
// their own; false if a thread could not be started (those started are joined).
template <class F>
bool run_parallel(int n, F&& fn) {
  std::vector<std::thread> pool;
  bool ok = true;
  try {
    for (int p = 1; p < n; ++p) pool.emplace_back(fn, p);
  } catch (...) { ok = false; }
  if (ok && n > 0) fn(0);
  for (auto& t : pool) t.join();
  return ok;
}

// Schedules days [d0, d1): the execution-order records (rec, order, level,
// rec_slot; at their final positions) into S, the rest into the partial schedule P
// (day_lvl, day_touch and day_blk then hold one entry per day of the range, indices
// into P's own arrays).
void schedule_days(int32_t d0, int32_t d1, int N, const std::vector<int64_t>& first,
                   const std::vector<int64_t>& by_pos, const int32_t* kind, const int32_t* node,
                   const int32_t* dest, const int32_t* count, const int32_t* cls, int df_blocks,
                   std::vector<int32_t>& lvl_of, Schedule& P, Schedule& S) {
  std::vector<int32_t> slot_of(N, -1), slot_day(N, -1), last_s(N, 0), last_a(N, 0), stamp(N, -1);
  std::vector<int64_t> bucket;
  OwnerScratch scratch;
  for (int32_t d = d0; d < d1; ++d) {
    P.day_lvl.push_back((int32_t)P.lvl_start.size());
    P.day_touch.push_back((int32_t)P.touched.size());
    const int32_t touch0 = P.day_touch.back();
    auto slot = [&](int v) {
      if (slot_day[v] != d) { slot_day[v] = d; slot_of[v] = (int32_t)P.touched.size() - touch0; P.touched.push_back(v); }
      return slot_of[v];
    };
    const int64_t s0 = first[(size_t)d], s1 = first[(size_t)d + 1];
    int32_t max_lvl = 0;
    auto touch = [&](int v) { if (stamp[v] != d) { stamp[v] = d; last_s[v] = 0; last_a[v] = 0; } };
    for (int64_t s = s0; s < s1; ++s) {
      const int64_t e = by_pos[(size_t)s];
      const int k = kind[e], v = node[e];
      touch(v);
      int32_t L;
      if (k == SIM_ENTER) {
        L = last_s[v] + 1;
        if (L > last_a[v]) last_a[v] = L;
      } else {
        L = (last_s[v] > last_a[v] ? last_s[v] : last_a[v]) + 1;
        if (k == SIM_EXTERNAL) {
          const int w = dest[e];
          touch(w);
          if (last_s[w] + 1 > L) L = last_s[w] + 1;
          if (L > last_a[w]) last_a[w] = L;
        }
        last_s[v] = L;
      }
      lvl_of[(size_t)s] = L;
      if (L > max_lvl) max_lvl = L;
    }
    bucket.assign((size_t)max_lvl + 2, 0);
    for (int64_t s = s0; s < s1; ++s) bucket[(size_t)lvl_of[(size_t)s] + 1]++;
    for (int32_t L = 0; L <= max_lvl; ++L) bucket[(size_t)L + 1] += bucket[(size_t)L];
    for (int32_t L = 1; L <= max_lvl; ++L) P.lvl_start.push_back((int32_t)(s0 + bucket[(size_t)L]));
    for (int64_t s = s0; s < s1; ++s) {
      const int64_t e = by_pos[(size_t)s];
      const size_t slot = (size_t)(s0 + bucket[(size_t)lvl_of[(size_t)s]]++);
      const uint32_t packed = (uint32_t)kind[e] | ((uint32_t)(cls[e] + 1) << 2) | ((uint32_t)count[e] << 4);
      S.rec[slot] = make_int4(node[e], kind[e] == SIM_EXTERNAL ? dest[e] : -1, (int32_t)s, (int32_t)packed);
      S.order[slot] = s;
      S.level[slot] = lvl_of[(size_t)s];
    }
    for (int64_t k = s0; k < s1; ++k) {          // slots in execution order
      const int4 rc = S.rec[(size_t)k];
      const int32_t a = slot(rc.x);
      const int32_t b = rc.y >= 0 ? slot(rc.y) : -1;
      S.rec_slot[(size_t)k] = make_int4(a, b, rc.z, rc.w);
    }
    build_owner_form(P, s0, s1, touch0, by_pos, kind, node, dest, count, cls, slot_of, lvl_of, df_blocks, scratch);
  }
}

// Validates the events and builds the execution schedule: stable sort by day,
// then per day a dependency level for each event.  A sampling event on node v
// (exit, aging, transfer source) gets 1 + the highest level of any earlier event
// of the day touching v; an add to w (enter, transfer destination) gets 1 + the
// highest level of an earlier sampling of w; adds to one node commute and may
// share a level.  Within a level events keep their day-stable order.  Applying
// the levels in order, each level in any order, equals applying the events in
// input order.  O(n + max_days) time.
sim_status build_schedule(sim_handle* h, int N, int na, int32_t T, int64_t n, const int32_t* day,
                          const int32_t* kind, const int32_t* node, const int32_t* dest,
                          const int32_t* count, const int32_t* cls, int df_blocks, Schedule& S) {
  if (n < 0 || n >= ((int64_t)1 << 31)) return fail(h, SIM_E_INVALID_ARG, "event count out of range");
  if (n > 0 && (!day || !kind || !node || !dest || !count || !cls))
    return fail(h, SIM_E_INVALID_ARG, "null event array");
  int32_t dmax = T;
  for (int64_t e = 0; e < n; ++e) {
    const int k = kind[e];
    if (day[e] < 0) return fail(h, SIM_E_INVALID_ARG, "event %lld: day < 0", (long long)e);
    if (k < SIM_EXIT || k > SIM_EXTERNAL) return fail(h, SIM_E_INVALID_ARG, "event %lld: unknown kind %d", (long long)e, k);
    if (node[e] < 0 || node[e] >= N) return fail(h, SIM_E_INVALID_ARG, "event %lld: node %d out of range", (long long)e, node[e]);
    if (count[e] < 0 || count[e] >= (1 << 28)) return fail(h, SIM_E_INVALID_ARG, "event %lld: count %d out of range [0, 2^28)", (long long)e, count[e]);
    if (cls[e] < -1 || cls[e] >= na) return fail(h, SIM_E_INVALID_ARG, "event %lld: class %d out of range", (long long)e, cls[e]);
    if (k == SIM_INTERNAL && (cls[e] < 0 || cls[e] >= na - 1))
      return fail(h, SIM_E_INVALID_ARG, "event %lld: aging needs a class with a next class", (long long)e);
    if (k == SIM_EXTERNAL && (dest[e] < 0 || dest[e] >= N || dest[e] == node[e]))
      return fail(h, SIM_E_INVALID_ARG, "event %lld: bad destination %d", (long long)e, dest[e]);
    if (day[e] + 1 > dmax) dmax = day[e] + 1;
  }
  std::vector<int64_t> first, by_pos;
  std::vector<int32_t> lvl_of;
  try {
    first.assign((size_t)dmax + 1, 0);
    by_pos.resize((size_t)n);
    S.day_lvl.assign((size_t)T + 1, 0);
  } catch (...) { return fail(h, SIM_E_OOM, "host allocation"); }
  for (int64_t e = 0; e < n; ++e) first[(size_t)day[e] + 1]++;
  for (int32_t d = 0; d < dmax; ++d) first[(size_t)d + 1] += first[(size_t)d];
  {
    std::vector<int64_t> fill(first.begin(), first.end() - 1);
    for (int64_t e = 0; e < n; ++e) by_pos[(size_t)fill[(size_t)day[e]]++] = e;
  }
  const int64_t n_run = first[(size_t)T];          // events on days < max_days
  try {
    lvl_of.resize((size_t)n_run);
    S.rec.resize((size_t)n_run);
    S.order.resize((size_t)n_run);
    S.level.resize((size_t)n_run);
    S.rec_slot.resize((size_t)n_run);
    S.day_touch.assign((size_t)T + 1, 0);
  } catch (...) { return fail(h, SIM_E_OOM, "host allocation"); }
  // Days are independent: contiguous ranges of them, balanced by event count, are
  // scheduled on separate threads into partial schedules, which are then joined in
  // day order (their indices into the joined arrays shifted).  The records in
  // execution order go straight to their final positions.
  const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const int n_part = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, n_run / 65536 + 1, (int64_t)T}));
  std::vector<int32_t> part_d(n_part + 1, T);
  part_d[0] = 0;
  for (int p = 1, d = 0; p < n_part; ++p) {
    while (d < T && first[(size_t)d] < n_run * p / n_part) ++d;
    part_d[p] = std::max(d, part_d[p - 1]);
  }
  std::vector<Schedule> parts(n_part);
  std::vector<char> part_oom(n_part, 0);
  const bool threads_ok = run_parallel(n_part, [&](int p) {
    try {
      schedule_days(part_d[p], part_d[p + 1], N, first, by_pos, kind, node, dest, count, cls, df_blocks, lvl_of,
                    parts[p], S);
    } catch (...) { part_oom[p] = 1; }
  });
  if (!threads_ok) return fail(h, SIM_E_OOM, "host threads");
  for (int p = 0; p < n_part; ++p)
    if (part_oom[p]) return fail(h, SIM_E_OOM, "host allocation");
  // the join: each part's arrays at the offsets of the parts before it
  std::vector<size_t> o_lvl(n_part + 1, 0), o_tch(n_part + 1, 0), o_blk(n_part + 1, 0), o_rec(n_part + 1, 0),
      o_tdf(n_part + 1, 0), o_thr(n_part + 1, 0);
  for (int p = 0; p < n_part; ++p) {
    const Schedule& P = parts[p];
    o_lvl[p + 1] = o_lvl[p] + P.lvl_start.size();
    o_tch[p + 1] = o_tch[p] + P.touched.size();
    o_blk[p + 1] = o_blk[p] + P.blk_meta.size();
    o_rec[p + 1] = o_rec[p] + P.rec_df.size();
    o_tdf[p + 1] = o_tdf[p] + P.touched_df.size();
    o_thr[p + 1] = o_thr[p] + P.thr_off.size();
  }
  if (o_tdf[n_part] >= ((size_t)1 << 31) || o_thr[n_part] >= ((size_t)1 << 31))
    return fail(h, SIM_E_INVALID_ARG, "event schedule exceeds 32-bit indices");
  try {
    S.lvl_start.resize(o_lvl[n_part]);
    S.touched.resize(o_tch[n_part]);
    S.day_blk.resize((size_t)T);
    S.blk_meta.resize(o_blk[n_part]);
    S.rec_df.resize(o_rec[n_part]);
    S.wait_df.resize(o_rec[n_part]);
    S.touched_df.resize(o_tdf[n_part]);
    S.thr_off.resize(o_thr[n_part]);
    S.thr_id.resize(o_thr[n_part]);
  } catch (...) { return fail(h, SIM_E_OOM, "host allocation"); }
  const bool join_ok = run_parallel(n_part, [&](int p) {
    Schedule& P = parts[p];
    for (int32_t d = part_d[p]; d < part_d[p + 1]; ++d) {
      const size_t i = (size_t)(d - part_d[p]);
      S.day_lvl[d] = P.day_lvl[i] + (int32_t)o_lvl[p];
      S.day_touch[d] = P.day_touch[i] + (int32_t)o_tch[p];
      S.day_blk[d] = P.day_blk[i] + (int32_t)o_blk[p];
    }
    std::copy(P.lvl_start.begin(), P.lvl_start.end(), S.lvl_start.begin() + o_lvl[p]);
    std::copy(P.touched.begin(), P.touched.end(), S.touched.begin() + o_tch[p]);
    std::copy(P.rec_df.begin(), P.rec_df.end(), S.rec_df.begin() + o_rec[p]);
    std::copy(P.wait_df.begin(), P.wait_df.end(), S.wait_df.begin() + o_rec[p]);
    std::copy(P.touched_df.begin(), P.touched_df.end(), S.touched_df.begin() + o_tdf[p]);
    std::copy(P.thr_off.begin(), P.thr_off.end(), S.thr_off.begin() + o_thr[p]);
    std::copy(P.thr_id.begin(), P.thr_id.end(), S.thr_id.begin() + o_thr[p]);
    for (size_t b = 0; b < P.blk_meta.size(); ++b) {
      const int4 m = P.blk_meta[b];
      S.blk_meta[o_blk[p] + b] = make_int4(m.x + (int32_t)o_rec[p], m.y + (int32_t)o_tdf[p], m.z + (int32_t)o_thr[p], m.w);
    }
    P = Schedule();
  });
  if (!join_ok) return fail(h, SIM_E_OOM, "host threads");
  S.day_lvl[T] = (int32_t)S.lvl_start.size();
  S.day_touch[T] = (int32_t)S.touched.size();
  S.lvl_start.push_back((int32_t)n_run);
  S.day_blk.push_back((int32_t)S.blk_meta.size());
  S.blk_meta.push_back(make_int4((int32_t)S.rec_df.size(), (int32_t)S.touched_df.size(), (int32_t)S.thr_off.size(), 0));
  return SIM_OK;
}

// Launches `fn` on `st`, bracketed by a pair of pooled CUDA events when tracing.
template <class F>
cudaError_t traced(sim_handle* h, int kind, cudaStream_t st, F&& fn) {
  if (!h->profiling) return fn();
  if (h->ev_used + 2 > h->ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      h->ev_pool.push_back(e);
    }
  }
  // under stream capture the records must be external to become event-record nodes
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(st, &cap);
  if (err != cudaSuccess) return err;
  const unsigned flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  err = cudaEventRecordWithFlags(h->ev_pool[h->ev_used], st, flags);
  if (err != cudaSuccess) return err;
  err = fn();
  if (err != cudaSuccess) return err;
  err = cudaEventRecordWithFlags(h->ev_pool[h->ev_used + 1], st, flags);
  h->ev_used += 2;
  h->ev_kind.push_back(kind);
  return err;
}

}  // namespace

namespace episim {
sim_status handle_score_view(sim_handle* h, HandleScoreView* out) {
  if (!h->d_score) return fail(h, SIM_E_STATE, "created without SIM_FLAG_SCORE");
  out->score = h->d_score; out->prev_i = h->d_prev_i; out->prev_n = h->d_prev_n;
  out->N = h->cfg.n_nodes; out->R = h->cfg.n_replicates; out->max_days = h->cfg.max_days;
  return SIM_OK;
}
sim_status handle_fail(sim_handle* h, sim_status s, const char* msg) { return fail(h, s, "%s", msg); }
sim_status handle_cuda_fail(sim_handle* h, cudaError_t e, const char* what) { return cuda_fail(h, e, what); }
sim_status handle_check_latched(sim_handle* h) { return check_latched(h); }
}  // namespace episim

extern "C" {

namespace {

// Caller device memory for the state: on the current device, 16-byte aligned.
bool usable_device_buffer(const void* ptr) {
  if (!ptr || ((uintptr_t)ptr & 15u)) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

sim_status create_impl(const sim_config* cfg, const int32_t* u0, const double* phi0, const sim_params* p,
                       int32_t* dev_counts, double* dev_phi, sim_handle** out);

}  // namespace

sim_status sim_create(const sim_config* cfg, const int32_t* u0, const double* phi0,
                      const sim_params* p, sim_handle** out) {
  return create_impl(cfg, u0, phi0, p, nullptr, nullptr, out);
}

sim_status sim_create_on(const sim_config* cfg, const int32_t* u0, const double* phi0, const sim_params* p,
                         int32_t* dev_counts, double* dev_phi, void* stream, sim_handle** out) {
  if (!dev_counts || !dev_phi) return fail(nullptr, SIM_E_INVALID_ARG, "dev_counts and dev_phi are required");
  if (!usable_device_buffer(dev_counts) || !usable_device_buffer(dev_phi))
    return fail(nullptr, SIM_E_INVALID_ARG, "dev_counts / dev_phi must be 16-byte aligned device memory of the current device");
  // the caller's earlier work on its buffers completes before the library writes them
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronize");
  return create_impl(cfg, u0, phi0, p, dev_counts, dev_phi, out);
}

namespace {

sim_status create_impl(const sim_config* cfg, const int32_t* u0, const double* phi0, const sim_params* p,
                       int32_t* dev_counts, double* dev_phi, sim_handle** out) {
  if (!cfg || !u0 || !phi0 || !p || !out) return fail(nullptr, SIM_E_INVALID_ARG, "null argument");
  if (cfg->model != SIM_SISE && cfg->model != SIM_SISE3)
    return fail(nullptr, SIM_E_INVALID_ARG, "model must be SIM_SISE (1) or SIM_SISE3 (3)");
  if (cfg->n_nodes < 1 || cfg->n_replicates < 1 || cfg->max_days < 0)
    return fail(nullptr, SIM_E_INVALID_ARG, "n_nodes, n_replicates must be >= 1 and max_days >= 0");
  if (cfg->underflow_policy != SIM_UNDERFLOW_CLAMP && cfg->underflow_policy != SIM_UNDERFLOW_ERROR)
    return fail(nullptr, SIM_E_INVALID_ARG, "unknown underflow policy");
  if (cfg->flags & ~(SIM_FLAG_PHI_PRE_EVENT | SIM_FLAG_SCORE | SIM_FLAG_SCORE_REVERSE))
    return fail(nullptr, SIM_E_INVALID_ARG, "unknown flag bits");
  if (cfg->replicate_base < 0 || (int64_t)cfg->replicate_base + cfg->n_replicates > ((int64_t)1 << 32) ||
      cfg->reserved != 0)
    return fail(nullptr, SIM_E_INVALID_ARG, "replicate_base out of range or reserved field set");
  if (!p->upsilon || !p->gamma || !p->alpha || !p->beta || !p->epsilon)
    return fail(nullptr, SIM_E_INVALID_ARG, "null parameter array");
  sim_handle* h = new (std::nothrow) sim_handle();
  if (!h) return fail(nullptr, SIM_E_OOM, "host allocation");
  h->cfg = *cfg;
  if (h->cfg.flags & SIM_FLAG_SCORE_REVERSE) h->cfg.flags |= SIM_FLAG_SCORE;
  h->n_age = cfg->model == SIM_SISE3 ? 3 : 1;
  h->nc = 2 * h->n_age;
  const int N = cfg->n_nodes, R = cfg->n_replicates;
  try {
    h->u0.assign(u0, u0 + (size_t)h->nc * N);
    h->phi0.assign(phi0, phi0 + N);
    h->params.resize(R);
  } catch (...) {
    delete h;
    return fail(nullptr, SIM_E_OOM, "host allocation");
  }
  for (size_t i = 0; i < h->u0.size(); ++i)
    if (h->u0[i] < 0) { delete h; return fail(nullptr, SIM_E_INVALID_ARG, "u0[%zu] < 0", i); }
  for (int v = 0; v < N; ++v) {
    int64_t tot = 0;
    for (int c = 0; c < h->nc; ++c) tot += h->u0[(size_t)c * N + v];
    if (tot > (1 << 30)) { delete h; return fail(nullptr, SIM_E_INVALID_ARG, "node %d holds more than 2^30 animals", v); }
    if (!finite_nonneg(phi0[v])) { delete h; return fail(nullptr, SIM_E_INVALID_ARG, "phi0[%d] must be finite and >= 0", v); }
  }
  {
    const sim_status ps = fill_params(h, nullptr, p, h->params);
    if (ps != SIM_OK) { delete h; return ps; }
  }
  cudaError_t e = cudaSuccess;
  {
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    h->sm_count = sms > 0 ? sms : 1;
  }
  const size_t stats = (size_t)R * (cfg->max_days > 0 ? cfg->max_days : 1);
  if (dev_counts) {
    h->owns_state = false;
    h->d_counts = dev_counts;
    h->d_phi = dev_phi;
  } else {
    if (e == cudaSuccess) e = dalloc(&h->d_counts, n_counts(h));
    if (e == cudaSuccess) e = dalloc(&h->d_phi, n_phi(h));
  }
  if (e == cudaSuccess) e = dalloc(&h->d_params, (size_t)R);
  if (e == cudaSuccess) e = dalloc(&h->d_prev_i, stats);
  if (e == cudaSuccess) e = dalloc(&h->d_prev_n, stats);
  if (e == cudaSuccess) e = dalloc(&h->d_ctr, (size_t)R * 4);
  if (e == cudaSuccess) e = dalloc(&h->d_err, 1);
  if (e == cudaSuccess) e = dalloc(&h->d_u0, h->u0.size());
  if (e == cudaSuccess) e = dalloc(&h->d_phi0, h->phi0.size());
  if (e == cudaSuccess && (h->cfg.flags & SIM_FLAG_SCORE)) {
    e = dalloc(&h->d_score, n_phi(h) * kScoreTerms);
    if (e == cudaSuccess) e = dalloc(&h->d_tang, n_phi(h) * 2);
    if (e == cudaSuccess) e = dalloc(&h->d_per_rep, (size_t)R * kScoreTerms);
  }
  if (e == cudaSuccess && (h->cfg.flags & SIM_FLAG_SCORE_REVERSE))
    e = dalloc(&h->d_traj, (size_t)3 * (cfg->max_days > 0 ? cfg->max_days : 1) * n_phi(h));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_params, h->params.data(), R * sizeof(DevParams), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_u0, h->u0.data(), h->u0.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_phi0, h->phi0.data(), h->phi0.size() * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    sim_status s = cuda_fail(nullptr, e, "device allocation / upload");
    free_all(h);
    delete h;
    return s;
  }
  h->node_lo = 0;
  h->node_hi = N;
  sim_status s = reset_state(h);
  if (s == SIM_OK) s = set_order(h, -1);
  if (s != SIM_OK) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return SIM_OK;
}

}  // namespace

sim_status sim_load_events(sim_handle* h, int64_t n, const int32_t* day, const int32_t* kind,
                           const int32_t* node, const int32_t* dest, const int32_t* count,
                           const int32_t* cls) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->events_loaded) return fail(h, SIM_E_STATE, "events already loaded (sim_reset(h, 1) drops them)");
  if (h->day != 0) return fail(h, SIM_E_STATE, "events must be loaded at day 0");
  Schedule S;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  // owner-computes blocks per replicate and day: enough to spread one replicate
  // over the SMs (two 256-thread blocks fit on one), one per replicate once the
  // replicates fill them
  const int df_blocks = std::max(1, 2 * sms / std::max(1, h->cfg.n_replicates));
  sim_status st = build_schedule(h, h->cfg.n_nodes, h->n_age, h->cfg.max_days, n, day, kind, node, dest,
                                 count, cls, df_blocks, S);
  if (st != SIM_OK) return st;
  free_events(h);
  const int32_t T = h->cfg.max_days;
  cudaError_t err = cudaSuccess;
  if (err == cudaSuccess) err = dalloc(&h->d_rec, S.rec.size());
  if (err == cudaSuccess) err = dalloc(&h->d_lvl_start, S.lvl_start.size());
  if (err == cudaSuccess) err = dalloc(&h->d_day_lvl, (size_t)T + 1);
  if (err == cudaSuccess && !S.rec.empty()) err = cudaMemcpy(h->d_rec, S.rec.data(), S.rec.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(h->d_lvl_start, S.lvl_start.data(), S.lvl_start.size() * 4, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(h->d_day_lvl, S.day_lvl.data(), S.day_lvl.size() * 4, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = dalloc(&h->d_rec_slot, S.rec_slot.size());
  if (err == cudaSuccess) err = dalloc(&h->d_touched, S.touched.size());
  if (err == cudaSuccess) err = dalloc(&h->d_day_touch, S.day_touch.size());
  if (err == cudaSuccess && !S.rec_slot.empty()) err = cudaMemcpy(h->d_rec_slot, S.rec_slot.data(), S.rec_slot.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && !S.touched.empty()) err = cudaMemcpy(h->d_touched, S.touched.data(), S.touched.size() * 4, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(h->d_day_touch, S.day_touch.data(), S.day_touch.size() * 4, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) { free_events(h); return cuda_fail(h, err, "event upload"); }
  {
    auto up = [&](auto** dst, const auto& v, size_t elem) {
      if (err == cudaSuccess) err = dalloc(dst, v.size());
      if (err == cudaSuccess && !v.empty()) err = cudaMemcpy(*dst, v.data(), v.size() * elem, cudaMemcpyHostToDevice);
    };
    up(&h->d_rec_df, S.rec_df, sizeof(int4));
    up(&h->d_wait_df, S.wait_df, sizeof(int4));
    up(&h->d_thr_off, S.thr_off, 4);
    up(&h->d_touched_df, S.touched_df, 4);
    up(&h->d_blk_meta, S.blk_meta, sizeof(int4));
    up(&h->d_thr_id, S.thr_id, 4);
    if (err != cudaSuccess) { free_events(h); return cuda_fail(h, err, "event upload"); }
    // shared memory of a day's launch: its largest block (0: owner-computes not used)
    h->day_df.assign((size_t)T, 0);
    h->day_nblk.assign((size_t)T, 0);
    h->day_blk0.assign((size_t)T, 0);
    for (int32_t d = 0; d < T; ++d) {
      const int32_t b0 = S.day_blk[(size_t)d], b1 = S.day_blk[(size_t)d + 1];
      size_t most = 0;
      for (int32_t b = b0; b < b1; ++b) {
        const int64_t ne = S.blk_meta[(size_t)b + 1].x - S.blk_meta[(size_t)b].x;
        const int64_t nt = S.blk_meta[(size_t)b + 1].y - S.blk_meta[(size_t)b].y;
        most = std::max(most, events_df_smem_bytes(ne, nt, h->nc));
      }
      h->day_nblk[(size_t)d] = b1 - b0;
      h->day_blk0[(size_t)d] = b0;
      h->day_df[(size_t)d] = (most <= kEventsSmemLimit) ? (int32_t)most : 0;
    }
  }
  h->day_smem.assign((size_t)T, 0);
  for (int32_t d = 0; d < T; ++d) {
    const int64_t nl = S.day_lvl[(size_t)d + 1] - S.day_lvl[(size_t)d];
    const int64_t ne = S.lvl_start[(size_t)S.day_lvl[(size_t)d + 1]] - S.lvl_start[(size_t)S.day_lvl[(size_t)d]];
    const int64_t nt = S.day_touch[(size_t)d + 1] - S.day_touch[(size_t)d];
    const size_t b = events_smem_bytes(ne, nl, nt, h->nc);
    h->day_smem[(size_t)d] = (b <= kEventsSmemLimit && !h->force_global_events) ? (int32_t)b : 0;
  }
  {
    cudaError_t e2 = dalloc(&h->d_day_smem, (size_t)T);
    if (e2 == cudaSuccess && T > 0) e2 = cudaMemcpy(h->d_day_smem, h->day_smem.data(), (size_t)T * 4, cudaMemcpyHostToDevice);
    if (e2 != cudaSuccess) { free_events(h); return cuda_fail(h, e2, "event upload"); }
  }
  // the events of the run's days in day-stable order, for the dataflow schedule
  try {
    h->ev_first.assign((size_t)T + 1, 0);
    for (int64_t e = 0; e < n; ++e)
      if (day[e] < T) h->ev_first[(size_t)day[e] + 1]++;
    for (int32_t d = 0; d < T; ++d) h->ev_first[(size_t)d + 1] += h->ev_first[(size_t)d];
    h->ev_host.resize((size_t)h->ev_first[(size_t)T]);
    std::vector<int64_t> fill(h->ev_first.begin(), h->ev_first.end() - 1);
    for (int64_t e = 0; e < n; ++e) {
      if (day[e] >= T) continue;
      const int64_t s = fill[(size_t)day[e]]++;
      const uint32_t packed = (uint32_t)kind[e] | ((uint32_t)(cls[e] + 1) << 2) | ((uint32_t)count[e] << 4);
      h->ev_host[(size_t)s] = make_int4(node[e], kind[e] == SIM_EXTERNAL ? dest[e] : -1, (int32_t)s, (int32_t)packed);
    }
  } catch (...) { free_events(h); return fail(h, SIM_E_OOM, "host allocation"); }
  h->sched_order.swap(S.order);
  h->sched_level.swap(S.level);
  h->day_lvl.swap(S.day_lvl);
  h->touched_host.swap(S.touched);
  h->day_touch_host.swap(S.day_touch);
  h->events_loaded = true;
  free_graph(h);
  return build_split(h);
}

sim_status sim_schedule_events(int32_t n_nodes, int32_t model, int32_t max_days, int64_t n,
                               const int32_t* day, const int32_t* kind, const int32_t* node,
                               const int32_t* dest, const int32_t* count, const int32_t* cls,
                               int64_t* order, int32_t* level, int64_t* n_scheduled) {
  if (n_nodes < 1 || max_days < 0 || (model != SIM_SISE && model != SIM_SISE3))
    return fail(nullptr, SIM_E_INVALID_ARG, "bad n_nodes / model / max_days");
  Schedule S;
  sim_status st = build_schedule(nullptr, n_nodes, model == SIM_SISE3 ? 3 : 1, max_days, n, day, kind,
                                 node, dest, count, cls, 1, S);
  if (st != SIM_OK) return st;
  if (order) std::memcpy(order, S.order.data(), S.order.size() * 8);
  if (level) std::memcpy(level, S.level.data(), S.level.size() * 4);
  if (n_scheduled) *n_scheduled = (int64_t)S.order.size();
  return SIM_OK;
}

}  // extern "C"

extern "C" {

// Enqueues the launches of days [d0, d0 + ndays) on st (no state change).
// Arguments of the three event-step kernels of a handle.
struct DayEventArgs {
  EvArgs ev;
  EvSmemArgs es;
  EvDfArgs df;
};

static DayEventArgs day_event_args(sim_handle* h) {
  DayEventArgs E{};
  EvArgs& ev = E.ev;
  EvSmemArgs& es = E.es;
  EvDfArgs& df = E.df;
  ev.counts = h->d_counts; ev.rec = h->d_rec; ev.lvl_start = h->d_lvl_start; ev.day_lvl = h->d_day_lvl;
  ev.ctr = h->d_ctr; ev.err = h->d_err; ev.seed = h->cfg.seed; ev.rep_base = h->cfg.replicate_base;
  ev.N = h->cfg.n_nodes; ev.R = h->cfg.n_replicates; ev.Nc = h->nc;
  ev.underflow_error = h->cfg.underflow_policy == SIM_UNDERFLOW_ERROR;
  es.counts = h->d_counts; es.rec = h->d_rec_slot; es.lvl_start = h->d_lvl_start; es.day_lvl = h->d_day_lvl;
  es.touched = h->d_touched; es.day_touch = h->d_day_touch; es.ctr = h->d_ctr; es.err = h->d_err;
  es.seed = h->cfg.seed; es.rep_base = h->cfg.replicate_base;
  es.N = h->cfg.n_nodes; es.R = h->cfg.n_replicates; es.Nc = h->nc; es.underflow_error = ev.underflow_error;
  df.counts = h->d_counts; df.rec = h->d_rec_df; df.wait = h->d_wait_df; df.thr_off = h->d_thr_off;
  df.touched = h->d_touched_df; df.blk_meta = h->d_blk_meta; df.thr_id = h->d_thr_id; df.ctr = h->d_ctr;
  df.err = h->d_err; df.seed = h->cfg.seed; df.rep_base = h->cfg.replicate_base;
  df.N = h->cfg.n_nodes; df.R = h->cfg.n_replicates; df.Nc = h->nc; df.underflow_error = ev.underflow_error;
  df.spin_limit = 1 << 24;
  df.overlap = h->overlap;
  return E;
}

// The event step of day d (nothing when the day has no events): the
// owner-computes kernel where the day's largest block fits in shared memory,
// else the level-staged kernel, else the global-memory one.
static sim_status launch_day_events(sim_handle* h, DayEventArgs& E, int32_t d, cudaStream_t st) {
  if (!(h->events_loaded && h->day_lvl[(size_t)d + 1] > h->day_lvl[(size_t)d])) return SIM_OK;
  if (h->event_variant == 0 && h->day_df[(size_t)d] > 0) {
    E.df.day = d;
    E.df.nblk = h->day_nblk[(size_t)d];
    E.df.blk0 = h->day_blk0[(size_t)d];
    E.df.smem_bytes = h->day_df[(size_t)d];
    CK(h, traced(h, 1, st, [&] { return launch_events_day_df(E.df, h->n_age, st); }), "event step launch");
  } else if (h->event_variant != 1 && h->day_smem[(size_t)d] > 0) {
    E.es.day = d;
    E.es.smem_bytes = h->day_smem[(size_t)d];
    CK(h, traced(h, 1, st, [&] { return launch_events_day_smem(E.es, h->n_age, st); }), "event step launch");
  } else {
    E.ev.day = d;
    CK(h, traced(h, 1, st, [&] { return launch_events_day(E.ev, h->n_age, st); }), "event step launch");
  }
  return SIM_OK;
}

static sim_status enqueue_days(sim_handle* h, int32_t d0, int32_t ndays, cudaStream_t st) {
  const bool score = (h->cfg.flags & SIM_FLAG_SCORE) != 0;
  SsaArgs a = ssa_args(h);
  DayEventArgs E = day_event_args(h);
  // Split day step: after a day d with events, the stochastic step of day d + 1
  // runs as two launches -- the herds d's events leave untouched, on the side
  // stream as soon as day d's stochastic step is complete (alongside d's event
  // step), and the touched herds after the event step; the side launch is joined
  // before the event step of day d + 1.  Without events the day is one launch.
  const bool split = h->split && !score && h->events_loaded && h->d_skip && h->d_tlist && h->n_regions == 0 &&
                     h->node_lo == 0 && h->node_hi == h->cfg.n_nodes;
  const size_t words = ((size_t)h->cfg.n_nodes + 31) / 32;
  if (split && !h->side) {
    CK(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "side stream");
    CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "fork event");
    CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "join event");
  }
  auto has_events = [&](int32_t d) { return h->events_loaded && h->day_lvl[(size_t)d + 1] > h->day_lvl[(size_t)d]; };
  for (int32_t d = d0; d < d0 + ndays; ++d) {
    a.day = d;
    a.prologue = d > d0;
    if (split && d > d0 && has_events(d - 1)) {
      // touched herds of day d - 1 (the untouched ones were launched on the side stream)
      SsaArgs at = a;
      const int32_t b0 = h->day_touch_host[(size_t)d - 1], b1 = h->day_touch_host[(size_t)d];
      at.order = h->d_tlist + b0;
      at.n_list = b1 - b0;
      at.n_big = h->tlist_nbig[(size_t)d - 1];
      at.n_mid = h->tlist_nmid[(size_t)d - 1];
      if (at.n_list > 0)
        CK(h, traced(h, 0, st, [&] { return launch_ssa_day(at, h->n_age, score, st); }), "stochastic step launch");
      CK(h, cudaStreamWaitEvent(st, h->ev_join, 0), "join");
    } else {
      CK(h, traced(h, 0, st, [&] { return launch_ssa_day(a, h->n_age, score, st); }), "stochastic step launch");
    }
    if (split && d + 1 < d0 + ndays && has_events(d)) {
      CK(h, cudaEventRecord(h->ev_fork, st), "fork");
      CK(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0), "fork");
      SsaArgs au = a;
      au.day = d + 1;
      au.prologue = 1;
      au.skip = h->d_skip + (size_t)d * words;
      au.overlap = 0;                                // after an event wait: plain stream order
      au.max_per_sm = 1;                             // one block of up to 12 warps per SM: with
      au.max_warps = 12;                             // 128 registers a thread, room for an event block
      CK(h, traced(h, 0, h->side, [&] { return launch_ssa_day(au, h->n_age, score, h->side); }),
         "stochastic step launch");
      CK(h, cudaEventRecord(h->ev_join, h->side), "join");
    }
    {
      const sim_status es = launch_day_events(h, E, d, st);
      if (es != SIM_OK) return es;
    }
    if (h->n_regions > 0)                            // region totals of the state after day d
      CK(h, launch_region_day(h->d_counts, h->d_reg_nodes, h->d_reg_off, h->cfg.n_nodes, h->cfg.n_replicates,
                              h->nc, h->n_regions, d, h->d_s1, h->d_s2, st), "region statistics launch");
  }
  a.day = d0 + ndays - 1;
  CK(h, traced(h, 2, st, [&] { return launch_finalize(a, h->n_age, score, st); }), "phi update launch");
  return SIM_OK;
}

// Dataflow schedule: per day, the connected components of the day's transfer
// graph (union-find over the herds the events name), longest first (ties by first
// event); per component its herds in order of first appearance (their slots) and
// its events in day-stable order as {src slot, dst slot, position, packed}.
static sim_status build_flow(sim_handle* h) {
  free_flow(h);
  const int N = h->cfg.n_nodes;
  const int32_t T = h->cfg.max_days;
  std::vector<int4> rec;
  std::vector<int32_t> cev(1, 0), cnode, cnoff(1, 0), cunit, cuoff(1, 0);
  std::vector<int32_t> day_comp((size_t)T + 1, 0), day_long((size_t)std::max<int32_t>(T, 1), 0);
  // the stochastic-step unit of every herd of the node order (warp herds one each,
  // group herds four to a unit, thread herds 32 to a unit)
  const int nb = h->n_big, nm = h->n_mid, no = h->n_order;
  const int U1 = nb + (nm + 3) / 4 + (no - nb - nm + 31) / 32;
  std::vector<int32_t> K;
  try {
    std::vector<int32_t> unit_of(N, -1), ustamp((size_t)std::max(U1, 1), -1), kday((size_t)std::max(U1, 1), 0);
    for (int i = 0; i < no; ++i) {
      const int v = h->order_host[(size_t)i];
      unit_of[v] = i < nb ? i : (i < nb + nm ? nb + (i - nb) / 4 : nb + (nm + 3) / 4 + (i - nb - nm) / 32);
    }
    K.assign(((size_t)T + 1) * (size_t)U1, 0);
    rec.reserve(h->ev_host.size());
    std::vector<int32_t> stamp(N, -1), local(N, 0), slot_of(N, -1);
    std::vector<int32_t> par, first_ev, comp_of_root, ev_comp, order, count, fill, nodes_of;
    std::vector<int32_t> lnode;                    // local index -> herd
    for (int32_t d = 0; d < T; ++d) {
      day_comp[(size_t)d] = (int32_t)(cev.size() - 1);
      if (d > 0)
        for (int u = 0; u < U1; ++u) {
          K[(size_t)d * U1 + u] = K[(size_t)(d - 1) * U1 + u] + kday[(size_t)u];
          kday[(size_t)u] = 0;
        }
      if (h->ev_first.empty()) continue;
      const int64_t s0 = h->ev_first[(size_t)d], s1 = h->ev_first[(size_t)d + 1];
      const int n = (int)(s1 - s0);
      if (n == 0) continue;
      lnode.clear();
      par.clear();
      auto loc = [&](int v) {
        if (stamp[v] != d) { stamp[v] = d; local[v] = (int32_t)lnode.size(); lnode.push_back(v); par.push_back(local[v]); }
        return local[v];
      };
      auto find = [&](int x) {
        while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
        return x;
      };
      for (int64_t s = s0; s < s1; ++s) {
        const int4 e = h->ev_host[(size_t)s];
        const int a = loc(e.x);
        if (e.y >= 0) {
          const int b = loc(e.y);
          const int ra = find(a), rb = find(b);
          if (ra != rb) par[std::max(ra, rb)] = std::min(ra, rb);
        }
      }
      // components in order of first event; event counts
      comp_of_root.assign(lnode.size(), -1);
      ev_comp.resize((size_t)n);
      count.clear();
      first_ev.clear();
      for (int i = 0; i < n; ++i) {
        const int rt = find(local[h->ev_host[(size_t)(s0 + i)].x]);
        if (comp_of_root[rt] < 0) { comp_of_root[rt] = (int32_t)count.size(); count.push_back(0); first_ev.push_back(i); }
        ev_comp[(size_t)i] = comp_of_root[rt];
        count[(size_t)comp_of_root[rt]]++;
      }
      const int nc = (int)count.size();
      order.resize((size_t)nc);
      for (int c = 0; c < nc; ++c) order[(size_t)c] = c;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return count[a] > count[b]; });
      // rank of each component in the sorted order, then the events bucketed by rank
      std::vector<int32_t> rank((size_t)nc);
      for (int c = 0; c < nc; ++c) rank[(size_t)order[(size_t)c]] = c;
      fill.assign((size_t)nc + 1, 0);
      for (int c = 0; c < nc; ++c) fill[(size_t)rank[(size_t)c] + 1] = count[(size_t)c];
      for (int c = 0; c < nc; ++c) fill[(size_t)c + 1] += fill[(size_t)c];
      std::vector<int32_t> evs((size_t)n);
      {
        std::vector<int32_t> f2(fill.begin(), fill.end() - 1);
        for (int i = 0; i < n; ++i) evs[(size_t)f2[(size_t)rank[(size_t)ev_comp[(size_t)i]]]++] = i;
      }
      for (int c = 0; c < nc; ++c) day_long[(size_t)d] += count[(size_t)order[(size_t)c]] >= kFlowLong ? 1 : 0;
      for (int c = 0; c < nc; ++c) {
        const int32_t nbase = (int32_t)cnode.size();
        int32_t k = 0;
        for (int32_t j = fill[(size_t)c]; j < fill[(size_t)c + 1]; ++j) {
          const int4 e = h->ev_host[(size_t)(s0 + evs[(size_t)j])];
          auto slot = [&](int v) {
            if (slot_of[v] < 0 || slot_of[v] >= k || cnode[(size_t)(nbase + slot_of[v])] != v) {
              slot_of[v] = k++;
              cnode.push_back(v);
            }
            return slot_of[v];
          };
          const int sx = slot(e.x);
          const int sy = e.y >= 0 ? slot(e.y) : -1;
          rec.push_back(make_int4(sx, sy, e.z, e.w));
        }
        cev.push_back((int32_t)rec.size());
        cnoff.push_back((int32_t)cnode.size());
        // the component's distinct units; each counts once towards the next day
        const int32_t cid = (int32_t)cev.size() - 2;
        for (int32_t j = nbase; j < (int32_t)cnode.size(); ++j) {
          const int u = unit_of[cnode[(size_t)j]];
          if (ustamp[(size_t)u] != cid) { ustamp[(size_t)u] = cid; cunit.push_back(u); kday[(size_t)u]++; }
        }
        cuoff.push_back((int32_t)cunit.size());
      }
    }
    day_comp[(size_t)T] = (int32_t)(cev.size() - 1);
    if (T > 0)
      for (int u = 0; u < U1; ++u) K[(size_t)T * U1 + u] = K[(size_t)(T - 1) * U1 + u] + kday[(size_t)u];
  } catch (...) { return fail(h, SIM_E_OOM, "host allocation"); }
  if (rec.size() >= ((size_t)1 << 31) || cnode.size() >= ((size_t)1 << 31))
    return fail(h, SIM_E_INVALID_ARG, "dataflow schedule exceeds 32-bit indices");
  cudaError_t err = cudaSuccess;
  auto up = [&](auto** dst, const auto& v, size_t elem) {
    if (err == cudaSuccess) err = dalloc(dst, std::max<size_t>(v.size(), 1));
    if (err == cudaSuccess && !v.empty()) err = cudaMemcpy(*dst, v.data(), v.size() * elem, cudaMemcpyHostToDevice);
  };
  up(&h->d_fl_rec, rec, sizeof(int4));
  up(&h->d_fl_cev, cev, 4);
  up(&h->d_fl_cnode, cnode, 4);
  up(&h->d_fl_cnoff, cnoff, 4);
  up(&h->d_fl_day_comp, day_comp, 4);
  up(&h->d_fl_day_long, day_long, 4);
  up(&h->d_fl_cunit, cunit, 4);
  up(&h->d_fl_cuoff, cuoff, 4);
  up(&h->d_fl_K, K, 4);
  if (err == cudaSuccess) err = dalloc(&h->d_rdy, (size_t)h->cfg.n_replicates * std::max(U1, 1));
  if (err == cudaSuccess && !h->d_flow_next) err = dalloc(&h->d_flow_next, 1);
  if (err == cudaSuccess && !h->d_flow_abort) err = dalloc(&h->d_flow_abort, 1);
  if (err != cudaSuccess) { free_flow(h); return cuda_fail(h, err, "dataflow schedule upload"); }
  h->flow_day_comp.swap(day_comp);
  h->flow_day_long.swap(day_long);
  h->flow_U1 = U1;
  h->flow_built = true;
  return SIM_OK;
}

// Whether sim_run_days can take the dataflow loop (else it falls back to stream
// launches): not in score mode, with region statistics, or on a node range.
static bool flow_usable(const sim_handle* h) {
  return !(h->cfg.flags & SIM_FLAG_SCORE) && h->n_regions == 0 && h->node_lo == 0 &&
         h->node_hi == h->cfg.n_nodes;
}

// Days [d0, d0 + ndays) as one dataflow launch, then the phi update and statistics
// of the last day.  stall (test hook): the first unit's first wait (replicate 0)
// asks for a count that is never reached, so that it runs out.
static sim_status enqueue_flow(sim_handle* h, int32_t d0, int32_t ndays, cudaStream_t st, long long spin_limit,
                               bool stall = false) {
  if (!h->flow_built) {
    const sim_status s = build_flow(h);
    if (s != SIM_OK) return s;
  }
  const int R = h->cfg.n_replicates;
  const long long units = (long long)R * (h->n_big + (h->n_mid + 3) / 4 + (h->n_order - h->n_big - h->n_mid + 31) / 32);
  std::vector<long long> item_off((size_t)ndays + 1, 0);
  for (int32_t k = 0; k < ndays; ++k) {
    const int32_t d = d0 + k;
    const long long nc = h->flow_day_comp[(size_t)d + 1] - h->flow_day_comp[(size_t)d];
    const long long nl = h->flow_day_long[(size_t)d];
    item_off[(size_t)k + 1] = item_off[(size_t)k] + units + (long long)R * (nl + (nc - nl + 31) / 32);
  }
  if (ndays + 1 > h->item_cap) {
    CK(h, cudaStreamSynchronize(st), "stream synchronize");
    cudaFree(h->d_item_off);
    h->d_item_off = nullptr;
    h->item_cap = 0;
    CK(h, dalloc(&h->d_item_off, (size_t)ndays + 1), "item table allocation");
    h->item_cap = ndays + 1;
  }
  // a synchronous copy: the host table goes away when this call returns, and an
  // earlier launch may still read the device table
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  CK(h, cudaMemcpy(h->d_item_off, item_off.data(), item_off.size() * sizeof(long long), cudaMemcpyHostToDevice),
     "item table upload");
  FlowArgs f{};
  f.a.ssa = ssa_args(h);
  f.a.ev = day_event_args(h).ev;
  f.a.err_word = h->d_err;
  f.rec = h->d_fl_rec; f.cev = h->d_fl_cev; f.cnode = h->d_fl_cnode; f.cnoff = h->d_fl_cnoff;
  f.day_comp = h->d_fl_day_comp;
  f.day_long = h->d_fl_day_long;
  f.cunit = h->d_fl_cunit; f.cuoff = h->d_fl_cuoff; f.K = h->d_fl_K; f.U1 = h->flow_U1;
  f.unit_cnt = h->d_rdy; f.next = h->d_flow_next; f.abort = h->d_flow_abort;
  f.spin_limit = spin_limit;
  f.stall_extra = stall ? (1u << 30) : 0u;
  f.d0 = d0; f.ndays = ndays;
  f.units = units;
  f.item_off = h->d_item_off;
  CK(h, traced(h, 0, st, [&] { return launch_flow(f, h->n_age, h->sm_count, st); }), "dataflow launch");
  if (stall) return SIM_OK;
  SsaArgs a = ssa_args(h);
  a.day = d0 + ndays - 1;
  CK(h, traced(h, 2, st, [&] { return launch_finalize(a, h->n_age, false, st); }), "phi update launch");
  return SIM_OK;
}

sim_status sim_run_days(sim_handle* h, int32_t ndays, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->phase) return fail(h, SIM_E_STATE, "the event step of day %d is due (sim_run_day_events)", h->day);
  if (ndays < 0 || (int64_t)h->day + ndays > h->cfg.max_days)
    return fail(h, SIM_E_INVALID_ARG, "ndays %d from day %d passes max_days %d", ndays, h->day, h->cfg.max_days);
  if (ndays == 0) return SIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t d0 = h->day;
  if (h->launch_mode == 2 && !h->profiling && h->n_regions > 0)
    return fail(h, SIM_E_STATE, "region statistics need the stream or graph launch mode");
  if (h->launch_mode == SIM_LAUNCH_FLOW && flow_usable(h)) {
    const sim_status s = enqueue_flow(h, d0, ndays, st, h->flow_spin_limit);
    if (s != SIM_OK) return s;
    h->day = d0 + ndays;
    return SIM_OK;
  }
  if (h->launch_mode == 2 && !h->profiling) {
    const int32_t until = d0 + ndays;
    sim_handle* one[1] = {h};
    sim_status s = sim_run_batch(one, 1, &until, stream);
    if (s != SIM_OK) return fail(h, s, "%s", sim_last_error(nullptr));
    return SIM_OK;
  }
  if (h->launch_mode == 1 && h->profiling) {
    // traced graph mode: a one-shot graph with the event records inside, so the
    // per-kernel times carry no host launch gaps
    cudaStream_t cs;
    CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sim_status s = SIM_OK;
    if (e == cudaSuccess) s = enqueue_days(h, d0, ndays, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && s == SIM_OK) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (s != SIM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(h, e, "traced graph capture");
    e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return cuda_fail(h, e, "traced graph launch");
    h->day = d0 + ndays;
    return SIM_OK;
  }
  if (h->launch_mode == 1 && !h->profiling) {
    if (!h->graph_exec || h->graph_d0 != d0 || h->graph_nd != ndays) {
      free_graph(h);
      // capture on a private stream so that the caller's stream may be the legacy default stream
      cudaStream_t cs;
      CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      sim_status s = SIM_OK;
      if (e == cudaSuccess) s = enqueue_days(h, d0, ndays, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess && s == SIM_OK) e = cudaGraphInstantiate(&h->graph_exec, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (s != SIM_OK) return s;
      if (e != cudaSuccess) { h->graph_exec = nullptr; return cuda_fail(h, e, "daily-loop graph capture"); }
      h->graph_d0 = d0;
      h->graph_nd = ndays;
    }
    CK(h, cudaGraphLaunch(h->graph_exec, st), "daily-loop graph launch");
    h->day = d0 + ndays;
    return SIM_OK;
  }
  sim_status s = enqueue_days(h, d0, ndays, st);
  if (s != SIM_OK) return s;
  h->day = d0 + ndays;
  return SIM_OK;
}

sim_status sim_sync(sim_handle* h, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  CK(h, cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  return check_latched(h);
}

sim_status sim_shard(sim_handle* h, int32_t node_lo, int32_t node_hi) {
  if (!h) return SIM_E_INVALID_ARG;
  if (node_lo < 0 || node_hi < node_lo || node_hi > h->cfg.n_nodes)
    return fail(h, SIM_E_INVALID_ARG, "node range [%d, %d) outside [0, %d]", node_lo, node_hi, h->cfg.n_nodes);
  if (h->day != 0 || h->phase) return fail(h, SIM_E_STATE, "a node range is set at day 0");
  if (h->cfg.flags & SIM_FLAG_SCORE) return fail(h, SIM_E_STATE, "score mode runs every node");
  if (h->n_regions > 0) return fail(h, SIM_E_STATE, "region statistics need every node");
  CK(h, cudaDeviceSynchronize(), "synchronize");
  h->node_lo = node_lo;
  h->node_hi = node_hi;
  return set_order(h, h->warp_threshold);
}

sim_status sim_run_day_stochastic(sim_handle* h, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->phase) return fail(h, SIM_E_STATE, "the event step of day %d is due (sim_run_day_events)", h->day);
  if (h->day >= h->cfg.max_days) return fail(h, SIM_E_INVALID_ARG, "day %d is max_days", h->day);
  if (h->cfg.flags & SIM_FLAG_SCORE) return fail(h, SIM_E_STATE, "score mode runs whole days (sim_run_days)");
  if (h->n_regions > 0) return fail(h, SIM_E_STATE, "region statistics run whole days (sim_run_days)");
  cudaStream_t st = (cudaStream_t)stream;
  SsaArgs a = ssa_args(h);
  a.day = h->day;
  a.prologue = 0;
  CK(h, traced(h, 0, st, [&] { return launch_ssa_day(a, h->n_age, false, st); }), "stochastic step launch");
  h->phase = 1;
  return SIM_OK;
}

sim_status sim_run_day_events(sim_handle* h, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (!h->phase) return fail(h, SIM_E_STATE, "no stochastic step of day %d ran (sim_run_day_stochastic)", h->day);
  cudaStream_t st = (cudaStream_t)stream;
  DayEventArgs E = day_event_args(h);
  const sim_status s = launch_day_events(h, E, h->day, st);
  if (s != SIM_OK) return s;
  SsaArgs a = ssa_args(h);
  a.day = h->day;
  CK(h, traced(h, 2, st, [&] { return launch_finalize(a, h->n_age, false, st); }), "phi update launch");
  h->phase = 0;
  h->day += 1;
  return SIM_OK;
}

int32_t sim_touched_count(const sim_handle* h, int32_t day) {
  if (!h || day < 0 || day >= h->cfg.max_days) return -1;
  if (!h->events_loaded) return 0;
  return h->day_touch_host[(size_t)day + 1] - h->day_touch_host[(size_t)day];
}

sim_status sim_touched_nodes(const sim_handle* h, int32_t day, int32_t* nodes) {
  if (!h || !nodes || day < 0 || day >= h->cfg.max_days) return SIM_E_INVALID_ARG;
  if (!h->events_loaded) return SIM_OK;
  const int32_t b = h->day_touch_host[(size_t)day], e = h->day_touch_host[(size_t)day + 1];
  for (int32_t i = b; i < e; ++i) nodes[i - b] = h->touched_host[(size_t)i];
  return SIM_OK;
}

sim_status sim_pack_touched(sim_handle* h, int32_t* dev_out, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (!h->phase) return fail(h, SIM_E_STATE, "pack after the day's stochastic step (sim_run_day_stochastic)");
  const int32_t n_t = sim_touched_count(h, h->day);
  if (n_t <= 0) return SIM_OK;
  if (!dev_out) return fail(h, SIM_E_INVALID_ARG, "null output buffer");
  const int32_t b = h->day_touch_host[(size_t)h->day];
  CK(h, launch_pack_touched(h->d_counts, h->d_touched + b, n_t, h->cfg.n_nodes,
                            (int64_t)h->cfg.n_replicates * h->nc, dev_out, (cudaStream_t)stream), "pack launch");
  return SIM_OK;
}

sim_status sim_unpack_touched(sim_handle* h, const int32_t* dev_in, int32_t world, const int32_t* bounds,
                              void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (!h->phase) return fail(h, SIM_E_STATE, "unpack after the day's stochastic step (sim_run_day_stochastic)");
  if (world < 1 || world > (1 << 16) || !bounds) return fail(h, SIM_E_INVALID_ARG, "world must be in [1, 65536]");
  if (bounds[0] != 0 || bounds[world] != h->cfg.n_nodes)
    return fail(h, SIM_E_INVALID_ARG, "bounds must run from 0 to n_nodes");
  for (int k = 0; k < world; ++k)
    if (bounds[k + 1] < bounds[k]) return fail(h, SIM_E_INVALID_ARG, "bounds must not decrease");
  const int32_t n_t = sim_touched_count(h, h->day);
  if (n_t <= 0) return SIM_OK;
  if (!dev_in) return fail(h, SIM_E_INVALID_ARG, "null input buffer");
  cudaStream_t st = (cudaStream_t)stream;
  if (world + 1 > h->pack_bounds_cap) {
    CK(h, cudaStreamSynchronize(st), "stream synchronize");
    cudaFree(h->d_pack_touched);
    h->d_pack_touched = nullptr;
    h->pack_bounds_cap = 0;
    CK(h, dalloc(&h->d_pack_touched, (size_t)world + 1), "bounds allocation");
    h->pack_bounds_cap = world + 1;
  }
  // a synchronous copy: the caller's host array may go away when this call returns
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  CK(h, cudaMemcpy(h->d_pack_touched, bounds, ((size_t)world + 1) * 4, cudaMemcpyHostToDevice), "bounds upload");
  const int32_t b = h->day_touch_host[(size_t)h->day];
  CK(h, launch_unpack_touched(h->d_counts, h->d_touched + b, n_t, h->cfg.n_nodes,
                              (int64_t)h->cfg.n_replicates * h->nc, dev_in, h->d_pack_touched, world, st),
     "unpack launch");
  return SIM_OK;
}

sim_status sim_state(sim_handle* h, int32_t* counts, double* phi, int32_t* day, int32_t where,
                     void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->phase) return fail(h, SIM_E_STATE, "the event step of day %d is due (sim_run_day_events)", h->day);
  if (where != SIM_HOST && where != SIM_DEVICE) return fail(h, SIM_E_INVALID_ARG, "where must be SIM_HOST or SIM_DEVICE");
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == SIM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (counts) CK(h, cudaMemcpyAsync(counts, h->d_counts, n_counts(h) * 4, k, st), "copy counts");
  if (phi) CK(h, cudaMemcpyAsync(phi, h->d_phi, n_phi(h) * 8, k, st), "copy phi");
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  if (day) *day = h->day;
  return check_latched(h);
}

sim_status sim_set_state(sim_handle* h, const int32_t* counts, const double* phi, int32_t day,
                         int32_t where, void* stream) {
  if (!h || !counts || !phi) return SIM_E_INVALID_ARG;
  if (h->phase) return fail(h, SIM_E_STATE, "the event step of day %d is due (sim_run_day_events)", h->day);
  if (where != SIM_HOST && where != SIM_DEVICE) return fail(h, SIM_E_INVALID_ARG, "where must be SIM_HOST or SIM_DEVICE");
  if (day < 0 || day > h->cfg.max_days) return fail(h, SIM_E_INVALID_ARG, "day %d out of range", day);
  if (where == SIM_HOST) {
    for (size_t i = 0; i < n_counts(h); ++i)
      if (counts[i] < 0) return fail(h, SIM_E_INVALID_ARG, "counts[%zu] < 0", i);
    for (size_t i = 0; i < n_phi(h); ++i)
      if (!finite_nonneg(phi[i])) return fail(h, SIM_E_INVALID_ARG, "phi[%zu] must be finite and >= 0", i);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == SIM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(h, cudaMemcpyAsync(h->d_counts, counts, n_counts(h) * 4, k, st), "copy counts");
  CK(h, cudaMemcpyAsync(h->d_phi, phi, n_phi(h) * 8, k, st), "copy phi");
  const int T = h->cfg.max_days;
  if (T > day) {
    const size_t w = (size_t)(T - day) * 8, pitch = (size_t)T * 8;
    CK(h, cudaMemset2DAsync(h->d_prev_i + day, pitch, 0, w, h->cfg.n_replicates, st), "clear stats");
    CK(h, cudaMemset2DAsync(h->d_prev_n + day, pitch, 0, w, h->cfg.n_replicates, st), "clear stats");
  }
  if (h->n_regions > 0 && T > day) {
    const size_t row = (size_t)h->n_regions * h->nc, bytes = (size_t)(T - day) * row * 8;
    CK(h, cudaMemsetAsync(h->d_s1 + (size_t)day * row, 0, bytes, st), "clear region statistics");
    CK(h, cudaMemsetAsync(h->d_s2 + (size_t)day * row, 0, bytes, st), "clear region statistics");
  }
  if (h->d_score) {
    CK(h, cudaMemsetAsync(h->d_score, 0, n_phi(h) * kScoreTerms * 8, st), "clear score");
    CK(h, cudaMemsetAsync(h->d_tang, 0, n_phi(h) * 2 * 8, st), "clear tangents");
  }
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  h->day = day;
  h->score_day0 = day;
  return SIM_OK;
}

sim_status sim_stats(sim_handle* h, int64_t* infected, int64_t* animals, int64_t* counters, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t stats = (size_t)h->cfg.n_replicates * h->cfg.max_days;
  if (infected && stats) CK(h, cudaMemcpyAsync(infected, h->d_prev_i, stats * 8, cudaMemcpyDeviceToHost, st), "copy stats");
  if (animals && stats) CK(h, cudaMemcpyAsync(animals, h->d_prev_n, stats * 8, cudaMemcpyDeviceToHost, st), "copy stats");
  if (counters) CK(h, cudaMemcpyAsync(counters, h->d_ctr, (size_t)h->cfg.n_replicates * 32, cudaMemcpyDeviceToHost, st), "copy counters");
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  return check_latched(h);
}

sim_status sim_score(sim_handle* h, double* score, void* stream) {
  if (!h || !score) return SIM_E_INVALID_ARG;
  if (!h->d_score) return fail(h, SIM_E_STATE, "created without SIM_FLAG_SCORE");
  cudaStream_t st = (cudaStream_t)stream;
  CK(h, cudaMemcpyAsync(score, h->d_score, n_phi(h) * kScoreTerms * 8, cudaMemcpyDeviceToHost, st), "copy score");
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  return check_latched(h);
}

sim_status sim_score_backward(sim_handle* h, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (!h->d_traj) return fail(h, SIM_E_STATE, "created without SIM_FLAG_SCORE_REVERSE");
  // the sweep covers [score_day0, day); days before score_day0 hold no trajectory
  const int32_t nd = h->day - h->score_day0;
  if (nd <= 0) return SIM_OK;
  CK(h, launch_phi_backward(h->d_traj + (size_t)h->score_day0 * n_phi(h),
                            h->d_params, h->d_score, h->cfg.n_nodes, h->cfg.n_replicates,
                            h->cfg.max_days, nd, (cudaStream_t)stream), "phi backward launch");
  return SIM_OK;
}

sim_status sim_gradient_moments(sim_handle* h, const int32_t* days, int32_t n_days, double* per_rep,
                                double* out, void* stream) {
  if (!h || n_days < 0 || (n_days > 0 && (!days || !out))) return SIM_E_INVALID_ARG;
  if (!h->d_score) return fail(h, SIM_E_STATE, "created without SIM_FLAG_SCORE");
  for (int i = 0; i < n_days; ++i)
    if (days[i] < 0 || days[i] >= h->cfg.max_days) return fail(h, SIM_E_INVALID_ARG, "days[%d] out of range", i);
  cudaStream_t st = (cudaStream_t)stream;
  if (n_days > h->moments_cap) {
    cudaFree(h->d_moments); cudaFree(h->d_days);
    h->d_moments = nullptr; h->d_days = nullptr; h->moments_cap = 0;
    CK(h, dalloc(&h->d_moments, (size_t)n_days * kMoments), "moments allocation");
    CK(h, dalloc(&h->d_days, (size_t)n_days), "moments allocation");
    h->moments_cap = n_days;
  }
  if (n_days > 0) CK(h, cudaMemcpyAsync(h->d_days, days, (size_t)n_days * 4, cudaMemcpyHostToDevice, st), "copy days");
  CK(h, launch_gradient_moments(h->d_score, h->d_prev_i, h->d_prev_n, h->d_days, n_days, h->cfg.n_nodes,
                                h->cfg.n_replicates, h->cfg.max_days, h->d_per_rep, h->d_moments, st),
     "gradient moments launch");
  if (per_rep) CK(h, cudaMemcpyAsync(per_rep, h->d_per_rep, (size_t)h->cfg.n_replicates * kScoreTerms * 8, cudaMemcpyDeviceToHost, st), "copy scores");
  if (n_days > 0) CK(h, cudaMemcpyAsync(out, h->d_moments, (size_t)n_days * kMoments * 8, cudaMemcpyDeviceToHost, st), "copy moments");
  CK(h, cudaStreamSynchronize(st), "stream synchronize");
  return check_latched(h);
}

sim_status sim_gradient_estimate(const double* moments, int32_t n_chunks, int32_t n_days, int64_t R,
                                 const double* jac, int32_t n_params, double* mean_f, double* grad,
                                 double* se) {
  if (!moments || !jac || n_chunks < 1 || n_days < 0 || n_params < 1 || R < 2) return SIM_E_INVALID_ARG;
  constexpr int kM = kMoments;
  const double dR = (double)R;
  for (int i = 0; i < n_days; ++i) {
    double m[kM] = {0};
    for (int c = 0; c < n_chunks; ++c)
      for (int q = 0; q < kM; ++q) m[q] += moments[((size_t)c * n_days + i) * kM + q];
    const double sf = m[0];
    const double mu = sf / dR;
    if (mean_f) mean_f[i] = mu;
    double cov[kScoreTerms], var8[kScoreTerms];
    for (int k = 0; k < kScoreTerms; ++k) {
      const double s_k = m[2 + 4 * k], s2_k = m[3 + 4 * k], fs_k = m[4 + 4 * k], fs2_k = m[5 + 4 * k];
      const double fss_k = m[2 + 4 * kScoreTerms + k];
      cov[k] = (fs_k - sf * s_k / dR) / (dR - 1.0);
      // variance of the centred product (f - mu) s_k, whose mean the covariance
      // estimates (the score has mean zero): E[(f - mu)^2 s^2] - (E[(f - mu) s])^2
      const double e2 = (fs2_k - 2.0 * mu * fss_k + mu * mu * s2_k) / dR;
      const double e1 = (fs_k - mu * s_k) / dR;
      const double v = e2 - e1 * e1;
      var8[k] = (v > 0.0 ? v : 0.0) / dR;
    }
    for (int c = 0; c < n_params; ++c) {
      double g = 0.0, v = 0.0;
      for (int k = 0; k < kScoreTerms; ++k) {
        const double j = jac[(size_t)k * n_params + c];
        g += cov[k] * j;
        v += var8[k] * j * j;
      }
      if (grad) grad[(size_t)i * n_params + c] = g;
      if (se) se[(size_t)i * n_params + c] = std::sqrt(v);
    }
  }
  return SIM_OK;
}

sim_status sim_set_params(sim_handle* h, const sim_params* p) {
  if (!h || !p) return SIM_E_INVALID_ARG;
  std::vector<DevParams> next((size_t)h->cfg.n_replicates);
  const sim_status s = fill_params(h, h, p, next);
  if (s != SIM_OK) return s;
  CK(h, cudaDeviceSynchronize(), "synchronize");
  CK(h, cudaMemcpy(h->d_params, next.data(), next.size() * sizeof(DevParams), cudaMemcpyHostToDevice),
     "parameter upload");
  h->params.swap(next);
  return SIM_OK;
}

sim_status sim_set_regions(sim_handle* h, const int32_t* region_of_node, int32_t n_regions) {
  if (!h) return SIM_E_INVALID_ARG;
  if (n_regions > 0 && (h->node_lo != 0 || h->node_hi != h->cfg.n_nodes))
    return fail(h, SIM_E_STATE, "region statistics need every node (the handle is sharded)");
  CK(h, cudaDeviceSynchronize(), "synchronize");
  free_regions(h);
  free_graph(h);
  if (n_regions == 0) return SIM_OK;
  const int N = h->cfg.n_nodes;
  if (n_regions < 0 || !region_of_node) return fail(h, SIM_E_INVALID_ARG, "n_regions must be >= 0 with a region array");
  std::vector<int32_t> off((size_t)n_regions + 1, 0), nodes((size_t)N);
  for (int v = 0; v < N; ++v) {
    const int32_t j = region_of_node[v];
    if (j < 0 || j >= n_regions) return fail(h, SIM_E_INVALID_ARG, "node %d: region %d out of range", v, j);
    off[(size_t)j + 1]++;
  }
  for (int32_t j = 0; j < n_regions; ++j) off[(size_t)j + 1] += off[(size_t)j];
  {
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int v = 0; v < N; ++v) nodes[(size_t)fill[(size_t)region_of_node[v]]++] = v;
  }
  const size_t rows = (size_t)std::max(1, h->cfg.max_days) * n_regions * h->nc;
  cudaError_t e = dalloc(&h->d_reg_nodes, nodes.size());
  if (e == cudaSuccess) e = dalloc(&h->d_reg_off, off.size());
  if (e == cudaSuccess) e = dalloc(&h->d_s1, rows);
  if (e == cudaSuccess) e = dalloc(&h->d_s2, rows);
  if (e == cudaSuccess) e = dalloc(&h->d_goal, 2);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_reg_nodes, nodes.data(), nodes.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_reg_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_s1, 0, rows * 8);
  if (e == cudaSuccess) e = cudaMemset(h->d_s2, 0, rows * 8);
  if (e != cudaSuccess) { free_regions(h); return cuda_fail(h, e, "region statistics"); }
  h->n_regions = n_regions;
  return SIM_OK;
}

sim_status sim_region_moments(sim_handle* h, uint64_t* s1, uint64_t* s2) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->n_regions == 0) return fail(h, SIM_E_STATE, "no regions set");
  CK(h, cudaDeviceSynchronize(), "synchronize");
  const size_t rows = (size_t)h->cfg.max_days * h->n_regions * h->nc;
  if (s1 && rows) CK(h, cudaMemcpy(s1, h->d_s1, rows * 8, cudaMemcpyDeviceToHost), "copy region statistics");
  if (s2 && rows) CK(h, cudaMemcpy(s2, h->d_s2, rows * 8, cudaMemcpyDeviceToHost), "copy region statistics");
  return check_latched(h);
}

sim_status sim_goal(sim_handle* h, const int64_t* ref, int32_t day0, int32_t ndays, double* g2, double* vg2) {
  if (!h || !ref || !g2 || !vg2) return SIM_E_INVALID_ARG;
  if (h->n_regions == 0) return fail(h, SIM_E_STATE, "no regions set");
  if (day0 < 0 || ndays < 1 || (int64_t)day0 + ndays > h->cfg.max_days)
    return fail(h, SIM_E_INVALID_ARG, "days [%d, %d + %d) outside [0, max_days)", day0, day0, ndays);
  const size_t row = (size_t)h->n_regions * h->nc, count = (size_t)ndays * row;
  CK(h, cudaDeviceSynchronize(), "synchronize");
  if (h->ref_cap < count) {
    cudaFree(h->d_ref);
    h->d_ref = nullptr;
    h->ref_cap = 0;
    CK(h, dalloc(&h->d_ref, count), "goal reference allocation");
    h->ref_cap = count;
  }
  CK(h, cudaMemcpy(h->d_ref, ref, count * 8, cudaMemcpyHostToDevice), "goal reference upload");
  CK(h, launch_goal(h->d_s1, h->d_s2, h->d_ref, (long long)((size_t)day0 * row), (long long)count,
                    h->cfg.n_replicates, h->d_goal, 0), "goal launch");
  double out[2];
  CK(h, cudaMemcpy(out, h->d_goal, 16, cudaMemcpyDeviceToHost), "goal copy");
  *g2 = out[0];
  *vg2 = out[1];
  return check_latched(h);
}

sim_status sim_reset(sim_handle* h, int32_t clear_events) {
  if (!h) return SIM_E_INVALID_ARG;
  CK(h, cudaDeviceSynchronize(), "synchronize");
  h->phase = 0;
  if (clear_events) { free_events(h); free_graph(h); }
  return reset_state(h);
}

void sim_destroy(sim_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

sim_status sim_debug_event_variant(sim_handle* h, int32_t global_only) {
  if (!h) return SIM_E_INVALID_ARG;
  if (global_only < 0 || global_only > 2) return fail(h, SIM_E_INVALID_ARG, "variant must be 0, 1 or 2");
  h->event_variant = global_only;
  if (global_only == 2) return SIM_OK;
  h->force_global_events = global_only != 0;
  for (size_t d = 0; d < h->day_smem.size(); ++d)
    if (h->force_global_events) h->day_smem[d] = 0;
  if (h->d_day_smem && !h->day_smem.empty())
    CK(h, cudaMemcpy(h->d_day_smem, h->day_smem.data(), h->day_smem.size() * 4, cudaMemcpyHostToDevice), "upload");
  return SIM_OK;
}

namespace {
long long g_batch_spin_limit = 5000000;   // ~2 s of polling per wait
bool g_batch_stall = false;               // test switch, see sim_debug_batch_stall
BatchShape g_batch_shape = BatchShape::k256x2;   // see sim_batch_shape
}

sim_status sim_run_batch(sim_handle** hs, int32_t n, const int32_t* until, void* stream) {
  if (n < 0 || (n > 0 && !hs)) return fail(nullptr, SIM_E_INVALID_ARG, "bad handle list");
  if (n == 0) return SIM_OK;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(nullptr, SIM_E_INVALID_ARG, "handle %d is NULL", i);
    if (hs[i]->phase || hs[i]->node_lo != 0 || hs[i]->node_hi != hs[i]->cfg.n_nodes)
      return fail(hs[i], SIM_E_STATE, "handle %d is sharded or between the halves of a day", i);
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(nullptr, SIM_E_INVALID_ARG, "handle %d listed twice", i);
    const int32_t u = until ? until[i] : hs[i]->cfg.max_days;
    if (u < hs[i]->day || u > hs[i]->cfg.max_days)
      return fail(hs[i], SIM_E_INVALID_ARG, "until day %d outside [day %d, max_days %d]", u, hs[i]->day, hs[i]->cfg.max_days);
  }
  cudaStream_t st = (cudaStream_t)stream;
  // instances with days to run, longest horizon first
  std::vector<int> idx;
  for (int i = 0; i < n; ++i) {
    const int32_t u = until ? until[i] : hs[i]->cfg.max_days;
    if (u > hs[i]->day) idx.push_back(i);
  }
  if (idx.empty()) return SIM_OK;
  auto nd = [&](int i) { return (until ? until[i] : hs[i]->cfg.max_days) - hs[i]->day; };
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return nd(a) > nd(b); });
  const int ni = (int)idx.size();
  std::vector<BatchInst> inst(ni);
  std::vector<long long> cumA(ni + 1, 0), cumB(ni + 1, 0), cumF(ni + 1, 0);
  long long n_counters = 0;
  int smem_cap = 0;
  const BatchShape shape = g_batch_shape;
  const int threads = batch_threads(shape);
  // two blocks an SM share its 228 KB of shared memory; a day whose staged event
  // step needs more takes the global-memory variant
  const int smem_limit = batch_min_blocks(shape) > 1 ? (int)(kBatchSmemSM / batch_min_blocks(shape)) : (int)kEventsSmemLimit;
  bool score_any = false;
  const int wpb = threads / 32;
  for (int k = 0; k < ni; ++k) {
    sim_handle* h = hs[idx[k]];
    BatchInst& I = inst[k];
    std::memset(&I, 0, sizeof I);
    I.ssa = ssa_args(h);
    I.ssa.warp_blocks = (h->n_big + wpb - 1) / wpb;
    I.na = h->n_age;
    I.score = (h->cfg.flags & SIM_FLAG_SCORE) ? 1 : 0;
    if (I.score) { I.ssa.n_big = 0; I.ssa.warp_blocks = 0; }
    const int n_thread = h->cfg.n_nodes - I.ssa.n_big;
    I.subs = kBatchSubs;
    I.n_thread = n_thread;
    I.bpr = I.ssa.warp_blocks + (n_thread + threads * kBatchSubs - 1) / (threads * kBatchSubs);
    I.tbpr = (h->cfg.n_nodes + threads - 1) / threads;
    score_any = score_any || I.score;
    I.day0 = h->day;
    I.ndays = nd(idx[k]);
    I.has_events = h->events_loaded ? 1 : 0;
    I.day_smem = h->d_day_smem;
    EvArgs& ev = I.evg;
    ev.counts = h->d_counts; ev.rec = h->d_rec; ev.lvl_start = h->d_lvl_start; ev.day_lvl = h->d_day_lvl;
    ev.ctr = h->d_ctr; ev.err = h->d_err; ev.seed = h->cfg.seed; ev.rep_base = h->cfg.replicate_base;
    ev.N = h->cfg.n_nodes; ev.R = h->cfg.n_replicates; ev.Nc = h->nc;
    ev.underflow_error = h->cfg.underflow_policy == SIM_UNDERFLOW_ERROR;
    EvSmemArgs& es = I.evs;
    es.counts = h->d_counts; es.rec = h->d_rec_slot; es.lvl_start = h->d_lvl_start; es.day_lvl = h->d_day_lvl;
    es.touched = h->d_touched; es.day_touch = h->d_day_touch; es.ctr = h->d_ctr; es.err = h->d_err;
    es.seed = h->cfg.seed; es.rep_base = h->cfg.replicate_base;
    es.N = h->cfg.n_nodes; es.R = h->cfg.n_replicates; es.Nc = h->nc; es.underflow_error = ev.underflow_error;
    if (h->events_loaded)
      for (int32_t d = I.day0; d < I.day0 + I.ndays; ++d)
        if (h->day_smem[(size_t)d] <= smem_limit) smem_cap = std::max(smem_cap, h->day_smem[(size_t)d]);
    const long long R = h->cfg.n_replicates;
    cumA[k + 1] = cumA[k] + R * I.bpr;
    cumB[k + 1] = cumB[k] + R;
    cumF[k + 1] = cumF[k] + R * I.tbpr;
    n_counters += 2 * R;
  }
  const int S = inst[0].ndays;
  std::vector<int32_t> active(S);
  std::vector<long long> step_off(S + 1, 0);
  for (int s = 0, a = ni; s < S; ++s) {
    while (a > 0 && inst[a - 1].ndays <= s) --a;
    active[s] = a;
    step_off[s + 1] = step_off[s] + cumA[a] + cumB[a];
  }
  // workspace: counters, control words, descriptors and tables (freed below)
  const size_t bytes_inst = sizeof(BatchInst) * ni;
  const size_t bytes_tab = sizeof(long long) * (3 * (ni + 1) + S + 1) + sizeof(int32_t) * S;
  const size_t bytes_ctr = sizeof(unsigned) * n_counters + 64;
  unsigned char* ws = nullptr;
  CK(nullptr, cudaMalloc(&ws, bytes_inst + bytes_tab + bytes_ctr + 256), "batch workspace");
  unsigned char* p = ws;
  BatchInst* d_inst = (BatchInst*)p; p += (bytes_inst + 15) / 16 * 16;
  long long* d_cumA = (long long*)p; p += 8 * (ni + 1);
  long long* d_cumB = (long long*)p; p += 8 * (ni + 1);
  long long* d_cumF = (long long*)p; p += 8 * (ni + 1);
  long long* d_step = (long long*)p; p += 8 * (S + 1);
  int32_t* d_active = (int32_t*)p; p += 4 * S;
  p = (unsigned char*)(((uintptr_t)p + 15) / 16 * 16);
  unsigned long long* d_next = (unsigned long long*)p; p += 8;
  int* d_abort = (int*)p; p += 4;
  int* d_err = (int*)p; p += 4;
  unsigned* d_ctr = (unsigned*)p;
  {
    unsigned* c = d_ctr;
    std::vector<unsigned> init((size_t)n_counters);
    size_t o = 0;
    for (int k = 0; k < ni; ++k) {
      const int R = inst[k].ssa.R;
      inst[k].ssa_done = c + o;
      for (int r = 0; r < R; ++r) init[o++] = 0;
      inst[k].ev_done = c + o;
      for (int r = 0; r < R; ++r) init[o++] = (unsigned)inst[k].day0;
      if (g_batch_stall && k == 0) init[o - R] = 0;   // replicate 0 waits for a day that never comes
    }
    cudaError_t e = cudaMemcpyAsync(d_ctr, init.data(), init.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_inst, inst.data(), bytes_inst, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cumA, cumA.data(), 8 * (ni + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cumB, cumB.data(), 8 * (ni + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cumF, cumF.data(), 8 * (ni + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_step, step_off.data(), 8 * (S + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_active, active.data(), 4 * S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, 16, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host vectors go out of scope
    if (e != cudaSuccess) { cudaFree(ws); return cuda_fail(nullptr, e, "batch upload"); }
  }
  BatchCtl c{};
  c.inst = d_inst; c.cumA = d_cumA; c.cumB = d_cumB; c.cumF = d_cumF; c.step_off = d_step; c.active = d_active;
  c.next = d_next; c.abort = d_abort; c.err = d_err;
  c.total_main = step_off[S];
  c.total = c.total_main + cumF[ni];
  c.spin_limit = g_batch_spin_limit;
  c.n_inst = ni; c.n_steps = S;
  c.smem_cap = smem_cap;
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = batch_occupancy(shape, score_any, smem_cap, &per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  const long long want = (long long)sms * per_sm;
  const int grid = (int)std::max(1LL, std::min(want, c.total));
  if (e == cudaSuccess) e = launch_batch(c, shape, score_any, grid, st);
  int berr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&berr, d_err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ws);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch kernel");
  for (int k = 0; k < ni; ++k) hs[idx[k]]->day = inst[k].day0 + inst[k].ndays;
  if (berr & kBatchTimeout) {
    for (int k = 0; k < ni; ++k) fail(hs[idx[k]], SIM_E_TIMEOUT, "a batch dependency wait ran out");
    return fail(nullptr, SIM_E_TIMEOUT, "a batch dependency wait ran out (state of the batch is undefined)");
  }
  return SIM_OK;
}

sim_status sim_debug_flow_stall(sim_handle* h, int32_t ndays, int64_t spin_limit) {
  if (!h) return SIM_E_INVALID_ARG;
  if (h->phase) return fail(h, SIM_E_STATE, "the event step of day %d is due (sim_run_day_events)", h->day);
  if (h->day < 1 || ndays < 1 || (int64_t)h->day + ndays > h->cfg.max_days || spin_limit < 1)
    return fail(h, SIM_E_INVALID_ARG, "the stall needs day >= 1, ndays >= 1 within max_days, spin_limit >= 1");
  if (!flow_usable(h)) return fail(h, SIM_E_STATE, "the handle cannot take the dataflow loop");
  const sim_status s = enqueue_flow(h, h->day, ndays, nullptr, (long long)spin_limit, true);
  if (s != SIM_OK) return s;
  CK(h, cudaStreamSynchronize(nullptr), "stream synchronize");
  return check_latched(h);
}

sim_status sim_batch_shape(int32_t threads, int32_t blocks_per_sm) {
  if (threads == 256 && blocks_per_sm == 1) g_batch_shape = BatchShape::k256x1;
  else if (threads == 256 && blocks_per_sm == 2) g_batch_shape = BatchShape::k256x2;
  else if (threads == 128 && blocks_per_sm == 4) g_batch_shape = BatchShape::k128x4;
  else return fail(nullptr, SIM_E_INVALID_ARG, "batch shape %d x %d is not one of 256x1, 256x2, 128x4",
                   threads, blocks_per_sm);
  return SIM_OK;
}

sim_status sim_debug_batch_spin_limit(int64_t limit) {
  if (limit < 1) return SIM_E_INVALID_ARG;
  g_batch_spin_limit = limit;
  return SIM_OK;
}

sim_status sim_debug_batch_stall(sim_handle* h, int32_t until, int64_t spin_limit) {
  // A batch run whose first dependency can never be met: replicate 0's event
  // counter starts at 0 while the run starts at day >= 1, so its first chunk
  // waits for event steps that are never scheduled.  The bounded wait must run
  // out, abort the launch and report SIM_E_TIMEOUT; the device stays usable.
  if (!h || h->day < 1 || until <= h->day || spin_limit < 1) return SIM_E_INVALID_ARG;
  const long long saved = g_batch_spin_limit;
  g_batch_spin_limit = spin_limit;
  g_batch_stall = true;
  const int32_t d0 = h->day;
  sim_handle* one[1] = {h};
  sim_status s = sim_run_batch(one, 1, &until, nullptr);
  g_batch_spin_limit = saved;
  g_batch_stall = false;
  h->day = d0;
  return s;
}

sim_status sim_tune(sim_handle* h, int32_t warp_herd_threshold) {
  if (!h) return SIM_E_INVALID_ARG;
  CK(h, cudaDeviceSynchronize(), "synchronize");
  return set_order(h, warp_herd_threshold);
}

int32_t sim_warp_nodes(const sim_handle* h) { return h ? h->n_big : -1; }

sim_status sim_set_option(sim_handle* h, int32_t option, int64_t value) {
  if (!h) return SIM_E_INVALID_ARG;
  switch (option) {
    case SIM_OPT_WARP_THRESHOLD:
      return sim_tune(h, (int32_t)std::max<int64_t>(-1, std::min<int64_t>(value, 1 << 30)));
    case SIM_OPT_LAUNCH:
      if (value < SIM_LAUNCH_STREAM || value > SIM_LAUNCH_FLOW)
        return fail(h, SIM_E_INVALID_ARG, "unknown launch mode %lld", (long long)value);
      CK(h, cudaDeviceSynchronize(), "synchronize");
      free_graph(h);
      h->launch_mode = (int32_t)value;
      return SIM_OK;
    case SIM_OPT_OVERLAP:
      if (value != 0 && value != 1) return fail(h, SIM_E_INVALID_ARG, "overlap must be 0 or 1");
      CK(h, cudaDeviceSynchronize(), "synchronize");
      free_graph(h);
      h->overlap = (int32_t)value;
      return SIM_OK;
    case SIM_OPT_GROUP_THRESHOLD:
      if (value < -1) return fail(h, SIM_E_INVALID_ARG, "group threshold must be >= -1");
      CK(h, cudaDeviceSynchronize(), "synchronize");
      h->group_threshold = (int32_t)std::min<int64_t>(value, 1 << 30);
      return set_order(h, h->warp_threshold);
    case SIM_OPT_SPLIT:
      if (value != 0 && value != 1) return fail(h, SIM_E_INVALID_ARG, "split must be 0 or 1");
      CK(h, cudaDeviceSynchronize(), "synchronize");
      free_graph(h);
      h->split = (int32_t)value;
      return SIM_OK;
    case SIM_OPT_CLOCK_MARGIN:
      if (value < 0 || value > 17)
        return fail(h, SIM_E_INVALID_ARG, "clock margin exponent %lld outside [0, 17]", (long long)value);
      CK(h, cudaDeviceSynchronize(), "synchronize");
      free_graph(h);
      h->clock_margin_log2 = (int32_t)value;
      return SIM_OK;
    default:
      return fail(h, SIM_E_INVALID_ARG, "unknown option %d", option);
  }
}

sim_status sim_profile(sim_handle* h, int32_t enable) {
  if (!h) return SIM_E_INVALID_ARG;
  CK(h, cudaDeviceSynchronize(), "synchronize");
  h->profiling = enable != 0;
  h->ev_used = 0;
  h->ev_kind.clear();
  return SIM_OK;
}

sim_status sim_profile_read(sim_handle* h, double* ms, int64_t* launches) {
  if (!h) return SIM_E_INVALID_ARG;
  double acc[3] = {0, 0, 0};
  int64_t cnt[3] = {0, 0, 0};
  for (size_t i = 0; i < h->ev_kind.size(); ++i) {
    CK(h, cudaEventSynchronize(h->ev_pool[2 * i + 1]), "event synchronize");
    float t = 0.f;
    CK(h, cudaEventElapsedTime(&t, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]), "event elapsed time");
    acc[h->ev_kind[i]] += t;
    cnt[h->ev_kind[i]] += 1;
  }
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = cnt[k];
  }
  return SIM_OK;
}

const char* sim_last_error(const sim_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

sim_status sim_debug_neglog(const uint64_t* j_dev, double* out_dev, int64_t n) {
  if (n < 0 || (n > 0 && (!j_dev || !out_dev))) return SIM_E_INVALID_ARG;
  cudaError_t e = launch_debug_neglog(j_dev, out_dev, n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SIM_OK : SIM_E_CUDA;
}

sim_status sim_debug_neglog_f32(const uint64_t* j_dev, float* out_dev, int64_t n) {
  if (n < 0 || (n > 0 && (!j_dev || !out_dev))) return SIM_E_INVALID_ARG;
  cudaError_t e = launch_debug_neglog_f32(j_dev, out_dev, n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SIM_OK : SIM_E_CUDA;
}

sim_status sim_debug_div(const double* x, const double* y, double* out, double* ref, int64_t n, int32_t where) {
  if (n < 0 || (n > 0 && (!x || !y || !out || !ref))) return SIM_E_INVALID_ARG;
  if (where == SIM_HOST) {
    for (int64_t i = 0; i < n; ++i) { out[i] = episim::div_pos(x[i], y[i]); ref[i] = x[i] / y[i]; }
    return SIM_OK;
  }
  cudaError_t e = launch_debug_div(x, y, out, ref, n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SIM_OK : SIM_E_CUDA;
}

sim_status sim_debug_schedule(const sim_handle* h, int64_t* order, int32_t* level) {
  if (!h) return SIM_E_INVALID_ARG;
  if (order) std::memcpy(order, h->sched_order.data(), h->sched_order.size() * 8);
  if (level) std::memcpy(level, h->sched_level.data(), h->sched_level.size() * 4);
  return SIM_OK;
}

int64_t sim_debug_schedule_size(const sim_handle* h) { return h ? (int64_t)h->sched_order.size() : -1; }

}  // extern "C"
