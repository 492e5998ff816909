// Host side of the general compartment model (include/episim_general.h): model
// validation and its dependency graph (Sec. 3.3), device memory, the per-day
// decomposition of the events into components of the transfer graph, and the
// per-day launch sequence (Alg. 1: stochastic step, events, continuous update).
#include "../../include/episim_general.h"
#include "general.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

using namespace episim;

struct gen_handle {
  gen_config cfg{};
  GenModelDev model{};
  int nc = 0, nt = 0, ny = 0, n_select = 0, n_shift = 0;
  std::vector<GenRepParams> params;
  int32_t* d_counts = nullptr;      // [R][Nc][N]
  double* d_y = nullptr;            // [R][Ny][N]
  double* d_mid = nullptr;          // [R][Ny][2][N] (midpoint variant)
  int32_t* d_order = nullptr;       // [N]
  GenModelDev* d_model = nullptr;
  GenRepParams* d_params = nullptr;
  unsigned long long* d_ctr = nullptr;
  int32_t* d_err = nullptr;
  // events
  int4* d_rec = nullptr;
  int32_t* d_comp_ev = nullptr;
  int32_t* d_comp_off = nullptr;
  std::vector<int32_t> day_comp;    // [max_days + 1] first component of each day
  int32_t day = 0;
  int32_t launch_mode = 0;          // 0 stream, 1 CUDA graph
  std::vector<int64_t> pop_sorted;  // initial node populations in the node order (descending)
  int32_t warp_threshold = -1;      // initial population from which a node gets a warp (-1: automatic)
  int32_t clock_margin_log2 = 16;   // binary32 clock margin 2^-k of the thread method (0: exact only)
  int32_t group_threshold = -1;     // ... an 8-lane segment (-1: automatic)
  int32_t n_big = 0;                // nodes simulated one per warp
  int32_t n_mid = 0;                // nodes simulated four per warp
  cudaGraphExec_t graph_exec = nullptr;
  int32_t graph_d0 = -1, graph_nd = -1;
  std::string err;
};

namespace {

thread_local std::string g_gen_create_error;

sim_status gfail(gen_handle* h, sim_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_gen_create_error = buf;
  return s;
}

sim_status gcuda(gen_handle* h, cudaError_t e, const char* what) {
  return gfail(h, e == cudaErrorMemoryAllocation ? SIM_E_OOM : SIM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GCK(h, call, what)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return gcuda(h, e_, what); \
  } while (0)

template <class T>
cudaError_t galloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

// Validates m and fills the device descriptor (change lists, dependency graph).
sim_status build_model(const gen_model* m, GenModelDev* out, char* why, size_t wn) {
  auto bad = [&](const char* fmt, auto... args) {
    snprintf(why, wn, fmt, args...);
    return SIM_E_INVALID_ARG;
  };
  if (!m) return bad("model is NULL");
  const int nc = m->n_comp, nt = m->n_trans, ny = m->n_cont;
  if (nc < 1 || nc > kGenMaxComp) return bad("n_comp %d outside [1, %d]", nc, kGenMaxComp);
  if (nt < 0 || nt > kGenMaxTrans) return bad("n_trans %d outside [0, %d]", nt, kGenMaxTrans);
  if (ny < 0 || ny > kGenMaxCont) return bad("n_cont %d outside [0, %d]", ny, kGenMaxCont);
  if (m->n_select < 0 || m->n_select > kGenMaxSelect) return bad("n_select %d outside [0, %d]", m->n_select, kGenMaxSelect);
  if (m->n_shift < 0 || m->n_shift > kGenMaxShift) return bad("n_shift %d outside [0, %d]", m->n_shift, kGenMaxShift);
  if (m->y_source < GEN_Y_POST_EVENT || m->y_source > GEN_Y_MIDPOINT) return bad("y_source %d unknown", m->y_source);
  if (nt > 0 && (!m->stoich || !m->trans)) return bad("stoich and trans are required");
  if (ny > 0 && !m->vars) return bad("vars is required");
  if (m->n_select > 0 && !m->select) return bad("select is required");
  if (m->n_shift > 0 && !m->shift) return bad("shift is required");
  const uint32_t all = nc == 32 ? ~0u : ((1u << nc) - 1u);
  std::memset(out, 0, sizeof *out);
  out->nc = nc; out->nt = nt; out->ny = ny; out->y_source = m->y_source;
  int nchg = 0;
  for (int j = 0; j < nt; ++j) {
    const gen_transition& t = m->trans[j];
    if (t.factor_a < -1 || t.factor_a >= nc) return bad("transition %d: factor_a %d", j, t.factor_a);
    if (t.factor_b < -1 || t.factor_b >= nc) return bad("transition %d: factor_b %d", j, t.factor_b);
    if (t.cont < -1 || t.cont >= ny) return bad("transition %d: cont %d", j, t.cont);
    if (t.pop_mask & ~all) return bad("transition %d: pop_mask names no compartment", j);
    out->fa[j] = t.factor_a; out->fb[j] = t.factor_b; out->fy[j] = t.cont; out->pop[j] = t.pop_mask;
    out->chg_off[j] = nchg;
    for (int c = 0; c < nc; ++c) {
      const int s = m->stoich[c * nt + j];
      if (s < -1 || s > 127) return bad("stoich[%d][%d] = %d outside [-1, 127]", c, j, s);
      if (s == -1 && c != t.factor_a && c != t.factor_b)
        return bad("transition %d decrements compartment %d, which is not a factor of its rate", j, c);
      if (s != 0) out->chg[nchg++] = ((uint32_t)s << 8) | (uint32_t)c;
    }
  }
  out->chg_off[nt] = nchg;
  for (int n = 0; n < nt; ++n) {
    uint32_t d = 0;
    for (int j = 0; j < nt; ++j) {
      const gen_transition& t = m->trans[j];
      bool hit = (t.factor_a >= 0 && m->stoich[t.factor_a * nt + n] != 0) ||
                 (t.factor_b >= 0 && m->stoich[t.factor_b * nt + n] != 0);
      if (t.pop_mask) {
        int net = 0;
        for (int c = 0; c < nc; ++c)
          if (t.pop_mask >> c & 1u) net += m->stoich[c * nt + n];
        hit = hit || net != 0;
      }
      if (hit) d |= 1u << j;
    }
    out->dep[n] = d;
  }
  for (int q = 0; q < ny; ++q) {
    if ((m->vars[q].num_mask | m->vars[q].den_mask) & ~all) return bad("variable %d: mask names no compartment", q);
    out->num[q] = m->vars[q].num_mask;
    out->den[q] = m->vars[q].den_mask;
  }
  for (int s = 0; s < m->n_select; ++s) {
    if (m->select[s] == 0 || (m->select[s] & ~all)) return bad("select %d: empty or names no compartment", s);
    out->select[s] = m->select[s];
  }
  for (int s = 0; s < m->n_shift; ++s)
    for (int c = 0; c < nc; ++c) {
      const int o = m->shift[s * nc + c];
      if (o <= -nc || o >= nc) return bad("shift[%d][%d] = %d out of range", s, c, o);
      out->shift[s][c] = (int8_t)o;
    }
  return SIM_OK;
}

void free_graph(gen_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
  h->graph_d0 = h->graph_nd = -1;
}

void free_events(gen_handle* h) {
  cudaFree(h->d_rec); cudaFree(h->d_comp_ev); cudaFree(h->d_comp_off);
  h->d_rec = nullptr; h->d_comp_ev = nullptr; h->d_comp_off = nullptr;
  h->day_comp.assign((size_t)h->cfg.max_days + 1, 0);
}

sim_status latched(gen_handle* h) {
  int32_t e = 0;
  GCK(h, cudaMemcpy(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost), "read device error word");
  if (e) {
    GCK(h, cudaMemset(h->d_err, 0, sizeof e), "clear device error word");
    return gfail(h, SIM_E_UNDERFLOW, "an event asked for more animals than present (ERROR policy)");
  }
  return SIM_OK;
}

constexpr int32_t kAutoWarpThreshold = 600;
constexpr int32_t kAutoGroupThreshold = 150;

void set_n_big(gen_handle* h) {
  const int64_t thr = h->warp_threshold < 0 ? kAutoWarpThreshold : h->warp_threshold;
  const int64_t gthr = h->group_threshold < 0 ? kAutoGroupThreshold : h->group_threshold;
  const int32_t N = (int32_t)h->pop_sorted.size();
  int32_t n = 0;
  while (n < N && h->pop_sorted[n] >= thr) ++n;
  int32_t g = n;
  while (g < N && h->pop_sorted[g] >= gthr) ++g;
  h->n_big = n;
  h->n_mid = g - n;
}

sim_status enqueue_days(gen_handle* h, int32_t d0, int32_t nd, cudaStream_t st) {
  const int N = h->cfg.n_nodes, R = h->cfg.n_replicates;
  for (int32_t d = d0; d < d0 + nd; ++d) {
    GenSsaArgs s{};
    s.counts = h->d_counts; s.y = h->d_y; s.mid = h->d_mid; s.model = h->d_model; s.params = h->d_params;
    s.order = h->d_order; s.ctr = h->d_ctr; s.seed = h->cfg.seed; s.rep_base = h->cfg.replicate_base;
    s.N = N; s.R = R; s.day = d; s.n_big = h->n_big; s.n_mid = h->n_mid;
    s.prologue = (d > d0 && h->ny > 0 && h->model.y_source != GEN_Y_PRE_EVENT) ? 1 : 0;
    s.clock_margin = h->clock_margin_log2 > 0 ? (1ull << (62 - h->clock_margin_log2)) : 0ull;
    GCK(h, launch_gen_ssa(s, h->nt, h->nc, st), "stochastic step launch");
    const int32_t c0 = h->day_comp[d], c1 = h->day_comp[d + 1];
    if (c1 > c0) {
      GenEvArgs e{};
      e.counts = h->d_counts; e.rec = h->d_rec; e.comp_ev = h->d_comp_ev; e.comp_off = h->d_comp_off;
      e.comp0 = c0; e.ncomp = c1 - c0; e.model = h->d_model; e.ctr = h->d_ctr; e.err = h->d_err;
      e.seed = h->cfg.seed; e.rep_base = h->cfg.replicate_base; e.N = N; e.R = R; e.day = d;
      e.underflow_error = h->cfg.underflow_policy == SIM_UNDERFLOW_ERROR;
      GCK(h, launch_gen_events(e, st), "event step launch");
    }
  }
  // the last day's continuous update (earlier days' run in the next day's prologue)
  if (nd > 0 && h->ny > 0 && h->model.y_source != GEN_Y_PRE_EVENT) {
    GenContArgs c{};
    c.counts = h->d_counts; c.y = h->d_y; c.mid = h->d_mid; c.model = h->d_model; c.params = h->d_params;
    c.N = N; c.R = R; c.day = d0 + nd - 1;
    GCK(h, launch_gen_cont(c, st), "continuous update launch");
  }
  return SIM_OK;
}

}  // namespace

extern "C" {

sim_status gen_model_check(const gen_model* m, uint32_t* dep) {
  GenModelDev d;
  char why[256] = {0};
  sim_status s = build_model(m, &d, why, sizeof why);
  if (s != SIM_OK) return gfail(nullptr, s, "%s", why);
  if (dep)
    for (int n = 0; n < m->n_trans; ++n) dep[n] = d.dep[n];
  return SIM_OK;
}

sim_status gen_create(const gen_model* m, const gen_config* cfg, const int32_t* u0, const double* y0,
                      const double* rates, const double* var_params, gen_handle** out) {
  if (!out) return gfail(nullptr, SIM_E_INVALID_ARG, "out is NULL");
  if (!cfg || !u0) return gfail(nullptr, SIM_E_INVALID_ARG, "cfg and u0 are required");
  GenModelDev md;
  char why[256] = {0};
  if (build_model(m, &md, why, sizeof why) != SIM_OK) return gfail(nullptr, SIM_E_INVALID_ARG, "%s", why);
  const int nc = m->n_comp, nt = m->n_trans, ny = m->n_cont;
  const int N = cfg->n_nodes, R = cfg->n_replicates;
  if (N < 1 || R < 1 || cfg->max_days < 0 || cfg->reserved != 0)
    return gfail(nullptr, SIM_E_INVALID_ARG, "n_nodes, n_replicates >= 1, max_days >= 0 and reserved = 0 required");
  if (cfg->underflow_policy != SIM_UNDERFLOW_CLAMP && cfg->underflow_policy != SIM_UNDERFLOW_ERROR)
    return gfail(nullptr, SIM_E_INVALID_ARG, "underflow_policy %d unknown", cfg->underflow_policy);
  if (cfg->replicate_base < 0 || (int64_t)cfg->replicate_base + R > ((int64_t)1 << 32))
    return gfail(nullptr, SIM_E_INVALID_ARG, "replicate_base out of range");
  if ((ny > 0 && (!y0 || !var_params)) || (nt > 0 && !rates))
    return gfail(nullptr, SIM_E_INVALID_ARG, "y0, var_params and rates are required when the model has them");
  if ((int64_t)R * nc * N > ((int64_t)1 << 31) || (int64_t)R * std::max(ny, 1) * 2 * N > ((int64_t)1 << 31))
    return gfail(nullptr, SIM_E_INVALID_ARG, "state too large");
  for (int64_t i = 0; i < (int64_t)nc * N; ++i)
    if (u0[i] < 0) return gfail(nullptr, SIM_E_INVALID_ARG, "u0[%lld] < 0", (long long)i);
  for (int v = 0; v < N; ++v) {
    int64_t tot = 0;
    for (int c = 0; c < nc; ++c) tot += u0[(size_t)c * N + v];
    if (tot > (1 << 30)) return gfail(nullptr, SIM_E_INVALID_ARG, "node %d holds more than 2^30 animals", v);
  }
  for (int64_t i = 0; i < (int64_t)ny * N; ++i)
    if (!finite_nonneg(y0[i])) return gfail(nullptr, SIM_E_INVALID_ARG, "y0[%lld] must be finite and >= 0", (long long)i);
  std::vector<GenRepParams> params((size_t)R);
  for (int r = 0; r < R; ++r) {
    GenRepParams& p = params[r];
    std::memset(&p, 0, sizeof p);
    for (int j = 0; j < nt; ++j) {
      p.rate[j] = rates[(size_t)r * nt + j];
      if (!finite_nonneg(p.rate[j])) return gfail(nullptr, SIM_E_INVALID_ARG, "rate[%d][%d] must be finite and >= 0", r, j);
    }
    for (int q = 0; q < ny; ++q) {
      const double* v = var_params + ((size_t)r * ny + q) * 6;
      p.alpha[q] = v[0];
      for (int s = 0; s < 4; ++s) p.beta[q][s] = v[1 + s];
      p.eps[q] = v[5];
      if (!finite_nonneg(v[0]) || !finite_nonneg(v[5]))
        return gfail(nullptr, SIM_E_INVALID_ARG, "alpha and epsilon of variable %d must be finite and >= 0", q);
      for (int s = 0; s < 4; ++s)
        if (!(v[1 + s] >= 0.0 && v[1 + s] <= 1.0)) return gfail(nullptr, SIM_E_INVALID_ARG, "beta of variable %d outside [0, 1]", q);
    }
  }
  gen_handle* h = new (std::nothrow) gen_handle;
  if (!h) return gfail(nullptr, SIM_E_OOM, "host allocation");
  h->cfg = *cfg; h->model = md; h->nc = nc; h->nt = nt; h->ny = ny; h->params = std::move(params);
  h->n_select = m->n_select; h->n_shift = m->n_shift;
  h->day_comp.assign((size_t)cfg->max_days + 1, 0);
  // nodes by initial population, largest first (warps hold nodes of similar work)
  std::vector<int64_t> tot((size_t)N, 0);
  for (int c = 0; c < nc; ++c)
    for (int v = 0; v < N; ++v) tot[v] += u0[(size_t)c * N + v];
  std::vector<int32_t> order((size_t)N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return tot[a] > tot[b]; });
  h->pop_sorted.resize((size_t)N);
  for (int i = 0; i < N; ++i) h->pop_sorted[i] = tot[order[i]];
  set_n_big(h);
  const size_t ncount = (size_t)R * nc * N, ncy = (size_t)R * ny * N;
  cudaError_t e = galloc(&h->d_counts, ncount);
  if (e == cudaSuccess) e = galloc(&h->d_y, ncy);
  if (e == cudaSuccess && m->y_source == GEN_Y_MIDPOINT) e = galloc(&h->d_mid, 2 * ncy);
  if (e == cudaSuccess) e = galloc(&h->d_order, (size_t)N);
  if (e == cudaSuccess) e = galloc(&h->d_model, 1);
  if (e == cudaSuccess) e = galloc(&h->d_params, (size_t)R);
  if (e == cudaSuccess) e = galloc(&h->d_ctr, (size_t)R * 4);
  if (e == cudaSuccess) e = galloc(&h->d_err, 1);
  for (int r = 0; r < R && e == cudaSuccess; ++r) {
    e = cudaMemcpy(h->d_counts + (size_t)r * nc * N, u0, (size_t)nc * N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ny > 0)
      e = cudaMemcpy(h->d_y + (size_t)r * ny * N, y0, (size_t)ny * N * 8, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(h->d_order, order.data(), (size_t)N * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_model, &h->model, sizeof(GenModelDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_params, h->params.data(), (size_t)R * sizeof(GenRepParams), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, (size_t)R * 4 * 8);
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 4);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    gcuda(nullptr, e, "device state");
    gen_destroy(h);
    return e == cudaErrorMemoryAllocation ? SIM_E_OOM : SIM_E_CUDA;
  }
  *out = h;
  return SIM_OK;
}

sim_status gen_load_events(gen_handle* h, int64_t n, const int32_t* day, const int32_t* kind, const int32_t* node,
                           const int32_t* dest, const int32_t* count, const int32_t* select, const int32_t* shift) {
  if (!h) return SIM_E_INVALID_ARG;
  if (n < 0 || n >= ((int64_t)1 << 31)) return gfail(h, SIM_E_INVALID_ARG, "n = %lld out of range", (long long)n);
  if (n > 0 && (!day || !kind || !node || !dest || !count || !select || !shift))
    return gfail(h, SIM_E_INVALID_ARG, "event arrays are required");
  const int N = h->cfg.n_nodes, T = h->cfg.max_days, nc = h->nc;
  const GenModelDev& m = h->model;
  for (int64_t e = 0; e < n; ++e) {
    if (day[e] < 0) return gfail(h, SIM_E_INVALID_ARG, "event %lld: day %d < 0", (long long)e, day[e]);
    if (kind[e] < SIM_EXIT || kind[e] > SIM_EXTERNAL) return gfail(h, SIM_E_INVALID_ARG, "event %lld: kind %d", (long long)e, kind[e]);
    if (node[e] < 0 || node[e] >= N) return gfail(h, SIM_E_INVALID_ARG, "event %lld: node %d", (long long)e, node[e]);
    if (kind[e] == SIM_EXTERNAL && (dest[e] < 0 || dest[e] >= N || dest[e] == node[e]))
      return gfail(h, SIM_E_INVALID_ARG, "event %lld: dest %d", (long long)e, dest[e]);
    if (count[e] < 0) return gfail(h, SIM_E_INVALID_ARG, "event %lld: count %d < 0", (long long)e, count[e]);
    if (select[e] < 0 || select[e] >= h->n_select)
      return gfail(h, SIM_E_INVALID_ARG, "event %lld: select %d", (long long)e, select[e]);
    if (shift[e] < -1 || shift[e] >= h->n_shift)
      return gfail(h, SIM_E_INVALID_ARG, "event %lld: shift %d", (long long)e, shift[e]);
    const int row = shift[e] < 0 ? kGenNoShift : shift[e];
    const uint32_t mask = m.select[select[e]];
    for (int c = 0; c < nc; ++c)
      if (mask >> c & 1u) {
        const int to = c + m.shift[row][c];
        if (to < 0 || to >= nc)
          return gfail(h, SIM_E_INVALID_ARG, "event %lld: shift moves compartment %d outside the model", (long long)e, c);
        if (kind[e] == SIM_ENTER) break;
        if (kind[e] == SIM_INTERNAL && (mask >> to & 1u))
          return gfail(h, SIM_E_INVALID_ARG, "event %lld: an internal move into the sampled mask (compartment %d)",
                       (long long)e, to);
      }
  }
  free_graph(h);
  free_events(h);
  // day-stable order of the events before the horizon (those after it come later
  // in that order, so dropping them leaves every position unchanged)
  std::vector<int64_t> first((size_t)T + 1, 0);
  for (int64_t e = 0; e < n; ++e)
    if (day[e] < T) first[day[e] + 1]++;
  for (int d = 0; d < T; ++d) first[d + 1] += first[d];
  const int64_t nk = first[T];
  if (nk == 0) return SIM_OK;
  std::vector<int32_t> order((size_t)nk);
  {
    std::vector<int64_t> fill(first.begin(), first.end() - 1);
    for (int64_t e = 0; e < n; ++e)
      if (day[e] < T) order[fill[day[e]]++] = (int32_t)e;
  }
  std::vector<int4> rec((size_t)nk);
  for (int64_t s = 0; s < nk; ++s) {
    const int32_t e = order[s];
    const int row = shift[e] < 0 ? kGenNoShift : shift[e];
    rec[s] = make_int4(node[e], kind[e] == SIM_EXTERNAL ? dest[e] : -1, count[e],
                       kind[e] | (select[e] << 8) | (row << 16));
  }
  // per day: components of the graph whose edges are the day's transfers
  std::vector<int32_t> parent((size_t)N, -1), comp_ev, comp_off;
  comp_ev.reserve((size_t)nk);
  comp_off.reserve((size_t)nk + 1);
  std::vector<int32_t> touched, root_comp((size_t)N, -1), roots, comp_of, csize, idx, cpos;
  auto find = [&](int32_t v) {
    while (parent[v] != v) { parent[v] = parent[parent[v]]; v = parent[v]; }
    return v;
  };
  for (int d = 0; d < T; ++d) {
    h->day_comp[d] = (int32_t)comp_off.size();
    const int64_t s0 = first[d], s1 = first[d + 1];
    if (s1 == s0) continue;
    touched.clear();
    auto touch = [&](int32_t v) { if (parent[v] < 0) { parent[v] = v; touched.push_back(v); } };
    for (int64_t s = s0; s < s1; ++s) {
      touch(rec[s].x);
      if (rec[s].y >= 0) {
        touch(rec[s].y);
        const int32_t a = find(rec[s].x), b = find(rec[s].y);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
      }
    }
    // components numbered by their first event, placed heaviest first (ties in
    // that numbering), each with its events in input order
    roots.clear();
    csize.clear();
    comp_of.resize((size_t)(s1 - s0));
    for (int64_t s = s0; s < s1; ++s) {
      const int32_t rt = find(rec[s].x);
      if (root_comp[rt] < 0) { root_comp[rt] = (int32_t)csize.size(); csize.push_back(0); roots.push_back(rt); }
      comp_of[(size_t)(s - s0)] = root_comp[rt];
      csize[(size_t)root_comp[rt]]++;
    }
    const int32_t ncomp = (int32_t)csize.size();
    idx.resize((size_t)ncomp);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return csize[(size_t)a] > csize[(size_t)b]; });
    cpos.resize((size_t)ncomp);
    for (int32_t q = 0, at = (int32_t)comp_ev.size(); q < ncomp; ++q) {
      comp_off.push_back(at);
      cpos[(size_t)idx[(size_t)q]] = at;
      at += csize[(size_t)idx[(size_t)q]];
    }
    comp_ev.resize(comp_ev.size() + (size_t)(s1 - s0));
    for (int64_t s = s0; s < s1; ++s) comp_ev[(size_t)cpos[(size_t)comp_of[(size_t)(s - s0)]]++] = (int32_t)s;
    for (int32_t v : touched) parent[v] = -1;
    for (int32_t rt : roots) root_comp[rt] = -1;
  }
  h->day_comp[T] = (int32_t)comp_off.size();
  comp_off.push_back((int32_t)comp_ev.size());
  // records in component order beside their positions: each thread streams its list
  std::vector<int4> rec_c(comp_ev.size());
  for (size_t i = 0; i < comp_ev.size(); ++i) rec_c[i] = rec[comp_ev[i]];
  cudaError_t e = galloc(&h->d_rec, rec_c.size());
  if (e == cudaSuccess) e = galloc(&h->d_comp_ev, comp_ev.size());
  if (e == cudaSuccess) e = galloc(&h->d_comp_off, comp_off.size());
  if (e == cudaSuccess) e = cudaMemcpy(h->d_rec, rec_c.data(), rec_c.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_comp_ev, comp_ev.data(), comp_ev.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_comp_off, comp_off.data(), comp_off.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_events(h);
    return gcuda(h, e, "event schedule upload");
  }
  return SIM_OK;
}

sim_status gen_run_days(gen_handle* h, int32_t ndays, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (ndays < 0 || (int64_t)h->day + ndays > h->cfg.max_days)
    return gfail(h, SIM_E_INVALID_ARG, "ndays %d from day %d passes max_days %d", ndays, h->day, h->cfg.max_days);
  if (ndays == 0) return SIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t d0 = h->day;
  if (h->launch_mode == 1) {
    if (!h->graph_exec || h->graph_d0 != d0 || h->graph_nd != ndays) {
      free_graph(h);
      cudaStream_t cs;
      GCK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
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
      if (e != cudaSuccess) { h->graph_exec = nullptr; return gcuda(h, e, "day-loop graph capture"); }
      h->graph_d0 = d0;
      h->graph_nd = ndays;
    }
    GCK(h, cudaGraphLaunch(h->graph_exec, st), "day-loop graph launch");
  } else {
    sim_status s = enqueue_days(h, d0, ndays, st);
    if (s != SIM_OK) return s;
  }
  h->day = d0 + ndays;
  return SIM_OK;
}

sim_status gen_state(gen_handle* h, int32_t* counts, double* y, int32_t* day, int32_t where, void* stream) {
  if (!h) return SIM_E_INVALID_ARG;
  if (where != SIM_HOST && where != SIM_DEVICE) return gfail(h, SIM_E_INVALID_ARG, "where must be SIM_HOST or SIM_DEVICE");
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == SIM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t R = (size_t)h->cfg.n_replicates, N = (size_t)h->cfg.n_nodes;
  if (counts) GCK(h, cudaMemcpyAsync(counts, h->d_counts, R * h->nc * N * 4, k, st), "copy counts");
  if (y && h->ny > 0) GCK(h, cudaMemcpyAsync(y, h->d_y, R * h->ny * N * 8, k, st), "copy y");
  GCK(h, cudaStreamSynchronize(st), "stream synchronize");
  if (day) *day = h->day;
  return latched(h);
}

sim_status gen_set_state(gen_handle* h, const int32_t* counts, const double* y, int32_t day, int32_t where,
                         void* stream) {
  if (!h || !counts || (h->ny > 0 && !y)) return SIM_E_INVALID_ARG;
  if (where != SIM_HOST && where != SIM_DEVICE) return gfail(h, SIM_E_INVALID_ARG, "where must be SIM_HOST or SIM_DEVICE");
  if (day < 0 || day > h->cfg.max_days) return gfail(h, SIM_E_INVALID_ARG, "day %d out of range", day);
  const size_t R = (size_t)h->cfg.n_replicates, N = (size_t)h->cfg.n_nodes;
  const size_t nx = R * h->nc * N, nyv = R * h->ny * N;
  if (where == SIM_HOST) {
    for (size_t i = 0; i < nx; ++i)
      if (counts[i] < 0) return gfail(h, SIM_E_INVALID_ARG, "counts[%zu] < 0", i);
    for (size_t i = 0; i < nyv; ++i)
      if (!finite_nonneg(y[i])) return gfail(h, SIM_E_INVALID_ARG, "y[%zu] must be finite and >= 0", i);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == SIM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GCK(h, cudaMemcpyAsync(h->d_counts, counts, nx * 4, k, st), "copy counts");
  if (nyv) GCK(h, cudaMemcpyAsync(h->d_y, y, nyv * 8, k, st), "copy y");
  GCK(h, cudaStreamSynchronize(st), "stream synchronize");
  free_graph(h);
  h->day = day;
  return SIM_OK;
}

sim_status gen_counters(gen_handle* h, int64_t* counters) {
  if (!h || !counters) return SIM_E_INVALID_ARG;
  GCK(h, cudaDeviceSynchronize(), "synchronize");
  GCK(h, cudaMemcpy(counters, h->d_ctr, (size_t)h->cfg.n_replicates * 4 * 8, cudaMemcpyDeviceToHost), "copy counters");
  return SIM_OK;
}

sim_status gen_set_option(gen_handle* h, int32_t option, int64_t value) {
  if (!h) return SIM_E_INVALID_ARG;
  if (option == GEN_OPT_LAUNCH) {
    if (value != 0 && value != 1) return gfail(h, SIM_E_INVALID_ARG, "launch mode %lld unknown", (long long)value);
    free_graph(h);
    h->launch_mode = (int32_t)value;
    return SIM_OK;
  }
  if (option == GEN_OPT_WARP_THRESHOLD) {
    if (value < -1 || value > INT32_MAX) return gfail(h, SIM_E_INVALID_ARG, "warp threshold %lld", (long long)value);
    free_graph(h);
    h->warp_threshold = (int32_t)value;
    set_n_big(h);
    return SIM_OK;
  }
  if (option == GEN_OPT_GROUP_THRESHOLD) {
    if (value < -1 || value > INT32_MAX) return gfail(h, SIM_E_INVALID_ARG, "group threshold %lld", (long long)value);
    free_graph(h);
    h->group_threshold = (int32_t)value;
    set_n_big(h);
    return SIM_OK;
  }
  if (option == GEN_OPT_CLOCK_MARGIN) {
    if (value < 0 || value > 16) return gfail(h, SIM_E_INVALID_ARG, "clock margin exponent %lld outside [0, 16]", (long long)value);
    free_graph(h);
    h->clock_margin_log2 = (int32_t)value;
    return SIM_OK;
  }
  return gfail(h, SIM_E_INVALID_ARG, "option %d unknown", option);
}

int32_t gen_warp_nodes(const gen_handle* h) { return h ? h->n_big : -1; }

int32_t gen_group_nodes(const gen_handle* h) { return h ? h->n_mid : -1; }

void gen_destroy(gen_handle* h) {
  if (!h) return;
  free_graph(h);
  cudaFree(h->d_counts); cudaFree(h->d_y); cudaFree(h->d_mid); cudaFree(h->d_order); cudaFree(h->d_model);
  cudaFree(h->d_params); cudaFree(h->d_ctr); cudaFree(h->d_err);
  cudaFree(h->d_rec); cudaFree(h->d_comp_ev); cudaFree(h->d_comp_off);
  delete h;
}

const char* gen_last_error(const gen_handle* h) { return h ? h->err.c_str() : g_gen_create_error.c_str(); }

}  // extern "C"
