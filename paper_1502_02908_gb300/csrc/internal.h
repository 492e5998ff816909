// Internal interfaces between the host side of libepisim (host.cpp) and its
// CUDA kernels.  Not part of the public ABI (include/episim.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/episim.h"

namespace episim {

constexpr int kMaxAge = 3;
constexpr int kMaxComp = 2 * kMaxAge;

// Per-replicate constants, 128 bytes.
struct DevParams {
  double ups[3];
  double gam[3];
  double alpha;
  double beta[4];
  double eps;
  double pad[4];
};
static_assert(sizeof(DevParams) == 128, "DevParams layout");

// Score-function accumulators per node: [upsilon_1..3, gamma_1..3, beta, alpha].
constexpr int kScoreTerms = 8;
// Moment sums per listed day of the score-function gradient (sim_gradient_moments):
// sum f, sum f^2; per score term k: sum s_k, sum s_k^2, sum f s_k, sum (f s_k)^2;
// then per k: sum f s_k^2.
constexpr int kMoments = 2 + 5 * kScoreTerms;

struct SsaArgs {
  int32_t* counts;            // [R][Nc][N]
  double* phi;                // [R][N]
  const DevParams* params;    // [R]
  unsigned long long* prev_i; // [R][max_days]
  unsigned long long* prev_n; // [R][max_days]
  unsigned long long* ctr;    // [R][4]
  double* score;              // [R][8][N] (score mode)
  double* tang;               // [R][2][N]: d phi/d beta, d phi/d alpha (score mode)
  uint64_t seed;
  int32_t rep_base;           // Philox replicate word = rep_base + r
  int32_t N, R, Nc, max_days;
  int32_t day;                // day simulated by this launch
  int32_t prologue;           // 1: first record stats of day-1 and (post-event mode) update phi
  int32_t pre_event;          // 1: phi update from post-SSA counts in the epilogue
  double* traj;               // reverse-mode score: [3][max_days][R][N] = c_d, phi_d, I_d/N_d (NULL otherwise)
  const int32_t* order;       // node order: first n_big nodes warp-cooperative, the rest per thread (NULL: identity)
  int32_t n_list;             // nodes in the order list (N, or a day's touched list)
  const uint32_t* skip;       // bitmap [N] of nodes this launch leaves out (NULL: none)
  int32_t n_big;              // nodes simulated one per warp
  int32_t n_mid;              // next nodes of the order, one per 8-lane group (dealt grid only)
  int32_t warp_blocks;        // blocks (of 8 warps) given to them
  uint64_t clock_margin;      // Q62 margin of the speculative binary32 clock (0: exact clock only)
  int32_t sm_count;           // SMs of the device (grid of the dealt mapping)
  int32_t overlap;            // launch with programmatic stream serialization
  int32_t max_per_sm;         // dealt grid: at most this many blocks per SM (0: as many as fit)
  int32_t max_warps;          // dealt grid: warps per block (0: 8)
  int32_t node_lo, node_hi;   // nodes this handle simulates without an order list: [node_lo, node_hi)
};

// One scheduled event, 16 bytes: node, dest, position in the day-stable order,
// and kind (bits 0-1) | (cls + 1) (bits 2-3) | count (bits 4-31).
struct EvArgs {
  int32_t* counts;
  const int4* rec;            // records sorted by (day, level, position)
  const int32_t* lvl_start;   // [n_levels + 1] record offsets
  const int32_t* day_lvl;     // [max_days + 1] level offsets of each day
  unsigned long long* ctr;    // [R][4]
  int32_t* err;               // bit 0: underflow under the ERROR policy
  uint64_t seed;
  int32_t rep_base;
  int32_t N, R, Nc;
  int32_t day;
  int32_t underflow_error;
};

// Shared-memory event step: the day's records refer to node slots of the day's
// touched-node list; counts of those nodes, the records, the first Philox block
// of every event and the level offsets are staged in shared memory.
struct EvSmemArgs {
  int32_t* counts;
  const int4* rec;            // {slot_src, slot_dst or -1, position, packed}, execution order
  const int32_t* lvl_start;   // global level offsets (records)
  const int32_t* day_lvl;     // [max_days + 1]
  const int32_t* touched;     // node ids of the day's slots
  const int32_t* day_touch;   // [max_days + 1] offsets into touched
  unsigned long long* ctr;
  int32_t* err;
  uint64_t seed;
  int32_t rep_base;
  int32_t N, R, Nc;
  int32_t day;
  int32_t underflow_error;
  int32_t smem_bytes;
};

cudaError_t launch_events_day_smem(const EvSmemArgs& a, int n_age, cudaStream_t st);

// Owner-computes event step (no levels on the device): thread t applies, in input
// order, the events of the nodes it owns, waiting on shared-memory counters for
// the transfers into a node that precede a sampling of it and for the samplings of
// a destination that precede a transfer into it.
constexpr int kDfThreads = 128;
constexpr int kEventWaitTimeout = 4;      // error bit: an event-step wait ran out
constexpr int kDfAcquire = 1;             // the event waited on another thread's counter
constexpr int kDfPublishSampling = 2;     // a later transfer into its node waits on it
constexpr int kDfPublishAdd = 4;          // a later sampling of its destination waits on it
struct EvDfArgs {
  int32_t* counts;
  const int4* rec;            // per block: grouped by owner thread, input order within
  const int4* wait;           // {adds into src before it, samplings of dst before it, flags, 0}
  const int32_t* thr_off;     // per block: event offsets of the owner threads in use (block-relative), + end
  const int32_t* thr_id;      // aligned with thr_off: those threads' indices
  const int32_t* touched;     // node ids per block slot
  const int4* blk_meta;       // [blocks + 1]: first record, first node, first thr_off entry,
                              // heavy warps | (1 << 16 when threads own whole components)
  unsigned long long* ctr;
  int32_t* err;
  uint64_t seed;
  int32_t rep_base;
  int32_t N, R, Nc;
  int32_t day;
  int32_t nblk;               // blocks per replicate this day
  int32_t blk0;               // the day's first block
  int32_t overlap;            // launch with programmatic stream serialization
  int32_t underflow_error;
  int32_t smem_bytes;
  int32_t spin_limit;
};
cudaError_t launch_events_day_df(const EvDfArgs& a, int n_age, cudaStream_t st);

// Launch with programmatic stream serialization when pdl is set: the kernel may
// be scheduled while the previous one in the stream finishes, and waits for it
// with griddepcontrol.wait where it reads that kernel's results.
template <class... P, class... A>
inline cudaError_t launch_maybe_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    bool pdl, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
size_t events_df_smem_bytes(int64_t n_events, int64_t n_touched, int nc);

// Dataflow day loop (flow.cu): one persistent kernel over a call's days; warps
// take stochastic-step units and groups of 32 transfer-graph components from one
// counter and wait on per-herd readiness words (half-days).
constexpr int kFlowThreads = 256;
constexpr int kFlowSlots = 8;     // herds of a component staged in a lane's shared-memory slots
constexpr int kFlowLong = 4;      // components of at least this many events get a warp each
struct FlowParts {
  SsaArgs ssa;                    // the stochastic step (day and prologue set per item)
  EvArgs ev;                      // the event step (counts, counters, error word, seed)
  int32_t* err_word;              // the handle's latched error word
};
struct FlowArgs {
  FlowParts a;
  const int4* rec;                // per component, input order: {src slot, dst slot, position, packed}
  const int32_t* cev;             // [components + 1] record offsets
  const int32_t* cnode;           // component herds by slot
  const int32_t* cnoff;           // [components + 1] offsets into cnode
  const int32_t* day_comp;        // [max_days + 1] first component of each day (longest first)
  const int32_t* day_long;        // [max_days] the day's components of >= kFlowLong events (they come first)
  const int32_t* cunit;           // the distinct stochastic-step units of each component's herds
  const int32_t* cuoff;           // [components + 1] offsets into cunit
  const int32_t* K;               // [max_days + 1][U1]: components touching each unit before each day
  int32_t U1;                     // stochastic-step units per replicate
  unsigned* unit_cnt;             // [R][U1] completion counters
  unsigned stall_extra;           // test hook: added to the first unit's first wait (0: none)
  unsigned long long* next;       // item counter
  int32_t* abort;
  long long spin_limit;           // polls a wait makes before giving up
  int32_t d0, ndays;
  long long units;                // stochastic-step units per day (all replicates)
  const long long* item_off;      // [ndays + 1] first item of each day of the call
};
// Clears the unit counters, the item counter and the abort flag, and launches
// the persistent kernel on a resident grid (sms x blocks per SM).
cudaError_t launch_flow(const FlowArgs& f, int n_age, int sms, cudaStream_t st);
// Shared memory the staged event step needs for a day (0 if the day has no events).
size_t events_smem_bytes(int64_t n_events, int64_t n_levels, int64_t n_touched, int nc);
constexpr size_t kEventsSmemLimit = 220 * 1024;
constexpr size_t kBatchSmemSM = 220 * 1024;       // shared memory of the persistent batch blocks of an SM

struct FinalizeArgs {
  SsaArgs s;                  // day = last simulated day; prologue semantics for day+1
};

cudaError_t launch_ssa_day(const SsaArgs& a, int n_age, bool score, cudaStream_t st);
// Region totals of day `day` for every replicate, added (and squared) into s1 / s2
// [max_days][J][Nc]; the goal terms over count entries of s1 / s2 from `first`.
cudaError_t launch_region_day(const int32_t* counts, const int32_t* reg_nodes, const int32_t* reg_off, int N, int R,
                              int Nc, int J, int day, unsigned long long* s1, unsigned long long* s2,
                              cudaStream_t st);
cudaError_t launch_goal(const unsigned long long* s1, const unsigned long long* s2, const long long* ref,
                        long long first, long long count, int R, double* out, cudaStream_t st);
cudaError_t launch_events_day(const EvArgs& a, int n_age, cudaStream_t st);
// After the last day of a call: phi update (post-event mode) and statistics of day a.day.
cudaError_t launch_finalize(const SsaArgs& a, int n_age, bool score, cudaStream_t st);
// node-sharded exchange (shard.cu): counts of the day's touched herds, [R][Nc][n_t]
cudaError_t launch_pack_touched(const int32_t* counts, const int32_t* touched, int n_t, int N, int64_t planes,
                                int32_t* out, cudaStream_t st);
cudaError_t launch_unpack_touched(int32_t* counts, const int32_t* touched, int n_t, int N, int64_t planes,
                                  const int32_t* in, const int32_t* bounds, int world, cudaStream_t st);
cudaError_t launch_debug_neglog(const uint64_t* j, double* out, int64_t n, cudaStream_t st);
cudaError_t launch_debug_neglog_f32(const uint64_t* j, float* out, int64_t n, cudaStream_t st);

// Reverse sweep of the phi recursion over days [0, ndays) for every (r, v):
// lambda_d = c_d + (1 - beta_d) lambda_{d+1}; adds -lambda_{d+1} phi_d to the
// beta score and lambda_{d+1} q_d to the alpha score of the node.
cudaError_t launch_phi_backward(const double* traj, const DevParams* params, double* score, int N, int R,
                                int max_days, int ndays, cudaStream_t st);
// Per replicate: f = infected/animals after each listed day, s = score summed over
// nodes; moments per listed day [n_days][34]: sum f, sum f^2, then per score term
// k: sum s_k, sum s_k^2, sum f s_k, sum (f s_k)^2.
cudaError_t launch_gradient_moments(const double* score, const unsigned long long* prev_i,
                                    const unsigned long long* prev_n, const int32_t* days, int n_days, int N,
                                    int R, int max_days, double* per_rep /*[R][8]*/, double* out, cudaStream_t st);
cudaError_t launch_debug_div(const double* x, const double* y, double* out, double* ref, int64_t n, cudaStream_t st);

}  // namespace episim

namespace episim {
// dst holds `copies` back-to-back copies of the `bytes` bytes at src (device pointers).
cudaError_t launch_broadcast(void* dst, const void* src, size_t bytes, int copies, cudaStream_t st);
}  // namespace episim

struct sim_handle;
namespace episim {
// Read-only view of a handle's score state for entry points outside host.cpp.
struct HandleScoreView {
  const double* score;
  const unsigned long long* prev_i;
  const unsigned long long* prev_n;
  int N, R, max_days;
};
sim_status handle_score_view(sim_handle* h, HandleScoreView* out);
sim_status handle_fail(sim_handle* h, sim_status s, const char* msg);
sim_status handle_cuda_fail(sim_handle* h, cudaError_t e, const char* what);
// The handle's latched device error (underflow under the ERROR policy, an event
// wait that ran out), read and cleared as every synchronising entry point does.
sim_status handle_check_latched(sim_handle* h);
}  // namespace episim
