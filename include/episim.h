/*
 * episim.h — C ABI of the GB300 event-based epidemic simulation library
 * (libepisim.so), after Bauer, Engblom & Widgren, "Fast event-based
 * epidemiological simulations on national scales" (arXiv:1502.02908).
 *
 * One simulated day, for every node (herd) and every replicate, is
 *   1. the stochastic step: Gillespie's direct method per node on [d, d+1)
 *      with the environmental variable phi frozen (Sec. 3.1 Eq. (numstep3);
 *      Sec. 3.3 Eqs. (sampling), (sampling2); the per-node loop of Alg. 1);
 *   2. the deterministic step: the day's scheduled events, applied so that the
 *      result equals their input order (Sec. 3.2 Eq. (event); Sec. 3.3; the event
 *      step of Alg. 1);
 *   3. the continuous-state update phi <- phi (1 - beta) + alpha I / N + epsilon
 *      (Eq. (numstep5) with Eq. (siminfpressure); the last step of Alg. 1's day).
 * Models: SISe (compartments S, I; S->I at upsilon phi S, I->S at gamma I) and
 * SISe3 (the same per age class; Sec. 4.1 Eqs. (vtectrans)-(recovery_rates)).
 *
 * Conventions
 *   - Compartments inside a node are class-major: SISe [S, I]; SISe3
 *     [S1, I1, S2, I2, S3, I3].  Count arrays are int32 [R][Nc][N] (replicate,
 *     compartment, node); phi is double [R][N].
 *   - "host" pointers are read or written by the CPU; "device" pointers are
 *     CUDA global-memory addresses on the current device.
 *   - Every call returns a sim_status and never aborts or prints; the text of
 *     the last error is sim_last_error(h).  Outputs are written only on SIM_OK.
 *   - A handle belongs to one host thread at a time.  It owns all device memory
 *     it allocates; it never frees memory the caller owns.
 *   - Randomness is counter-based (Philox4x32-10): results do not depend on the
 *     launch configuration, on how days are split across calls, or on which
 *     other replicates run alongside.
 */
#ifndef EPISIM_H
#define EPISIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sim_status {
    SIM_OK = 0,
    SIM_E_INVALID_ARG = 1,   /* an argument is out of range; nothing changed      */
    SIM_E_OOM = 2,           /* host or device allocation failed                  */
    SIM_E_CUDA = 3,          /* a CUDA call failed (launch, copy, stream)         */
    SIM_E_UNDERFLOW = 4,     /* ERROR policy: an event asked for absent animals   */
    SIM_E_TIMEOUT = 5,       /* a bounded device-side wait ran out                */
    SIM_E_STATE = 6          /* call not valid in the handle's current state      */
} sim_status;

enum { SIM_SISE = 1, SIM_SISE3 = 3 };
enum { SIM_UNDERFLOW_CLAMP = 0, SIM_UNDERFLOW_ERROR = 1 };
enum { SIM_EXIT = 0, SIM_ENTER = 1, SIM_INTERNAL = 2, SIM_EXTERNAL = 3 };
enum { SIM_HOST = 0, SIM_DEVICE = 1 };
/* sim_config.flags */
enum {
    SIM_FLAG_PHI_PRE_EVENT = 1,  /* phi from post-SSA, pre-event counts (Eq. (numstep5) as printed) */
    SIM_FLAG_SCORE = 2,          /* accumulate score-function terms (sim_score); the beta and
                                    alpha terms through forward tangents of phi */
    SIM_FLAG_SCORE_REVERSE = 4   /* score terms with the beta and alpha terms left to a reverse
                                    sweep (sim_score_backward) over a stored per-day trajectory
                                    of 24 bytes per node-day-replicate; implies SIM_FLAG_SCORE */
};

typedef struct sim_config {
    int32_t model;            /* SIM_SISE or SIM_SISE3 */
    int32_t n_nodes;          /* N >= 1 */
    int32_t n_replicates;     /* R >= 1 */
    int32_t max_days;         /* horizon; days [0, max_days) can be simulated */
    int32_t underflow_policy; /* SIM_UNDERFLOW_CLAMP (default) or SIM_UNDERFLOW_ERROR */
    int32_t flags;            /* SIM_FLAG_* */
    uint64_t seed;            /* Philox key */
    int32_t replicate_base;   /* replicate r of this handle draws as replicate
                                 replicate_base + r (disjoint streams when
                                 replicates are split across handles or GPUs) */
    int32_t reserved;         /* must be 0 */
} sim_config;

/* Per-replicate model constants, host arrays with a leading replicate axis:
 * upsilon, gamma [R][3] (SISe reads column 0), alpha, epsilon [R], beta [R][4]:
 * decay for day-of-year bins [0,91], (91,182], (182,273], (273,364] (Sec. 4.1). */
typedef struct sim_params {
    const double* upsilon;
    const double* gamma;
    const double* alpha;
    const double* beta;
    const double* epsilon;
} sim_params;

typedef struct sim_handle sim_handle;

/* Creates a simulation at day 0: the initial discrete state X (the Nc x N
 * integer state matrix of Sec. 2.2, Eq. (local)) and the continuous state Y = phi
 * (one variable per node, Sec. 2.3 Eq. (master_det); Sec. 4.1 Eq.
 * (siminfpressure)), with the rate constants of Sec. 4.1 Eqs. (vtectrans)-
 * (recovery_rates) -- the initialisation that precedes Alg. 1's time loop.
 * u0: host int32 [Nc][N] initial counts, the same for every replicate (>= 0);
 * phi0: host double [N]; params: see sim_params.  All inputs are copied.
 * Allocates the device state on the current device.  Errors: SIM_E_INVALID_ARG
 * (a size, count or constant out of range, named in sim_last_error(NULL)),
 * SIM_E_OOM, SIM_E_CUDA.  *out is set only on SIM_OK. */
sim_status sim_create(const sim_config* cfg, const int32_t* u0, const double* phi0,
                      const sim_params* params, sim_handle** out);

/* As sim_create, with the live state in the caller's device memory (e.g. the
 * storage of framework tensors): dev_counts int32 [R][Nc][N] and dev_phi double
 * [R][N], 16-byte aligned, on the current device.  The call synchronises
 * `stream` (so the caller's earlier work on the buffers is done), writes the
 * initial state into them, and from then on every step reads and writes them in
 * place; sim_state / sim_set_state still copy.  The library never frees them:
 * they must stay allocated until sim_destroy.  Errors as sim_create, and
 * SIM_E_INVALID_ARG for a buffer that is not aligned device memory of the
 * current device. */
sim_status sim_create_on(const sim_config* cfg, const int32_t* u0, const double* phi0,
                         const sim_params* params, int32_t* dev_counts, double* dev_phi, void* stream,
                         sim_handle** out);

/* Loads the scheduled events (Sec. 3.2 Eq. (event)): n host int32 arrays in
 * input order.  kind: SIM_EXIT / SIM_ENTER / SIM_INTERNAL (aging: class cls to
 * cls+1 of the same node) / SIM_EXTERNAL (node -> dest).  cls: age class, or -1
 * for "every class" (ENTER then means class 0).  count >= 0.  dest is read only
 * for SIM_EXTERNAL and must differ from node.  Events on days >= max_days are
 * kept but never reached.  Builds the per-day dependency levels (host, O(n)) and
 * uploads them.  Callable once per handle, at day 0 (again after sim_reset with
 * events cleared by sim_reset(h, 1)).  Errors: SIM_E_INVALID_ARG naming the first
 * bad event, SIM_E_OOM, SIM_E_STATE. */
sim_status sim_load_events(sim_handle* h, int64_t n, const int32_t* day, const int32_t* kind,
                           const int32_t* node, const int32_t* dest, const int32_t* count,
                           const int32_t* cls);

/* Advances every replicate by ndays days (ndays >= 0, day + ndays <= max_days):
 * per day the stochastic step, the day's events and the phi update, i.e. ndays
 * iterations of Alg. 1's time loop (Sec. 3.1 Eqs. (numstep3)-(numstep5), one
 * day per step of Eq. (numerical)), asynchronously on the CUDA stream `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Returns launch errors at once.  Device-side conditions
 * (SIM_E_UNDERFLOW under the ERROR policy) are latched and returned by the next
 * synchronising call (sim_state, sim_stats, sim_score, sim_sync). */
sim_status sim_run_days(sim_handle* h, int32_t ndays, void* stream);

/* Waits for the handle's work on `stream` and returns any latched device error
 * (the day boundary t_{n+1} of Alg. 1 made observable to the host). */
sim_status sim_sync(sim_handle* h, void* stream);

/* Copies the state at the start of the current day -- X (Sec. 2.2 Eq. (local))
 * and Y = phi (Sec. 2.3) after the previous day's events and phi update
 * (Eqs. (numstep4), (numstep5)): counts int32 [R][Nc][N], phi double [R][N]
 * (either may be NULL), and *day.  where = SIM_HOST or
 * SIM_DEVICE says what the output pointers are.  Synchronises `stream`. */
sim_status sim_state(sim_handle* h, int32_t* counts, double* phi, int32_t* day, int32_t where,
                     void* stream);

/* Replaces the state (checkpoint restore): X and Y = phi (Secs. 2.2, 2.3) at the
 * start of day `day` (0 <= day <= max_days), the point where Alg. 1's time loop
 * resumes: counts [R][Nc][N] (>= 0) and phi [R][N].  Errors: SIM_E_INVALID_ARG
 * (a negative count, a negative or non-finite phi, day out of range), SIM_E_CUDA.  Runs resumed from a state
 * taken by sim_state are bit-identical to uninterrupted runs.  Statistics of
 * days >= day are cleared.  Synchronises `stream`. */
sim_status sim_set_state(sim_handle* h, const int32_t* counts, const double* phi, int32_t day,
                         int32_t where, void* stream);

/* Daily statistics since day 0 -- the national totals of I and of all animals
 * that the goal function of Sec. 4.3 (Eq. (goal)) and the prevalence curves of
 * Sec. 4.1 aggregate: infected[R][max_days] and animals[R][max_days] (after each
 * day's events; int64), counters[R][4] = SSA transitions fired,
 * events applied, events clamped, events skipped (ERROR policy).  Any output
 * may be NULL.  Host pointers.  Synchronises `stream`. */
sim_status sim_stats(sim_handle* h, int64_t* infected, int64_t* animals, int64_t* counters,
                     void* stream);

/* Score-function terms (needs SIM_FLAG_SCORE): per node, d log p(path) /
 * d theta for theta = [upsilon_1..3, gamma_1..3, beta, alpha], double
 * [R][8][N] (host), accumulated since day 0 (or since the last sim_reset /
 * sim_set_state).  The likelihood of a path is the product of the fired
 * transitions' rates times exp(-integral of a0), from the direct method's
 * sampling law; phi's dependence on beta and alpha is carried through Eq.
 * (numstep5).  Synchronises `stream`. */
sim_status sim_score(sim_handle* h, double* score, void* stream);

/* Reverse sweep of the phi recursion (needs SIM_FLAG_SCORE_REVERSE), on the
 * device: for every node and replicate, over the days simulated since the score
 * was last cleared, lambda_d = c_d + (1 - beta_d) lambda_{d+1} with c_d the
 * node-day's d log p / d phi_d; adds sum_d -lambda_{d+1} phi_d to the beta term
 * and sum_d lambda_{d+1} (I_d / N_d) to the alpha term of the node's score
 * (Eq. (numstep5) with Eq. (siminfpressure) differentiated in reverse).  Call
 * once per run, after the last sim_run_days.  Asynchronous on `stream`. */
sim_status sim_score_backward(sim_handle* h, void* stream);

/* Moments for the score-function gradient estimate, on the device: for each
 * replicate, f = infected / animals after day days[i] (i < n_days) and s = its
 * score summed over nodes; writes per_rep [R][8] (may be NULL) and out
 * [n_days][42] = sum f, sum f^2, then for each of the 8 score terms k:
 * sum s_k, sum s_k^2, sum f s_k, sum (f s_k)^2, then for each k: sum f s_k^2
 * (replicates added in index order).  d E[f] / d theta_k is estimated by the
 * covariance of f and s_k (the likelihood-ratio identity; Sec. 3.3 Eqs.
 * (sampling), (sampling2) give the path's law).
 * Host outputs; synchronises `stream`. */
sim_status sim_gradient_moments(sim_handle* h, const int32_t* days, int32_t n_days, double* per_rep,
                                double* out, void* stream);

/* The score-function estimate from moment sums of sim_gradient_moments: the
 * likelihood-ratio identity d E[f] / d theta = E[f d log p / d theta] (log p the
 * path's log-likelihood under the direct method's law, Sec. 3.3 Eqs. (sampling),
 * (sampling2)), estimated by the sample covariance of f and the score.
 * moments: host double [n_chunks][n_days][42], each chunk the out array of one
 * sim_gradient_moments call (chunks of replicates, added in chunk order); R: the
 * total replicate count (>= 2); jac: host double [8][n_params], d theta_k / d
 * param_c for the 8 score terms of sim_score (e.g. the age-class ratios when one
 * parameter scales upsilon of every class).  Writes, host arrays:
 *   mean_f [n_days]            = sum f / R,
 *   grad   [n_days][n_params]  = sum_k cov(f, s_k) jac[k][c],
 *                               cov = (sum f s_k - sum f sum s_k / R) / (R - 1),
 *   se     [n_days][n_params]  = sqrt(sum_k (V_k / R) jac[k][c]^2), V_k the variance of the
 *                               centred product (f - mean f) s_k from the moment sums,
 *                               max(E[(f - mu)^2 s_k^2] - E[(f - mu) s_k]^2, 0) (the score's
 *                               mean is zero; covariances between terms are left out)
 * (any output may be NULL).  Host arithmetic only; no handle, no device.
 * Errors: SIM_E_INVALID_ARG (n_chunks < 1, n_days < 0, n_params < 1, R < 2, a
 * NULL input). */
sim_status sim_gradient_estimate(const double* moments, int32_t n_chunks, int32_t n_days, int64_t R,
                                 const double* jac, int32_t n_params, double* mean_f, double* grad,
                                 double* se);

/* The same result as sim_gradient_moments, from a call that allocates no
 * memory.  The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc -- code whose device memory belongs to another allocator (a
 * framework's caching pool, an application with a fixed memory budget) or that
 * must avoid the device synchronisation and fragmentation an allocation can
 * cause.  Its scratch is one fixed array in the library's device image (about
 * 690 KiB on every GPU that loads the library, kept until exit), which limits a
 * call to at most 8192 replicates and 512 days; larger requests return
 * SIM_E_INVALID_ARG.  Every call looks the array's address up on the current
 * device; with lazy module loading (the CUDA default) the first lookup on a
 * device is when the runtime places the array in device memory, so make the
 * first call on each device before any stream capture and before measuring free
 * memory.  Every call shares the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  Nothing needs clearing between calls.
 * Returns the handle's latched device error as sim_gradient_moments does.  Host
 * outputs; synchronises `stream`. */
sim_status sim_gradient_moments_noalloc(sim_handle* h, const int32_t* days, int32_t n_days,
                                        double* per_rep, double* out, void* stream);

/* Node-sharded single replicate (Sec. 3.4's split of the nodes over workers with
 * a daily exchange for the crossing events, and Sec. 5's multi-node outlook),
 * one handle per rank, each holding the whole state:
 *   sim_shard restricts the handle's stochastic step, phi update and statistics
 *   (Eqs. (numstep3), (numstep5)) to nodes [node_lo, node_hi); the daily
 *   statistics and the transition counter then sum those nodes only, while every
 *   rank applies the whole event list (Eq. (numstep4)) and counts every event.
 *   Call at day 0, after sim_load_events or before; not with SIM_FLAG_SCORE or
 *   region statistics (SIM_E_STATE), not in sim_run_batch.  Synchronises the device.
 *   A day then runs in two halves: sim_run_day_stochastic (the stochastic step of
 *   the current day, own nodes) and sim_run_day_events (the day's events on every
 *   node, then the phi update and statistics of the own nodes; the day advances).
 *   Between them the ranks exchange the post-stochastic-step counts of the herds
 *   the day's events touch: sim_touched_count(h, day) herds (host; -1 for a bad
 *   day), listed by sim_touched_nodes (host int32 [n]); sim_pack_touched writes
 *   their counts as device int32 [R][Nc][n] into the caller's buffer; the caller
 *   gathers the world ranks' packs back to back in rank order (e.g. an all-gather
 *   over NCCL) and sim_unpack_touched takes, for every touched herd, the counts
 *   from the pack of the rank that owns it -- bounds: host int32 [world + 1],
 *   rank k owns [bounds[k], bounds[k+1]), bounds[0] = 0, bounds[world] = N,
 *   non-decreasing.  With every rank doing this the counts of each rank's own
 *   nodes equal a single handle's sim_run_days bit for bit (the random numbers
 *   are keyed by node, day and event position, not by rank).  The two halves and
 *   the pack and unpack are asynchronous on `stream`; sim_unpack_touched
 *   synchronises it before reading `bounds`.  While a day is between its halves,
 *   sim_run_days, sim_state and sim_set_state return SIM_E_STATE.  Any handle
 *   (sharded or not) may run its days in halves; with no exchange an unsharded
 *   handle's halves equal sim_run_days. */
sim_status sim_shard(sim_handle* h, int32_t node_lo, int32_t node_hi);
sim_status sim_run_day_stochastic(sim_handle* h, void* stream);
sim_status sim_run_day_events(sim_handle* h, void* stream);
int32_t sim_touched_count(const sim_handle* h, int32_t day);
sim_status sim_touched_nodes(const sim_handle* h, int32_t day, int32_t* nodes);
sim_status sim_pack_touched(sim_handle* h, int32_t* dev_out, void* stream);
sim_status sim_unpack_touched(sim_handle* h, const int32_t* dev_in, int32_t world, const int32_t* bounds,
                              void* stream);

/* Back to day 0 with the initial counts and phi of sim_create (the initial
 * state X_0, Y_0 of Sec. 3.1's time discretisation); statistics and score
 * cleared.  clear_events = 1 also drops the loaded events (Sec. 3.2's lists
 * E1, E2).  Synchronises the device.  Errors: SIM_E_CUDA. */
sim_status sim_reset(sim_handle* h, int32_t clear_events);

/* Frees everything the handle owns (the device state X, Y and the event
 * schedule of Secs. 2.2, 2.3 and 3.4); caller-owned buffers of sim_create_on
 * are left alone.  Synchronises the device.  NULL is accepted. */
void sim_destroy(sim_handle* h);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle.  NULL handle: text of the last sim_create failure. */
const char* sim_last_error(const sim_handle* h);

/* Event preprocessing alone, on the host, with no device and no handle: the
 * validation and execution schedule sim_load_events builds (stable sort by day,
 * then per-day dependency levels; Sec. 3.4 rearrangement with the ordering rule
 * 2(b) of Sec. 3.6 applied per node).  For the n input events (same arrays and
 * rules as sim_load_events) it writes, for the *n_scheduled events on days
 * < max_days, in execution order (day, level, position): order[k] = the event's
 * position in the day-stable order, level[k] = its level (>= 1).  Outputs are
 * host arrays of at least n entries; any may be NULL.  Applying the levels in
 * order, each level in any order, equals applying the events in input order. */
sim_status sim_schedule_events(int32_t n_nodes, int32_t model, int32_t max_days, int64_t n,
                               const int32_t* day, const int32_t* kind, const int32_t* node,
                               const int32_t* dest, const int32_t* count, const int32_t* cls,
                               int64_t* order, int32_t* level, int64_t* n_scheduled);

/* Launch shape of the stochastic step.  Nodes whose initial herd has at least
 * warp_herd_threshold animals are simulated one per warp (the 32 lanes draw
 * and time 32 steps at once; suited to herds with many transitions per day);
 * the others one per thread.  -1 = automatic (warps for herds of >= 400 animals
 * while node-replicates number fewer than 152 x 1024, else none); a very large
 * value disables the warp path.  Results do not depend on this setting.  Score
 * mode always uses one thread per node.  Synchronises the device. */
sim_status sim_tune(sim_handle* h, int32_t warp_herd_threshold);
/* Number of nodes currently simulated one per warp (-1 for a NULL handle). */
int32_t sim_warp_nodes(const sim_handle* h);

/* Execution options (results never depend on them):
 *   SIM_OPT_WARP_THRESHOLD: as sim_tune.
 *   SIM_OPT_GROUP_THRESHOLD: herds below the warp threshold with at least this
 *     many animals (initial herd) are simulated four to a warp, eight lanes each
 *     drawing eight steps at a time; -1 = automatic (200 while node-replicates
 *     number fewer than 152 x 1024, else none), a very large value disables it.
 *   SIM_OPT_CLOCK_MARGIN: k in [0, 17].  The stochastic step (outside score
 *     mode) first runs each node-day with a binary32 clock accumulated in fixed
 *     point, whose distance to the binary64 clock of Eq. (numstep3) is bounded
 *     below 2^-17 of a day; a stop/continue decision within 2^-k of the day's end
 *     reruns the node-day with the exact binary64 arithmetic.  k = 17 (default)
 *     is the tightest safe margin; smaller k only reruns more node-days; 0 runs
 *     every node-day exactly.  Values outside [0, 17]: SIM_E_INVALID_ARG.
 *   SIM_OPT_OVERLAP: 1 (default) launches the day's stochastic-step and event
 *     kernels with programmatic dependent launch (each waits for the previous
 *     kernel only where it reads that kernel's results, so setup and launch
 *     latency overlap the previous kernel's tail); 0 plain stream order.
 *   SIM_OPT_SPLIT: 1 runs the stochastic step of a day that follows a
 *     day with events as two launches: the herds the previous day's events left
 *     untouched, on a second stream alongside that event step (they do not depend
 *     on it), and the touched herds after it; 0 (default) one launch per day.  The calling
 *     stream is joined before every event step and at the end of the call.
 *   SIM_OPT_LAUNCH: how sim_run_days issues a call's days -- SIM_LAUNCH_STREAM
 *     (two launches per day on the stream), SIM_LAUNCH_GRAPH (the call's launch
 *     sequence captured once as a CUDA graph, keyed by start day and day count,
 *     and replayed), SIM_LAUNCH_PERSISTENT (one persistent batch-kernel launch,
 *     synchronous), SIM_LAUNCH_FLOW (the call's days as one dataflow launch with
 *     no per-day barrier: warps take the stochastic step of groups of herds and
 *     the events of groups of transfer-graph components from one counter in day
 *     order, each waiting only for its own herds' previous half-day -- a herd
 *     the day's events leave untouched starts its next day as soon as its own
 *     day is done, as the paper's tasks do (Sec. 3.4, Alg. 2); the day's
 *     components are built on the host at the first such call; bounded waits
 *     return SIM_E_TIMEOUT from the next synchronising call; asynchronous; falls
 *     back to stream launches in score mode, with region statistics or on a
 *     node range).  Under tracing (sim_profile), SIM_LAUNCH_GRAPH runs a
 *     one-shot graph with the event records inside, the other modes stream
 *     launches. */
enum { SIM_OPT_WARP_THRESHOLD = 1, SIM_OPT_LAUNCH = 2, SIM_OPT_CLOCK_MARGIN = 3, SIM_OPT_OVERLAP = 4,
       SIM_OPT_SPLIT = 5, SIM_OPT_GROUP_THRESHOLD = 6 };
enum { SIM_LAUNCH_STREAM = 0, SIM_LAUNCH_GRAPH = 1, SIM_LAUNCH_PERSISTENT = 2, SIM_LAUNCH_FLOW = 3 };
sim_status sim_set_option(sim_handle* h, int32_t option, int64_t value);

/* Replaces every replicate's parameters (same layout and checks as sim_create;
 * invalid values: SIM_E_INVALID_ARG, nothing changed).  The state, events and
 * statistics stay; the next sim_run_days uses the new values.  Synchronises the
 * device.  (For parameter searches: no rebuild of the event schedule.) */
sim_status sim_set_params(sim_handle* h, const sim_params* p);

/* Region statistics of the parameter-fitting goal (Sec. 4.3, Eqs. (goal),
 * (goalvariance), (goalsigma)).  sim_set_regions assigns every node a region
 * (region_of_node [N] host, values in [0, n_regions); n_regions = 0 switches the
 * statistics off); from then on, after each simulated day d, every replicate's
 * region totals x_jc (sum over region j's nodes of compartment c) are added into
 * s1[d][j][c] = sum over replicates of x_jc and s2[d][j][c] = sum of x_jc^2, exact
 * uint64 (one extra launch per day; not with SIM_LAUNCH_PERSISTENT, which then
 * fails with SIM_E_STATE; the split day step is off meanwhile).  sim_set_state at
 * day D clears rows >= D; sim_reset clears all.
 * sim_region_moments copies s1, s2 [max_days][n_regions][Nc] to host (either may
 * be NULL).  sim_goal computes on the device, over days [day0, day0 + ndays),
 * with R = the handle's replicates as trajectories and ref [ndays][n_regions][Nc]
 * (host int64: a reference trajectory's region totals):
 *   g2  = sum (s1 / R - ref)^2,   vg2 = sum (s2 - s1^2 / R) / (R - 1)
 * (0 when R = 1), each difference and variance formed exactly in 128-bit integers
 * and summed in a fixed order.  Both synchronise the device. */
sim_status sim_set_regions(sim_handle* h, const int32_t* region_of_node, int32_t n_regions);
sim_status sim_region_moments(sim_handle* h, uint64_t* s1, uint64_t* s2);
sim_status sim_goal(sim_handle* h, const int64_t* ref, int32_t day0, int32_t ndays, double* g2, double* vg2);

/* Batched and uneven runs: advances every listed handle (all on the current
 * device; any mix of models, node and replicate counts, horizons, events and
 * parameters) to day until[i] (NULL: each handle's max_days) in ONE persistent
 * work-stealing kernel launch.  Blocks fetch work items -- stochastic-step
 * chunks of an (instance, replicate, day), event steps of an (instance,
 * replicate, day), finalisation chunks -- from one atomic counter in a
 * dependency-respecting order and wait for their inputs with bounded spins.
 * Results are identical to running each handle alone with sim_run_days.
 * Synchronous on `stream`.  A wait that runs out aborts the launch and returns
 * SIM_E_TIMEOUT (the batch's state is then undefined); device errors of a
 * handle are latched in it as for sim_run_days. */
sim_status sim_run_batch(sim_handle** handles, int32_t n, const int32_t* until, void* stream);

/* Block shape of sim_run_batch's persistent kernel (and of SIM_LAUNCH_PERSISTENT)
 * for the calls that follow, process-wide: `threads` threads a block and
 * `blocks_per_sm` resident blocks an SM, one of 256 x 2 (the default), 256 x 1
 * and 128 x 4.  A stochastic-step chunk is one block's worth of nodes, one a
 * thread (or of herds on the warp path, one a warp).  The blocks of an SM share
 * 220 KB of shared memory for the staged event step: a day whose staged step
 * needs more than 220 KB / blocks_per_sm runs the global-memory variant.  More
 * resident blocks hide more of the stochastic step's latency at a register budget
 * of 65,536 / (threads x blocks_per_sm) a thread.  Results do not depend on the
 * shape (every random number is keyed by node, day and event position).  The
 * paper has no counterpart: this is a launch-tuning knob.  Errors:
 * SIM_E_INVALID_ARG for any other shape. */
sim_status sim_batch_shape(int32_t threads, int32_t blocks_per_sm);

/* Test hook for the dataflow loop's failure path: runs ndays days from the
 * current day (>= 1) with SIM_LAUNCH_FLOW, but with the first stochastic-step
 * unit's herd (replicate 0) held at readiness 0, so that its wait makes
 * spin_limit polls, gives up and the launch returns; the call synchronises and
 * returns SIM_E_TIMEOUT with the device usable.  The handle's state is undefined
 * afterwards (sim_reset or sim_set_state it). */
sim_status sim_debug_flow_stall(sim_handle* h, int32_t ndays, int64_t spin_limit);

/* Test hooks for the batch kernel's failure path: sets the number of polls a
 * dependency wait makes before giving up (default ~2 s worth); runs h (whose
 * day must be >= 1) in a batch whose first dependency is never met, so that the
 * wait runs out and the call returns SIM_E_TIMEOUT with the device usable.  The
 * handle's state is undefined afterwards (sim_reset or sim_set_state it). */
sim_status sim_debug_batch_spin_limit(int64_t limit);
sim_status sim_debug_batch_stall(sim_handle* h, int32_t until, int64_t spin_limit);

/* Kernel timing (tracing).  While enabled, every kernel the handle launches is
 * bracketed by CUDA events on its stream.  sim_profile_read synchronises and
 * returns, per kernel kind (0 = stochastic step, 1 = events, 2 = phi/statistics
 * finalisation), the summed device time in ms and the number of launches since
 * the last enable; host arrays of 3 entries. */
sim_status sim_profile(sim_handle* h, int32_t enable);
sim_status sim_profile_read(sim_handle* h, double* ms, int64_t* launches);

/* FP64 pipe throughput of the current device, measured: a kernel whose threads
 * each run 8 independent chains of one binary64 instruction kind (kind 0: fused
 * multiply-add, kind 1: add) for `iters` iterations, over a whole number of waves
 * (blocks per SM from the occupancy API x SMs); best of three timed launches
 * after one warm-up, CUDA events on the legacy default stream.  Writes the
 * instruction-lanes retired per second (*lane_ops_per_s; one FMA counts as one)
 * and the best launch's time (*ms, may be NULL).  The paper has no counterpart:
 * this is the denominator of the stochastic step's arithmetic roofline, since the
 * simulation's specification is binary64 arithmetic (Sec. 3.3 Eqs. (sampling),
 * (sampling2)).  Allocates and frees a few KB of device memory; synchronous.
 * Errors: SIM_E_INVALID_ARG (kind not 0 or 1, iters < 1, NULL output),
 * SIM_E_CUDA. */
sim_status sim_fp64_peak(int32_t kind, int64_t iters, double* lane_ops_per_s, double* ms);

/* Test hook (not part of the simulation path): evaluates the library's
 * -log(u) for u = (2 j + 1) 2^-53 on the GPU, for n device inputs j (uint64)
 * into n device doubles.  Synchronous. */
sim_status sim_debug_neglog(const uint64_t* j_dev, double* out_dev, int64_t n);

/* Test hook (not part of the result): the binary32 -log(u) that the
 * speculative clock of the stochastic step uses (relative error below 2^-20 by
 * construction), for n device inputs j into n device floats.  The paper has no
 * counterpart; it exists so that tests can check that bound.  Synchronous. */
sim_status sim_debug_neglog_f32(const uint64_t* j_dev, float* out_dev, int64_t n);

/* Test hook: the library's integer-pipe IEEE division x / y for positive
 * operands, and the reference IEEE division, on n inputs: where = SIM_HOST runs
 * the same routine on the CPU (host pointers), SIM_DEVICE on the GPU (device
 * pointers; ref then comes from the hardware divide).  Synchronous. */
sim_status sim_debug_div(const double* x, const double* y, double* out, double* ref, int64_t n,
                         int32_t where);

/* Test hook: the event schedule built by sim_load_events, host int64 [n]:
 * the event's position in the day-stable order, listed in execution order
 * (day, then dependency level, then position), and the level of each listed
 * event (int32 [n]).  Either output may be NULL. */
sim_status sim_debug_schedule(const sim_handle* h, int64_t* order, int32_t* level);
/* Test hook choosing the event-step kernel (call before sim_load_events):
 * 0 (default) the owner-computes kernel (each node's events applied in input
 * order by the thread that owns the node, with counter waits for transfers) on
 * days whose working set fits in shared memory, else the level-staged kernel,
 * else the global-memory kernel; 1 the global-memory level kernel on every day;
 * 2 the level kernels only.  All give identical results. */
sim_status sim_debug_event_variant(sim_handle* h, int32_t variant);

/* Number of entries sim_debug_schedule writes (-1 for a NULL handle). */
int64_t sim_debug_schedule_size(const sim_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* EPISIM_H */
