/*
 * episim_general.h — C ABI of the general compartment model in libepisim.so,
 * after Bauer, Engblom & Widgren, "Fast event-based epidemiological
 * simulations on national scales" (arXiv:1502.02908).
 *
 * The model of Secs. 2.1-2.2 in general form (Eq. (vectorJSDE)): per node, Nc
 * compartment counts X (int32), Ny continuous variables Y (binary64), Nt
 * transitions with stoichiometric matrix S (Nc x Nt).  One simulated day, for
 * every node and replicate, is
 *   1. the stochastic step (Eq. (numstep3); Sec. 3.3 Eqs. (sampling),
 *      (sampling2)): the direct method on [d, d+1) with Y frozen.  The rate of
 *      transition j is
 *          a_j = k_j [* y_q] [* x_a] [* x_b] [/ P],   evaluated left to right,
 *      each bracketed factor present only when the transition names it (a
 *      continuous variable q, compartments a and b, a population P = the sum of
 *      the counts of a compartment mask; a_j = 0 when P = 0).  a0 and the
 *      selection thresholds are left-to-right partial sums of a_1..a_Nt; the
 *      transition fired is the first j with a_j > 0 and a0 u2 <= P_j (the last
 *      positive one when rounding leaves none).  After a firing only the rates
 *      in its dependency graph (Sec. 3.3) are recomputed;
 *   2. the deterministic step (Eq. (numstep4); Sec. 3.2 Eq. (event)): the
 *      day's events applied with the result of their input order;
 *   3. the continuous update (Eq. (numstep5), Euler with dt = 1) of each
 *      variable q:  y <- ((y (1 - beta_q(d))) + ((alpha_q U) / D)) + epsilon_q,
 *      U, D = sums of the counts of the variable's numerator and denominator
 *      masks (no division when the denominator mask is empty; the middle term
 *      is 0 when D = 0), from the post-event counts, the post-SSA counts, or
 *      the midpoint of the day's first and last states (Eq. (numstep2)).
 *
 * Conventions are those of episim.h: statuses, host/device pointers (SIM_HOST /
 * SIM_DEVICE), ownership (a handle owns what it allocates and copies its
 * inputs), one host thread per handle, counter-based Philox randomness (SSA
 * draw k of node v on day d of replicate r: counter (v, d, k, r); event at
 * day-stable position e: counter (e, d | 2^30, block, r)).  Counts are int32
 * [R][Nc][N], continuous variables double [R][Ny][N].
 */
#ifndef EPISIM_GENERAL_H
#define EPISIM_GENERAL_H

#include <stdint.h>

#include "episim.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { GEN_MAX_COMP = 16, GEN_MAX_TRANS = 32, GEN_MAX_CONT = 4, GEN_MAX_SELECT = 32, GEN_MAX_SHIFT = 32 };

/* Which counts the continuous update reads (step 3 above). */
enum {
    GEN_Y_POST_EVENT = 0,   /* after the day's events (Alg. 1 order) */
    GEN_Y_PRE_EVENT = 1,    /* after the stochastic step, before the events (Eq. (numstep5) as printed) */
    GEN_Y_MIDPOINT = 2      /* (X_n + X_{n+1}) / 2: X_n before the stochastic step, X_{n+1} after the
                               events (Eq. (numstep2)); U = (U_n + U_{n+1}) / 2, D likewise */
};

/* Propensity of one transition: a_j = k_j [* y_cont] [* x_factor_a] [* x_factor_b] [/ P(pop_mask)].
 * factor_a, factor_b: compartment index or -1; cont: continuous variable or -1;
 * pop_mask: bit c set = compartment c in the population (0: no division). */
typedef struct gen_transition {
    int32_t factor_a;
    int32_t factor_b;
    int32_t cont;
    uint32_t pop_mask;
} gen_transition;

/* Continuous variable q: compartment masks of U (numerator) and D (denominator; 0: none). */
typedef struct gen_variable {
    uint32_t num_mask;
    uint32_t den_mask;
} gen_variable;

/* The model, host arrays (copied by gen_create).
 *   stoich [n_comp][n_trans]: S[c][j] in [-1, 127]; a -1 entry only for a compartment
 *       that is factor_a or factor_b of the transition (its rate then vanishes with
 *       the count, so counts never turn negative);
 *   trans [n_trans], vars [n_cont];
 *   select [n_select]: nonzero compartment masks events sample from;
 *   shift [n_shift][n_comp]: per-compartment offsets events move animals by
 *       (compartment c -> c + shift[s][c]).
 * Limits: 1 <= n_comp <= 16, 0 <= n_trans <= 32, 0 <= n_cont <= 4, n_select and
 * n_shift <= 32. */
typedef struct gen_model {
    int32_t n_comp;
    int32_t n_trans;
    int32_t n_cont;
    int32_t n_select;
    int32_t n_shift;
    int32_t y_source;              /* GEN_Y_* */
    const int32_t* stoich;
    const gen_transition* trans;
    const gen_variable* vars;
    const uint32_t* select;
    const int32_t* shift;
} gen_model;

typedef struct gen_config {
    int32_t n_nodes;           /* N >= 1 */
    int32_t n_replicates;      /* R >= 1 */
    int32_t max_days;          /* horizon; days [0, max_days) can be simulated */
    int32_t underflow_policy;  /* SIM_UNDERFLOW_CLAMP or SIM_UNDERFLOW_ERROR */
    uint64_t seed;             /* Philox key */
    int32_t replicate_base;    /* replicate r draws as replicate_base + r */
    int32_t reserved;          /* must be 0 */
} gen_config;

typedef struct gen_handle gen_handle;

/* Validates a model and writes its dependency graph (Sec. 3.3): dep[n] (host,
 * n_trans words) has bit j set when firing transition n can change rate j, i.e.
 * S[.][n] changes factor_a or factor_b of j, or changes the sum of j's
 * population mask.  Host only: needs no device.  dep may be NULL. */
sim_status gen_model_check(const gen_model* m, uint32_t* dep);

/* Creates a simulation at day 0 on the current device.
 *   u0: host int32 [n_comp][N] initial counts (>= 0, at most 2^30 animals a node),
 *       the same for every replicate;
 *   y0: host double [n_cont][N] initial continuous variables (finite, >= 0);
 *   rates: host double [R][n_trans] rate constants k_j (finite, >= 0);
 *   var_params: host double [R][n_cont][6] = {alpha, beta[4], epsilon} per
 *       variable (alpha, epsilon finite >= 0; beta in [0, 1]; beta bin by day of
 *       year [0,91], (91,182], (182,273], (273,364]).
 * *out is set only on SIM_OK; the creation error text is gen_last_error(NULL). */
sim_status gen_create(const gen_model* m, const gen_config* cfg, const int32_t* u0, const double* y0,
                      const double* rates, const double* var_params, gen_handle** out);

/* Loads the scheduled events (Sec. 3.2 Eq. (event)), n host int32 arrays in
 * input order: day >= 0 (events on days >= max_days are kept but never reached);
 * kind SIM_EXIT / SIM_ENTER / SIM_INTERNAL /
 * SIM_EXTERNAL; node (and dest for SIM_EXTERNAL, != node) in [0, N); count >= 0;
 * select in [0, n_select); shift in [-1, n_shift) (-1: no offset).
 *   EXIT      removes count animals drawn uniformly without replacement from the
 *             compartments of select (ascending compartment order for the draw);
 *   ENTER     adds count animals to c0 + off[c0], c0 the lowest compartment of select;
 *   INTERNAL  moves count drawn animals within the node, c -> c + off[c];
 *   EXTERNAL  moves count drawn animals from node to dest, c -> c + off[c].
 * Every c + off[c] of the select mask must be a compartment, and for INTERNAL
 * none may lie in the mask (a moved animal is not drawn again).  More animals than
 * present: clamped and counted (CLAMP) or the event skipped, counted and
 * SIM_E_UNDERFLOW latched (ERROR).  Replaces earlier events; the handle keeps
 * per-day components of the transfer graph (events sharing a node), each applied
 * in input order by one device thread. */
sim_status gen_load_events(gen_handle* h, int64_t n, const int32_t* day, const int32_t* kind,
                           const int32_t* node, const int32_t* dest, const int32_t* count,
                           const int32_t* select, const int32_t* shift);

/* Simulates days [day, day + ndays) on stream (NULL: the legacy default stream),
 * asynchronously. */
sim_status gen_run_days(gen_handle* h, int32_t ndays, void* stream);

/* Copies the state out (counts [R][Nc][N], y [R][Ny][N]; either may be NULL)
 * after synchronising the stream; returns a latched SIM_E_UNDERFLOW. */
sim_status gen_state(gen_handle* h, int32_t* counts, double* y, int32_t* day, int32_t where, void* stream);

/* Replaces the state and the current day (counters are kept). */
sim_status gen_set_state(gen_handle* h, const int32_t* counts, const double* y, int32_t day, int32_t where,
                         void* stream);

/* Host int64 [R][4]: transitions fired, events applied, clamped, skipped. */
sim_status gen_counters(gen_handle* h, int64_t* counters);

/* Options (results never depend on them):
 *   GEN_OPT_LAUNCH: launch mode of gen_run_days, 0 stream launches, 1 the day loop
 *       as a CUDA graph (captured once per (first day, ndays));
 *   GEN_OPT_WARP_THRESHOLD: nodes whose initial population (sum of u0) is at least
 *       this run the stochastic step one per warp, 32 draws at a time with a
 *       fixed-point iteration over the lanes (-1: automatic, 600);
 *   GEN_OPT_GROUP_THRESHOLD: nodes below the warp threshold whose initial
 *       population is at least this run four per warp, 8 lanes and 8 draws at a
 *       time each (-1: automatic, 150); the rest one per thread;
 *   GEN_OPT_CLOCK_MARGIN: k in [0, 16].  Every node-day (one per thread, per
 *       warp or per 8-lane segment) first runs with binary32 rates and partial
 *       sums and a binary32 clock accumulated in fixed point, whose distance to
 *       the binary64 clock of Eq. (numstep3) is bounded below 2^-16 of a day
 *       (product-form rates of at most 32 transitions, constants and continuous
 *       variables within [2^-30, 2^30], populations below 2^21; other node-days
 *       run exactly); a selection is taken in binary32 only when decisive (Eq.
 *       (sampling2), else binary64), and a stop/continue decision within 2^-k of
 *       the day's end reruns the node-day with the binary64 arithmetic.  k = 16
 *       (default) is the tightest safe margin; smaller k only reruns more
 *       node-days; 0 runs every node-day exactly. */
enum { GEN_OPT_LAUNCH = 1, GEN_OPT_WARP_THRESHOLD = 2, GEN_OPT_GROUP_THRESHOLD = 3, GEN_OPT_CLOCK_MARGIN = 4 };
sim_status gen_set_option(gen_handle* h, int32_t option, int64_t value);

/* Nodes the stochastic step runs one per warp, and four per warp (-1 for a NULL handle). */
int32_t gen_warp_nodes(const gen_handle* h);
int32_t gen_group_nodes(const gen_handle* h);

void gen_destroy(gen_handle* h);

/* Text of the handle's last error (NULL: the calling thread's last gen_create error). */
const char* gen_last_error(const gen_handle* h);

#ifdef __cplusplus
}
#endif

#endif
