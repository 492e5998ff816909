/*
 * CPU oracle for the general compartment model: any stoichiometry, propensities
 * of a product form, continuous per-node variables, and general scheduled
 * events (Secs. 2.1-2.2, 3.1-3.3 of Bauer, Engblom & Widgren, arXiv:1502.02908).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code with the CUDA
 * library; both are written to the same statement below and must agree bit for
 * bit on counts and continuous variables.
 *
 * Model (Eq. vectorJSDE): Nc compartments per node, Nt transitions with
 * stoichiometric matrix S (Nc x Nt), Ny continuous variables y per node.
 * Transition j fires at rate
 *     a_j = k_j [* y_q] [* x_a] [* x_b] [/ P]          (left to right)
 * where each bracketed factor is present only when the model names it: a
 * continuous variable q, up to two compartments a, b, and a population P = the
 * sum of the counts of a compartment mask (a_j = 0 when P = 0).  This covers
 * the paper's SIR example (Eq. SIRstoich: beta x_S x_I, gamma x_I) and its SISe
 * models (upsilon phi S, gamma I).  A compartment that transition j decrements
 * must be one of its factors, so a rate vanishes before a count turns negative
 * (the requirement stated after Eq. scalarJSDE).
 *
 * Per replicate, per day d (Alg. 1; integer days are the windows of Sec. 4.1):
 *  (i)  stochastic step (Eq. numstep3): per node, the direct method (Sec. 3.3,
 *       Eqs. sampling and sampling2) on [d, d+1) with y frozen.  Step k draws
 *       Philox(node, day, k, replicate); a0 and the thresholds P_j are the
 *       left-to-right partial sums of the rates; the transition fired is the
 *       first j with a_j > 0 and r = a0 u2 <= P_j (the last j with a_j > 0 when
 *       rounding leaves none).  After a firing every rate is recomputed (the
 *       library recomputes only those in the dependency graph; the values
 *       agree because a rate is a function of the counts it reads);
 *  (ii) deterministic step (Eq. numstep4; Sec. 3.2 Eq. event): the day's
 *       events in input order.  An event names a compartment mask ("select")
 *       and optionally a per-compartment offset vector ("shift"):
 *         EXIT      remove n animals drawn uniformly without replacement from
 *                   the masked compartments;
 *         ENTER     add n animals to compartment c0 + off[c0], c0 the lowest
 *                   compartment of the mask;
 *         INTERNAL  move n drawn animals, each from c to c + off[c];
 *         EXTERNAL  move n drawn animals from node to dest, c to c + off[c].
 *       With a one-compartment mask these are the paper's X <- X + E n.
 *       Draws: Lemire's method on the event's Philox word stream; more
 *       animals than present are clamped (or the event is skipped under the
 *       ERROR policy);
 *  (iii) continuous update (Eq. numstep5, Euler with dt = 1), per variable q:
 *         y_q <- ((y_q * (1 - beta_q(d))) + ((alpha_q * U) / D)) + epsilon_q
 *       U, D = sums of the counts of the variable's numerator and denominator
 *       masks (no division when the denominator mask is empty; the middle term
 *       is 0 when D = 0), taken from the post-event counts (Alg. 1 order), the
 *       post-SSA counts (Eq. numstep5 as printed), or the midpoint of the day's
 *       first and last states (Eq. numstep2): U = (U_n + U_{n+1}) / 2 and D the
 *       same, U_n from the counts before the stochastic step.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_rng.h"

#define GO_MAX_COMP 16
#define GO_MAX_TRANS 32
#define GO_MAX_CONT 4
#define GO_MAX_SELECT 32
#define GO_MAX_SHIFT 32

enum { GO_EXIT = 0, GO_ENTER = 1, GO_INTERNAL = 2, GO_EXTERNAL = 3 };
enum { GO_Y_POST_EVENT = 0, GO_Y_PRE_EVENT = 1, GO_Y_MIDPOINT = 2 };

typedef struct {
    int32_t n_comp, n_trans, n_cont, n_select, n_shift, y_source;
    int32_t stoich[GO_MAX_COMP * GO_MAX_TRANS];     /* S[c][j] at c * n_trans + j */
    int32_t fa[GO_MAX_TRANS], fb[GO_MAX_TRANS];     /* compartment factors or -1 */
    int32_t fy[GO_MAX_TRANS];                       /* continuous factor or -1 */
    uint32_t pop[GO_MAX_TRANS];                     /* population mask or 0 */
    uint32_t num[GO_MAX_CONT], den[GO_MAX_CONT];
    uint32_t select[GO_MAX_SELECT];
    int32_t shift[GO_MAX_SHIFT * GO_MAX_COMP];      /* off[s][c] at s * GO_MAX_COMP + c */
} go_model;

typedef struct {
    int32_t n_nodes, replicate, underflow_error, pad;
    uint64_t seed;
    double rate[GO_MAX_TRANS];
    double alpha[GO_MAX_CONT], beta[GO_MAX_CONT][4], epsilon[GO_MAX_CONT];
} go_cfg;

typedef struct {
    int64_t transitions, events_applied, events_clamped, events_skipped;
} go_counters;

/* counts[c * N + v], y[q * N + v] */
#define GX(c, v) counts[(int64_t)(c) * N + (v)]

static int go_season(int32_t day)
{
    int dm = day % 365;
    return dm <= 91 ? 0 : dm <= 182 ? 1 : dm <= 273 ? 2 : 3;
}

static int64_t mask_sum(const int32_t* counts, int32_t N, int32_t v, uint32_t mask, int nc)
{
    int64_t s = 0;
    for (int c = 0; c < nc; ++c)
        if (mask >> c & 1u) s += GX(c, v);
    return s;
}

/* a_j = k_j [* y_q] [* x_a] [* x_b] [/ P], factors left to right. */
static double go_rate(const go_model* m, const go_cfg* g, const int32_t* counts, int32_t N, int32_t v,
                      const double* yv, int j)
{
    double a = g->rate[j];
    if (m->fy[j] >= 0) a = a * yv[m->fy[j]];
    if (m->fa[j] >= 0) a = a * (double)GX(m->fa[j], v);
    if (m->fb[j] >= 0) a = a * (double)GX(m->fb[j], v);
    if (m->pop[j]) {
        int64_t P = mask_sum(counts, N, v, m->pop[j], m->n_comp);
        a = P > 0 ? a / (double)P : 0.0;
    }
    return a;
}

/* Direct method for node v over [day, day + 1) with y frozen; returns the
 * number of transitions fired. */
static int64_t go_node_day(const go_model* m, const go_cfg* g, int32_t* counts, int32_t N, int32_t v,
                           int32_t day, const double* yv)
{
    const int nt = m->n_trans, nc = m->n_comp;
    double a[GO_MAX_TRANS];
    for (int j = 0; j < nt; ++j) a[j] = go_rate(m, g, counts, N, v, yv, j);
    double t = 0.0;
    int64_t fired = 0;
    const uint32_t key[2] = { (uint32_t)g->seed, (uint32_t)(g->seed >> 32) };
    for (uint32_t k = 0;; ++k) {
        double a0 = 0.0;
        for (int j = 0; j < nt; ++j) a0 = a0 + a[j];
        if (!(a0 > 0.0)) break;
        uint32_t ctr[4] = { (uint32_t)v, (uint32_t)day, k, (uint32_t)g->replicate }, w[4];
        orc_philox(ctr, key, w);
        double E = orc_neglog(((((uint64_t)w[1]) << 32) | w[0]) >> 12);
        double u2 = orc_uniform(w[2], w[3]);
        double tau = E / a0;
        if (t + tau >= 1.0) break;
        t = t + tau;
        double r = a0 * u2, P = 0.0;
        int chosen = -1, last = -1;
        for (int j = 0; j < nt; ++j) {
            P = P + a[j];
            if (!(a[j] > 0.0)) continue;
            last = j;
            if (r <= P) { chosen = j; break; }
        }
        if (chosen < 0) chosen = last;
        for (int c = 0; c < nc; ++c) GX(c, v) += m->stoich[c * nt + chosen];
        for (int j = 0; j < nt; ++j) a[j] = go_rate(m, g, counts, N, v, yv, j);
        ++fired;
    }
    return fired;
}

/* Continuous update of variable q of node v (Eq. numstep5 / Eq. numstep2). */
static double go_y_next(const go_model* m, const go_cfg* g, int q, int32_t day, double y, double U, double D)
{
    double omb = 1.0 - g->beta[q][go_season(day)];
    double mid;
    if (m->den[q] == 0) mid = g->alpha[q] * U;
    else mid = D > 0.0 ? (g->alpha[q] * U) / D : 0.0;
    return ((y * omb) + mid) + g->epsilon[q];
}

/* One scheduled event at day-stable position e. */
static void go_apply_event(const go_model* m, const go_cfg* g, int32_t* counts, int32_t N, int64_t e,
                           int32_t day, int32_t kind, int32_t node, int32_t dest, int32_t n,
                           int32_t sel, int32_t sh, go_counters* ctr)
{
    const int nc = m->n_comp;
    const uint32_t mask = m->select[sel];
    int off[GO_MAX_COMP];
    for (int c = 0; c < nc; ++c) off[c] = sh >= 0 ? m->shift[sh * GO_MAX_COMP + c] : 0;
    if (kind == GO_ENTER) {
        int c0 = 0;
        while (!(mask >> c0 & 1u)) ++c0;
        GX(c0 + off[c0], node) += n;
        ctr->events_applied++;
        return;
    }
    int64_t avail = mask_sum(counts, N, node, mask, nc);
    int32_t take = n;
    if ((int64_t)n > avail) {
        if (g->underflow_error) { ctr->events_skipped++; return; }
        take = (int32_t)avail;
        ctr->events_clamped++;
    }
    word_stream ws;
    orc_ws_start(&ws, g->seed, g->replicate, e, day);
    for (int32_t i = 0; i < take; ++i) {
        uint32_t slot = orc_ws_lemire(&ws, (uint32_t)(avail - i));
        int got = -1;
        for (int c = 0; c < nc && got < 0; ++c) {
            if (!(mask >> c & 1u)) continue;
            uint32_t have = (uint32_t)GX(c, node);
            if (slot < have) got = c; else slot -= have;
        }
        GX(got, node) -= 1;
        if (kind == GO_INTERNAL) GX(got + off[got], node) += 1;
        else if (kind == GO_EXTERNAL) GX(got + off[got], dest) += 1;
    }
    ctr->events_applied++;
}

/* Runs one replicate over days [d0, d0 + ndays).  counts [Nc][N] and y [Ny][N]
 * hold the state at the start of day d0 and are overwritten with the state at
 * the start of day d0 + ndays.  Event e of the day-stable order draws from
 * Philox counter word 0 = e.  Returns 0, or -1 on a bad argument. */
int go_run(const go_model* m, const go_cfg* g, int32_t* counts, double* y, int32_t d0, int32_t ndays,
           int64_t n_events, const int32_t* ev_day, const int32_t* ev_kind, const int32_t* ev_node,
           const int32_t* ev_dest, const int32_t* ev_count, const int32_t* ev_select,
           const int32_t* ev_shift, go_counters* ctr)
{
    const int32_t N = g->n_nodes;
    const int ny = m->n_cont;
    if (N < 1 || d0 < 0 || ndays < 0 || m->n_comp < 1 || m->n_comp > GO_MAX_COMP || m->n_trans < 0 ||
        m->n_trans > GO_MAX_TRANS || ny < 0 || ny > GO_MAX_CONT)
        return -1;
    int32_t dmax = d0 + ndays;
    for (int64_t e = 0; e < n_events; ++e) {
        if (ev_day[e] < 0) return -1;
        if (ev_day[e] > dmax) dmax = ev_day[e];
    }
    /* stable order by day, and the first position of each day */
    int64_t* first = (int64_t*)calloc((size_t)dmax + 2, sizeof(int64_t));
    int64_t* order = (int64_t*)malloc((size_t)(n_events > 0 ? n_events : 1) * sizeof(int64_t));
    double* U0 = (double*)malloc((size_t)(ny > 0 ? ny : 1) * N * sizeof(double));
    double* D0 = (double*)malloc((size_t)(ny > 0 ? ny : 1) * N * sizeof(double));
    if (!first || !order || !U0 || !D0) { free(first); free(order); free(U0); free(D0); return -1; }
    for (int64_t e = 0; e < n_events; ++e) first[ev_day[e] + 1]++;
    for (int32_t d = 0; d <= dmax; ++d) first[d + 1] += first[d];
    {
        int64_t* fill = (int64_t*)malloc((size_t)(dmax + 1) * sizeof(int64_t));
        if (!fill) { free(first); free(order); free(U0); free(D0); return -1; }
        memcpy(fill, first, (size_t)(dmax + 1) * sizeof(int64_t));
        for (int64_t e = 0; e < n_events; ++e) order[fill[ev_day[e]]++] = e;
        free(fill);
    }
    go_counters local = {0, 0, 0, 0};
    if (!ctr) ctr = &local;
    double yv[GO_MAX_CONT];

    for (int32_t d = d0; d < d0 + ndays; ++d) {
        if (m->y_source == GO_Y_MIDPOINT)
            for (int q = 0; q < ny; ++q)
                for (int32_t v = 0; v < N; ++v) {
                    U0[(int64_t)q * N + v] = (double)mask_sum(counts, N, v, m->num[q], m->n_comp);
                    D0[(int64_t)q * N + v] = (double)mask_sum(counts, N, v, m->den[q], m->n_comp);
                }
        /* (i) stochastic step */
        for (int32_t v = 0; v < N; ++v) {
            for (int q = 0; q < ny; ++q) yv[q] = y[(int64_t)q * N + v];
            ctr->transitions += go_node_day(m, g, counts, N, v, d, yv);
        }
        /* (iii) as printed in Eq. numstep5: from the post-SSA counts */
        if (m->y_source == GO_Y_PRE_EVENT)
            for (int q = 0; q < ny; ++q)
                for (int32_t v = 0; v < N; ++v) {
                    double U = (double)mask_sum(counts, N, v, m->num[q], m->n_comp);
                    double D = (double)mask_sum(counts, N, v, m->den[q], m->n_comp);
                    y[(int64_t)q * N + v] = go_y_next(m, g, q, d, y[(int64_t)q * N + v], U, D);
                }
        /* (ii) the day's events in input order */
        for (int64_t s = first[d]; s < first[d + 1]; ++s) {
            int64_t e = order[s];
            go_apply_event(m, g, counts, N, s, d, ev_kind[e], ev_node[e], ev_dest[e], ev_count[e],
                           ev_select[e], ev_shift[e], ctr);
        }
        /* (iii) Alg. 1 order (post-event counts) or Eq. numstep2 (midpoint) */
        if (m->y_source != GO_Y_PRE_EVENT)
            for (int q = 0; q < ny; ++q)
                for (int32_t v = 0; v < N; ++v) {
                    double U = (double)mask_sum(counts, N, v, m->num[q], m->n_comp);
                    double D = (double)mask_sum(counts, N, v, m->den[q], m->n_comp);
                    if (m->y_source == GO_Y_MIDPOINT) {
                        U = 0.5 * (U0[(int64_t)q * N + v] + U);
                        D = 0.5 * (D0[(int64_t)q * N + v] + D);
                    }
                    y[(int64_t)q * N + v] = go_y_next(m, g, q, d, y[(int64_t)q * N + v], U, D);
                }
    }
    free(first); free(order); free(U0); free(D0);
    return 0;
}
