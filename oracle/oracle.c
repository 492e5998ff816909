/*
 * CPU oracle for the event-based SISe / SISe3 metapopulation simulation of
 * Bauer, Engblom & Widgren, "Fast event-based epidemiological simulations on
 * national scales" (arXiv:1502.02908).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the simulation computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant generator with the CUDA library; the two are
 * written independently to the same arithmetic specification and must agree
 * bit for bit on counts.
 *
 * Per replicate, per day d (Alg. 1 of the paper, integer days as the
 * synchronisation windows of Sec. 4.1):
 *   (i)   stochastic step, Eq. numstep3: Gillespie's direct method in every node
 *         on [d, d+1) with the environmental state phi frozen at phi_d
 *         (Sec. 3.3, Eqs. sampling and sampling2);
 *   (ii)  deterministic step, Eq. numstep4: the day's scheduled events in input
 *         order (the list processor of Sec. 3.3; event records Eq. event);
 *   (iii) continuous-state update, Eq. numstep5 with the VTEC model of
 *         Eq. siminfpressure: phi <- phi*(1-beta) + alpha*I/N + epsilon, from the
 *         post-event counts (Alg. 1 order) or, on request, from the post-SSA
 *         counts (Eq. numstep5 as printed).
 *
 * Readings where the paper is silent (all fixed here and in the CUDA library):
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), counter-based,
 *     keyed by (replicate, node, day, draw index);
 *   - -log(rand) of Eq. sampling: an exact 64-bit fixed-point logarithm,
 *     rounded once to double (neglog_u below);
 *   - each day restarts the direct method (no Gibson-Bruck rescaling; exact in
 *     distribution by memorylessness);
 *   - events that remove more animals than present are clamped (or skipped under
 *     the ERROR policy); removed animals are sampled without replacement,
 *     uniformly, with Lemire's bounded-integer method.
 *
 * Compartments inside a node are class-major: SISe [S, I]; SISe3
 * [S1, I1, S2, I2, S3, I3].  Counts are int32, phi is IEEE binary64.
 *
 * Pinned by tests/test_oracle_*.py against closed forms, a matrix-exponential
 * law, invariants, published Philox answers and high-precision logarithms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include "oracle_rng.h"

#define ORC_SISE  1
#define ORC_SISE3 3

enum { EV_EXIT = 0, EV_ENTER = 1, EV_INTERNAL = 2, EV_EXTERNAL = 3 };

typedef struct {
    int32_t model;            /* ORC_SISE or ORC_SISE3 */
    int32_t n_nodes;
    int32_t replicate;        /* Philox counter word 3 */
    int32_t phi_pre_event;    /* 1: phi update from post-SSA, pre-event counts */
    int32_t underflow_error;  /* 1: skip events asking for more animals than present */
    int32_t score;            /* 1: accumulate score-function terms */
    uint64_t seed;            /* Philox key */
    double upsilon[3], gamma[3], alpha, beta[4], epsilon;
} orc_cfg;

typedef struct {
    int64_t transitions;      /* SSA transitions fired */
    int64_t events_applied;
    int64_t events_clamped;
    int64_t events_skipped;   /* ERROR policy */
} orc_counters;

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10: ten rounds of two 32x32->64 multiplies by fixed odd constants,
 * the high halves xored into the other words with the round key; the key is
 * bumped by the Weyl constants between rounds. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(pb >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)pb;
        uint32_t y2 = (uint32_t)(pa >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)pa;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

#define TAG_EVENTS 0x40000000u

static void ssa_block(const orc_cfg* c, int32_t node, int32_t day, uint32_t k, uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)node, (uint32_t)day, k, (uint32_t)c->replicate };
    uint32_t key[2] = { (uint32_t)c->seed, (uint32_t)(c->seed >> 32) };
    orc_philox(ctr, key, out);
}

/* Uniform on (0,1): the top 52 bits of a 64-bit word j give (2j+1) * 2^-53,
 * exact in binary64, never 0 or 1. */
double orc_uniform(uint32_t lo, uint32_t hi)
{
    uint64_t w = ((uint64_t)hi << 32) | lo;
    uint64_t j = w >> 12;
    return ldexp((double)(2 * j + 1), -53);
}

/* ------------------------------------------------------ -log(rand), fixed point */
/* R_i ~ 1024 / (1 + (2i+1)/256), the reciprocal of the centre of the i-th of 128
 * sub-intervals of [1, 2), rounded to an integer. */
static int64_t recip_tab(int i) { return (2 * 262144 + (257 + 2 * i)) / (2 * (257 + 2 * i)); }

/* ln(1024 / R_i), rounded to the nearest multiple of 2^-62 (values checked
 * against 300-bit arithmetic by the tests). */
static const int64_t LOGR_Q62[128] = {
  18049674776816854LL, 54362350727533905LL, 90963225532746762LL, 123229026447887969LL,
  160382790494758706LL, 193139703589494237LL, 226130955305116292LL, 264126523630095849LL,
  297631395580117410LL, 331381470028421725LL, 365380362437126994LL, 394723108417991391LL,
  429193959917810211LL, 463924411452969488LL, 493902974344939256LL, 529126061154515086LL,
  559532892311828680LL, 590141540197043218LL, 620954701722837312LL, 651975128224706936LL,
  683205626935200460LL, 714649062508412851LL, 746308358596809263LL, 778186499482548415LL,
  810286531765581918LL, 837208301265004118LL, 869723261000343774LL, 896995286182190935LL,
  924429549231742015LL, 957567555422974392LL, 985365626440019268LL, 1013332273811741246LL,
  1041469554620679147LL, 1069779563833499675LL, 1098264435237000457LL, 1126926342403200110LL,
  1155767499684606819LL, 1184790163240804979LL, 1213996632097549965LL, 1237495719979465513LL,
  1267038972958407263LL, 1296772705995433815LL, 1320698497759364959LL, 1350781357324981151LL,
  1374989738470859697LL, 1405430020730302915LL, 1429927746429893232LL, 1454556301725417873LL,
  1479317091508514926LL, 1510456210616749994LL, 1535519783278192789LL, 1560720316032852194LL,
  1586059313947995113LL, 1611538307037006498LL, 1637158850813754575LL, 1662922526862441371LL,
  1688830943423460540LL, 1708358224618079992LL, 1734523889241776865LL, 1760838859464412799LL,
  1787304848994123195LL, 1807254495180523925LL, 1833988981752507855LL, 1860879355424357132LL,
  1881150535397005931LL, 1908318131011264558LL, 1928799375712087812LL, 1956249968776523276LL,
  1976945677488765434LL, 1997734680469895947LL, 2025599937565400464LL, 2046609932986349629LL,
  2067716084327662311LL, 2096008725327687286LL, 2117342700236523210LL, 2138775826430563773LL,
  2160309029841231178LL, 2181943249431133721LL, 2203679437439746334LL, 2225518559634908415LL,
  2247461595570305017LL, 2269509538849103040LL, 2291663397393919824LL, 2313924193723307555LL,
  2336292965234943107LL, 2358770764495719430LL, 2381358659538941293LL, 2404057734168835207LL,
  2426869088272590598LL, 2442139585730020712LL, 2465140561182805815LL, 2488256830227227503LL,
  2511489554518897900LL, 2527043316373605573LL, 2550472762289454357LL, 2574021848447748151LL,
  2589788311730827704LL, 2613539536857544955LL, 2629441918195754679LL, 2653398782556185840LL,
  2669439445748877075LL, 2693605541319148873LL, 2709786912371171034LL, 2734165926070383412LL,
  2750490495394059822LL, 2775086212460075418LL, 2791556537175482246LL, 2808085895438980183LL,
  2832991551030960732LL, 2849670361321007686LL, 2866409711889995949LL, 2891633216985898728LL,
  2908525858652257796LL, 2925480605758512052LL, 2942497916648945873LL, 2968142205259571451LL,
  2985317964474498786LL, 3002557932284363737LL, 3019862590556484214LL, 3037232426603032179LL,
  3063410468617982509LL, 3080945417570454822LL, 3098547293971195362LL, 3116216610676088831LL,
  3133953886458616845LL, 3151759646101249955LL, 3169634420488610844LL, 3187578746702450052LL,
};
/* ln 2 rounded to the nearest multiple of 2^-62 */
static const uint64_t LN2_Q62 = 3196577161300663915ULL;

static int64_t mulq62(int64_t a, int64_t b)
{
    __int128 p = (__int128)a * (__int128)b;
    return (int64_t)(p >> 62);             /* arithmetic shift: floor */
}

/* E = -ln(u) for u = (2j+1) 2^-53, j < 2^52.  x = 2j+1 = 2^n * m with m in [1,2):
 *   E = (53 - n) ln 2 - ln m,
 *   ln m = ln(y) + ln(1024/R_i),  y = m R_i / 1024 = 1 + z, |z| < 2^-7.8,
 *   ln(1+z) = z - z^2/2 + ... + z^7/7 (Horner, Q62, truncating products).
 * (53 - n) ln 2 - ln m is formed in Q62 (128-bit), floored to Q58 and rounded
 * once to binary64.  The Q58 value is within 2^-56 of -ln(u). */
uint64_t orc_neglog_q58(uint64_t j)
{
    uint64_t x = 2 * j + 1;
    int n = 63 - __builtin_clzll(x);
    uint64_t M = x << (52 - n);                  /* [2^52, 2^53) */
    int i = (int)((M >> 45) & 127);
    int64_t z = (int64_t)(M * (uint64_t)recip_tab(i)) - ((int64_t)1 << 62);
    int64_t h = ((int64_t)1 << 62) / 7;
    for (int k = 6; k >= 1; --k) {
        int64_t ck = (((int64_t)1 << 62) + k / 2) / k;   /* round(2^62 / k) */
        h = ck - mulq62(z, h);
    }
    int64_t lnm = mulq62(z, h) + LOGR_Q62[i];      /* ln m in Q62 */
    __int128 e62 = (__int128)(53 - n) * (__int128)LN2_Q62 - (__int128)lnm;   /* E in Q62 */
    __int128 e = e62 >> 4;                       /* Q58, floor */
    if (e < 1) e = 1;                            /* E is at least 2^-58 */
    return (uint64_t)e;                          /* E * 2^58 < 2^64 */
}

double orc_neglog(uint64_t j)
{
    return ldexp((double)orc_neglog_q58(j), -58);
}

/* ------------------------------------------------------------ events RNG */

static void ws_init(word_stream* s, const orc_cfg* c, int64_t ev_index, int32_t day)
{
    s->key[0] = (uint32_t)c->seed; s->key[1] = (uint32_t)(c->seed >> 32);
    s->ctr[0] = (uint32_t)ev_index; s->ctr[1] = (uint32_t)day | TAG_EVENTS;
    s->ctr[2] = 0; s->ctr[3] = (uint32_t)c->replicate;
    s->q = 0;
}

static uint32_t ws_next(word_stream* s)
{
    if ((s->q & 3) == 0) { s->ctr[2] = s->q >> 2; orc_philox(s->ctr, s->key, s->buf); }
    return s->buf[s->q++ & 3];
}

/* Uniform integer in [0, s), s >= 1 (Lemire 2019, multiply-shift with rejection). */
static uint32_t lemire(word_stream* ws, uint32_t s)
{
    uint64_t m = (uint64_t)ws_next(ws) * s;
    uint32_t l = (uint32_t)m;
    if (l < s) {
        uint32_t t = (uint32_t)(-s) % s;
        while (l < t) { m = (uint64_t)ws_next(ws) * s; l = (uint32_t)m; }
    }
    return (uint32_t)(m >> 32);
}

void orc_ws_start(word_stream* s, uint64_t seed, int32_t replicate, int64_t ev_index, int32_t day)
{
    orc_cfg c; memset(&c, 0, sizeof c);
    c.seed = seed; c.replicate = replicate;
    ws_init(s, &c, ev_index, day);
}

uint32_t orc_ws_lemire(word_stream* s, uint32_t bound) { return lemire(s, bound); }

/* ---------------------------------------------------------------- model */
static int n_age(const orc_cfg* c) { return c->model == ORC_SISE3 ? 3 : 1; }

static int season(int32_t day)
{
    int dm = day % 365;
    return dm <= 91 ? 0 : dm <= 182 ? 1 : dm <= 273 ? 2 : 3;
}

/* counts[c * N + v], score[k * N + v] */
#define X(c, v) counts[(int64_t)(c) * N + (v)]
#define SC(k, v) score[(int64_t)(k) * N + (v)]

typedef struct {
    double n_inf[3], n_rec[3];     /* fired transitions of the node-day */
    double int_s[3], int_i[3];     /* time integrals of S_j, I_j over the day */
} day_terms;

/* Direct method for one node over [day, day+1) with frozen phi (Eqs. numstep3,
 * sampling, sampling2).  Rates, fixed order per class j:
 *   a_inf_j = (upsilon_j * phi) * S_j,  a_rec_j = gamma_j * I_j,
 *   A_j = a_inf_j + a_rec_j,  a0 = A_1 (SISe) or (A_1 + A_2) + A_3 (SISe3).
 * Step k: (u1, u2) from Philox(node, day, k, replicate);
 *   tau = E(u1) / a0;  stop if t + tau >= 1;  otherwise t = t + tau and the
 *   transition is the first one, in the order inf_1, rec_1, inf_2, ..., whose
 *   cumulative threshold reaches r = a0 * u2, where the thresholds are
 *   P_{j-1} + a_inf_j (inf_j) and P_j (rec_j), P_j = A_1 + ... + A_j summed
 *   left to right (P_0 = 0, so the first inf threshold is a_inf_1).  Classes
 *   and transitions with zero rate are never chosen. */
static int64_t ssa_node_day(const orc_cfg* c, int32_t* counts, int32_t N, int32_t v,
                            int32_t day, double phi, day_terms* terms)
{
    int na = n_age(c);
    double cinf[3], ainf[3], arec[3], A[3];
    double tlast[3];
    for (int j = 0; j < na; ++j) {
        cinf[j] = c->upsilon[j] * phi;
        ainf[j] = cinf[j] * (double)X(2 * j, v);
        arec[j] = c->gamma[j] * (double)X(2 * j + 1, v);
        A[j] = ainf[j] + arec[j];
        tlast[j] = 0.0;
        if (terms) { terms->n_inf[j] = terms->n_rec[j] = terms->int_s[j] = terms->int_i[j] = 0.0; }
    }
    double t = 0.0;
    int64_t fired = 0;
    for (uint32_t k = 0;; ++k) {
        double P[3];
        P[0] = A[0];
        for (int j = 1; j < na; ++j) P[j] = P[j - 1] + A[j];
        double a0 = P[na - 1];
        if (!(a0 > 0.0)) break;
        uint32_t w[4];
        ssa_block(c, v, day, k, w);
        uint64_t j1 = ((((uint64_t)w[1]) << 32) | w[0]) >> 12;
        double E = orc_neglog(j1);
        double u2 = orc_uniform(w[2], w[3]);
        double tau = E / a0;
        double tn = t + tau;
        if (tn >= 1.0) break;
        t = tn;
        double r = a0 * u2;
        /* class: first j with A_j > 0 and r <= P_j (the last positive class otherwise) */
        int cls = -1, last = -1;
        for (int j = 0; j < na; ++j) {
            if (!(A[j] > 0.0)) continue;
            last = j;
            if (r <= P[j]) { cls = j; break; }
        }
        if (cls < 0) cls = last;
        double thr = (cls == 0) ? ainf[0] : P[cls - 1] + ainf[cls];
        int infect = (ainf[cls] > 0.0) && (r <= thr || !(arec[cls] > 0.0));
        if (terms) {
            double dt = t - tlast[cls];
            terms->int_s[cls] += (double)X(2 * cls, v) * dt;
            terms->int_i[cls] += (double)X(2 * cls + 1, v) * dt;
            tlast[cls] = t;
            if (infect) terms->n_inf[cls] += 1.0; else terms->n_rec[cls] += 1.0;
        }
        if (infect) { X(2 * cls, v) -= 1; X(2 * cls + 1, v) += 1; }
        else        { X(2 * cls + 1, v) -= 1; X(2 * cls, v) += 1; }
        ainf[cls] = cinf[cls] * (double)X(2 * cls, v);
        arec[cls] = c->gamma[cls] * (double)X(2 * cls + 1, v);
        A[cls] = ainf[cls] + arec[cls];
        ++fired;
    }
    if (terms) {
        for (int j = 0; j < na; ++j) {
            double dt = 1.0 - tlast[j];
            terms->int_s[j] += (double)X(2 * j, v) * dt;
            terms->int_i[j] += (double)X(2 * j + 1, v) * dt;
        }
    }
    return fired;
}

/* Environmental update, Eq. numstep5 with Eq. siminfpressure and Delta t = 1:
 *   phi <- ((phi * (1 - beta(day))) + ((alpha * I) / N)) + epsilon,
 * I = sum_j I_j, N = sum_j (S_j + I_j); the middle term is 0 when N = 0. */
static double phi_next(const orc_cfg* c, const int32_t* counts, int32_t N, int32_t v,
                       int32_t day, double phi, double* i_over_n)
{
    int na = n_age(c);
    int64_t I = 0, tot = 0;
    for (int j = 0; j < na; ++j) { I += X(2 * j + 1, v); tot += X(2 * j, v) + X(2 * j + 1, v); }
    double omb = 1.0 - c->beta[season(day)];
    double q = (tot > 0) ? (c->alpha * (double)I) / (double)tot : 0.0;
    if (i_over_n) *i_over_n = (tot > 0) ? (double)I / (double)tot : 0.0;
    return ((phi * omb) + q) + c->epsilon;
}

/* Draws one animal without replacement, uniformly, from the listed
 * compartments of node v (in list order) and removes it; returns its compartment. */
static int take_one(int32_t* counts, int32_t N, int32_t v, const int* comp, int ncomp,
                    uint32_t avail, word_stream* ws)
{
    uint32_t slot = lemire(ws, avail);
    for (int q = 0; q < ncomp; ++q) {
        uint32_t have = (uint32_t)X(comp[q], v);
        if (slot < have) { X(comp[q], v) -= 1; return comp[q]; }
        slot -= have;
    }
    return -1;  /* unreachable when avail is the sum of the listed counts */
}

/* Applies one scheduled event (Eq. event; VTEC event kinds of Sec. 4.1). */
static void apply_event(const orc_cfg* c, int32_t* counts, int32_t N, int64_t e, int32_t day,
                        int32_t kind, int32_t node, int32_t dest, int32_t n, int32_t cls,
                        orc_counters* ctr)
{
    int na = n_age(c);
    if (kind == EV_ENTER) {
        int j = cls < 0 ? 0 : cls;
        X(2 * j, node) += n;
        ctr->events_applied++;
        return;
    }
    int comp[6], ncomp = 0;
    if (cls < 0) { for (int q = 0; q < 2 * na; ++q) comp[ncomp++] = q; }
    else { comp[ncomp++] = 2 * cls; comp[ncomp++] = 2 * cls + 1; }
    int64_t avail = 0;
    for (int q = 0; q < ncomp; ++q) avail += X(comp[q], node);
    int32_t take = n;
    if ((int64_t)n > avail) {
        if (c->underflow_error) { ctr->events_skipped++; return; }
        take = (int32_t)avail;
        ctr->events_clamped++;
    }
    word_stream ws;
    ws_init(&ws, c, e, day);
    for (int32_t a = 0; a < take; ++a) {
        int got = take_one(counts, N, node, comp, ncomp, (uint32_t)(avail - a), &ws);
        if (kind == EV_INTERNAL) X(got + 2, node) += 1;        /* same state, next class */
        else if (kind == EV_EXTERNAL) X(got, dest) += 1;
    }
    ctr->events_applied++;
}

/* Stable counting sort of event indices by day. */
static int64_t* sort_by_day(int64_t n, const int32_t* day, int32_t dmax)
{
    int64_t* cnt = (int64_t*)calloc((size_t)dmax + 2, sizeof(int64_t));
    int64_t* order = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!cnt || !order) { free(cnt); free(order); return NULL; }
    for (int64_t e = 0; e < n; ++e) cnt[day[e] + 1]++;
    for (int32_t d = 0; d <= dmax; ++d) cnt[d + 1] += cnt[d];
    for (int64_t e = 0; e < n; ++e) order[cnt[day[e]]++] = e;
    free(cnt);
    return order;
}

/* Runs one replicate over days [d0, d0+ndays).  counts [Nc][N] and phi [N] hold
 * the state at the start of day d0 (phi = phi_d0) and are overwritten with the
 * state at the start of day d0+ndays.  Events are given in input order; event
 * e of the day-stable order uses Philox counter word 0 = e.
 * prev_i / prev_n (optional, [ndays]): infected and total animals after the
 * events of each day.  score (optional, [8][N]): per-node accumulated
 * score-function terms d log p(path) / d theta for theta =
 * [upsilon_1..3, gamma_1..3, beta, alpha] (the trajectory's score is their sum
 * over nodes); tangents ([2][N], required with score) carry d phi / d beta and
 * d phi / d alpha across calls.  The likelihood of a path is the product of the
 * rates of the fired transitions times exp(-integral of a0), from Eqs. sampling
 * and sampling2; beta enters through phi only (a common shift of the four
 * seasonal values), as does alpha. 
 * Returns 0, or -1 on a bad argument / allocation failure. */
int orc_run(const orc_cfg* c, int32_t* counts, double* phi, int32_t d0, int32_t ndays,
            int64_t n_events, const int32_t* ev_day, const int32_t* ev_kind,
            const int32_t* ev_node, const int32_t* ev_dest, const int32_t* ev_count,
            const int32_t* ev_cls, int64_t* prev_i, int64_t* prev_n, orc_counters* ctr,
            double* score, double* tangents)
{
    const int32_t N = c->n_nodes;
    const int na = n_age(c);
    if (N < 0 || ndays < 0 || d0 < 0 || (c->model != ORC_SISE && c->model != ORC_SISE3)) return -1;
    if (c->score && (!score || !tangents)) return -1;
    int32_t dmax = d0 + ndays;
    for (int64_t e = 0; e < n_events; ++e) {
        if (ev_day[e] < 0) return -1;
        if (ev_day[e] > dmax) dmax = ev_day[e];
    }
    int64_t* order = sort_by_day(n_events, ev_day, dmax);
    if (!order) return -1;
    /* first sorted position of each day */
    int64_t* first = (int64_t*)calloc((size_t)dmax + 2, sizeof(int64_t));
    double* phi_tmp = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    double* q_tmp = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    day_terms* terms = c->score ? (day_terms*)malloc((size_t)(N > 0 ? N : 1) * sizeof(day_terms)) : NULL;
    if (!first || !phi_tmp || !q_tmp || (c->score && !terms)) {
        free(order); free(first); free(phi_tmp); free(q_tmp); free(terms); return -1;
    }
    for (int64_t s = 0; s < n_events; ++s) first[ev_day[order[s]] + 1]++;
    for (int32_t d = 0; d <= dmax; ++d) first[d + 1] += first[d];

    orc_counters local = {0, 0, 0, 0};
    if (!ctr) ctr = &local;
    double* dphi_b = tangents;
    double* dphi_a = tangents ? tangents + N : NULL;

    for (int32_t d = d0; d < d0 + ndays; ++d) {
        /* (i) stochastic step in every node */
        for (int32_t v = 0; v < N; ++v) {
            ctr->transitions += ssa_node_day(c, counts, N, v, d, phi[v], terms ? &terms[v] : NULL);
            if (terms) {
                day_terms* T = &terms[v];
                double ups_int = 0.0;
                for (int j = 0; j < na; ++j) {
                    SC(j, v) += (c->upsilon[j] > 0.0 ? T->n_inf[j] / c->upsilon[j] : 0.0) - phi[v] * T->int_s[j];
                    SC(3 + j, v) += (c->gamma[j] > 0.0 ? T->n_rec[j] / c->gamma[j] : 0.0) - T->int_i[j];
                    ups_int += c->upsilon[j] * T->int_s[j];
                }
                double ninf = 0.0;
                for (int j = 0; j < na; ++j) ninf += T->n_inf[j];
                /* d log p / d phi_d for this node-day */
                double cd = (phi[v] > 0.0 ? ninf / phi[v] : 0.0) - ups_int;
                if (dphi_b) { SC(6, v) += cd * dphi_b[v]; SC(7, v) += cd * dphi_a[v]; }
            }
        }
        /* (iii, Eq. numstep5 as printed) phi from the post-SSA counts */
        if (c->phi_pre_event)
            for (int32_t v = 0; v < N; ++v) phi_tmp[v] = phi_next(c, counts, N, v, d, phi[v], &q_tmp[v]);
        /* (ii) deterministic step: the day's events in input order */
        for (int64_t s = first[d]; s < first[d + 1]; ++s) {
            int64_t e = order[s];
            apply_event(c, counts, N, s, d, ev_kind[e], ev_node[e], ev_dest[e], ev_count[e], ev_cls[e], ctr);
        }
        /* (iii, Alg. 1 order) phi from the post-event counts */
        if (!c->phi_pre_event)
            for (int32_t v = 0; v < N; ++v) phi_tmp[v] = phi_next(c, counts, N, v, d, phi[v], &q_tmp[v]);
        for (int32_t v = 0; v < N; ++v) {
            if (dphi_b) {
                double omb = 1.0 - c->beta[season(d)];
                dphi_b[v] = dphi_b[v] * omb - phi[v];
                dphi_a[v] = dphi_a[v] * omb + q_tmp[v];
            }
            phi[v] = phi_tmp[v];
        }
        if (prev_i) {
            int64_t I = 0, tot = 0;
            for (int32_t v = 0; v < N; ++v)
                for (int j = 0; j < na; ++j) { I += X(2 * j + 1, v); tot += X(2 * j, v) + X(2 * j + 1, v); }
            prev_i[d - d0] = I;
            if (prev_n) prev_n[d - d0] = tot;
        }
    }
    free(order); free(first); free(phi_tmp); free(q_tmp); free(terms);
    return 0;
}

/* Test hooks: the tables and constants above, for comparison with
 * high-precision arithmetic. */
int64_t orc_logr_q62(int i) { return (i >= 0 && i < 128) ? LOGR_Q62[i] : 0; }
int64_t orc_recip(int i) { return (i >= 0 && i < 128) ? recip_tab(i) : 0; }
uint64_t orc_ln2_q62(void) { return LN2_Q62; }
uint32_t orc_lemire_draw(uint64_t seed, int32_t replicate, int64_t ev_index, int32_t day,
                         uint32_t s, uint32_t nth)
{
    orc_cfg c; memset(&c, 0, sizeof c);
    c.seed = seed; c.replicate = replicate;
    word_stream ws; ws_init(&ws, &c, ev_index, day);
    uint32_t r = 0;
    for (uint32_t i = 0; i <= nth; ++i) r = lemire(&ws, s);
    return r;
}

/* Applies n scheduled events in the listed order (no stochastic step, no phi
 * update); event k uses Philox counter word 0 = pos[k] and day day[k].  Used to
 * check that an execution schedule reproduces the input order. */
int orc_apply_events(const orc_cfg* c, int32_t* counts, int64_t n, const int64_t* pos,
                     const int32_t* day, const int32_t* kind, const int32_t* node,
                     const int32_t* dest, const int32_t* count, const int32_t* cls,
                     orc_counters* ctr)
{
    const int32_t N = c->n_nodes;
    orc_counters local = {0, 0, 0, 0};
    if (!ctr) ctr = &local;
    for (int64_t k = 0; k < n; ++k)
        apply_event(c, counts, N, pos[k], day[k], kind[k], node[k], dest[k], count[k], cls[k], ctr);
    return 0;
}

/* The steps of one day of orc_run, separately and over a node range: the
 * stochastic step (Eq. numstep3) of nodes [v0, v1) on day `day` with their
 * frozen phi, and the continuous-state update (Eq. numstep5) of nodes [v0, v1)
 * from the current counts.  orc_run is these two around the day's events
 * (orc_apply_events) for every node; the split is used to check a trajectory whose
 * nodes are divided among several workers.  No score terms. */
int orc_ssa_nodes(const orc_cfg* c, int32_t* counts, const double* phi, int32_t day, int32_t v0,
                  int32_t v1, orc_counters* ctr)
{
    const int32_t N = c->n_nodes;
    if (v0 < 0 || v1 < v0 || v1 > N || day < 0 || c->score) return -1;
    orc_counters local = {0, 0, 0, 0};
    if (!ctr) ctr = &local;
    for (int32_t v = v0; v < v1; ++v) ctr->transitions += ssa_node_day(c, counts, N, v, day, phi[v], NULL);
    return 0;
}

int orc_phi_nodes(const orc_cfg* c, const int32_t* counts, double* phi, int32_t day, int32_t v0, int32_t v1)
{
    const int32_t N = c->n_nodes;
    if (v0 < 0 || v1 < v0 || v1 > N || day < 0) return -1;
    for (int32_t v = v0; v < v1; ++v) phi[v] = phi_next(c, counts, N, v, day, phi[v], NULL);
    return 0;
}
