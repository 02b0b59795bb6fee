/*
 * FP64 CPU oracle of the sum-product LDPC decoder of arXiv:1609.01567.
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow reference that the CUDA
 * path is checked against. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, table or helper with the CUDA library.
 *
 * What it computes (the paper's Algorithms 1-6, read in the LLR domain):
 *
 *   Edges. An edge is a nonzero H[i][j] (Section II-B, Eqs. 1-2). Edge ids e
 *   are the COO entries stably sorted by column (Table 1: e, v, c); within a
 *   check, edges are kept in increasing e (Table 2: ebar is e stably sorted
 *   by check).
 *
 *   LLR convention. Probabilities on edges are P(bit = 1) (Algorithm 3 stores
 *   p_j = 1/(1+exp(-2 y_j / sigma^2)) as q; Algorithm 5 decides 1 when
 *   Q1 > Q0). So lambda_j = ln(P1/P0) = 2 y_j / sigma^2 and a positive LLR
 *   favours bit 1.
 *
 *   Bit-node rule (Algorithm 1, "Values to Check Nodes", normalised as in
 *   standard sum-product): q_ij = lambda_j + sum_{i' in M_j \ i} r_i'j.
 *
 *   Check-node rule (Algorithm 1, "Values to Variable Nodes"): from
 *   r0 - r1 = prod (1 - 2 q1), in sign-magnitude form
 *     |r_ij| = phi^(sum_{j' in N_i \ j} phi^(|q_ij'|)),
 *     r_ij > 0  iff an odd number of the other inputs q_ij' are > 0,
 *   with phi(x) = ln((e^x + 1)/(e^x - 1)) = log1p(2/expm1(x)) and the
 *   saturated phi^(x) = phi(clamp(x, phi(L_MAX), L_MAX)). The paper works
 *   with unsaturated FP64 probabilities; L_MAX (default 20) is the reading
 *   for the silent case.
 *
 *   Estimation (Algorithm 4): APP_j = lambda_j + sum_{i in M_j} r_ij, and
 *   c_j = 1 iff APP_j > 0 (the tie goes to 0, as in Algorithm 5).
 *
 *   Syndrome (Algorithm 6): z_i = xor_{j in N_i} c_j.
 *
 *   Loop (Algorithm 2): a check pass on q = lambda, estimation and syndrome
 *   test (success there gives 0 iterations), then up to max_iter iterations
 *   of bit pass, check pass, estimation, syndrome test. With early exit off
 *   every frame runs all max_iter iterations and reports the final syndrome.
 *
 *   Min-sum family (named by the paper as a derived algorithm the same
 *   edge-level parallel scheme supports; not part of its exact SP rule):
 *   |r_ij| = min(L_MAX, max(alpha * min_{j' in N_i \ j} |q_ij'| - beta, 0)),
 *   same sign rule; alpha < 1 is the normalised, beta > 0 the offset variant.
 *   An empty minimum (degree-1 check) is L_MAX.
 *
 *   Degree-adaptive min-sum (rule 3; the paper names adaptive MS only by
 *   citation, read here as one scale and offset per check degree): check i
 *   of degree d uses alpha_d = alpha_by_degree[min(d, n_degrees - 1)] and
 *   beta_d likewise in the min-sum rule above.
 *
 *   Tabulated phi (rule 2; the look-up-table direction the paper names for
 *   further speed-up): phi is replaced by its chords on a log-spaced grid. The bucket
 *   of x >= 0 is the top 15 bits of the IEEE single-precision pattern of x
 *   (sign, 8 exponent bits, 6 mantissa bits): 64 buckets per octave, bucket
 *   key k spanning [e_k, e_(k+1)) with e_k the float whose bits are k << 17.
 *   On a bucket, phi_T(x) = phi(e_k) + (x - e_k) (phi(e_(k+1)) - phi(e_k)) /
 *   (e_(k+1) - e_k), a continuous piecewise-linear function; the check rule
 *   is the sum-product rule with phi_T in place of phi (same saturation).
 *
 *   Quantised message storage (the reduced-precision direction the paper names for
 *   further speed-up; its own decoder keeps FP64): when qstep > 0 every
 *   check-to-bit message is stored as r = k * qstep, k = r / qstep rounded to
 *   the nearest integer (ties to even) and clamped to [-qlevels, qlevels].
 *   Everything computed from the stored messages (q, APP, the decision) uses
 *   the stored values; node arithmetic stays FP64. int8 storage is
 *   qstep = 20/127, qlevels = 127.
 *
 *   Floating-point message storage (the same direction, 16-bit formats): each
 *   message is rounded to the nearest value of a binary format with p
 *   significand bits and minimum normal exponent emin, ties to even, as IEEE
 *   754 defines round-to-nearest: at exponent e (2^e <= |r| < 2^(e+1)) the
 *   values are spaced 2^(max(e, emin) - p + 1), so magnitudes below 2^emin
 *   keep the subnormal spacing. binary16: p = 11, emin = -14; bfloat16:
 *   p = 8, emin = -126. Stored messages stay far below either format's
 *   largest value (|r| <= L_MAX), so overflow does not arise.
 *
 *   Channel (BER-simulator section, Eqs. 3-4): x = 2c - 1, y = x + sigma z,
 *   lambda = 2 y / sigma^2, with z from Philox-4x64-10 (Salmon et al., SC'11)
 *   and the Box-Muller transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Tanner graph as plain adjacency lists                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t m, n;
    int64_t E;
    int32_t *var_of;   /* [E] variable of edge e                        */
    int32_t *chk_of;   /* [E] check of edge e                           */
    int64_t *vstart;   /* [n+1] M_j = edges vstart[j] .. vstart[j+1]-1   */
    int64_t *cstart;   /* [m+1] N_i = cedge[cstart[i] .. cstart[i+1]-1]  */
    int64_t *cedge;    /* [E] edges grouped by check, increasing e        */
} orc_graph;

static void graph_free(orc_graph *g) {
    free(g->var_of); free(g->chk_of); free(g->vstart); free(g->cstart); free(g->cedge);
}

/* Returns 0, or -1 on bad input / allocation failure. */
static int graph_build(int32_t m, int32_t n, int64_t E, const int32_t *rows, const int32_t *cols,
                       orc_graph *g) {
    memset(g, 0, sizeof(*g));
    g->m = m; g->n = n; g->E = E;
    g->var_of = malloc(sizeof(int32_t) * (E ? E : 1));
    g->chk_of = malloc(sizeof(int32_t) * (E ? E : 1));
    g->vstart = calloc((size_t)n + 1, sizeof(int64_t));
    g->cstart = calloc((size_t)m + 1, sizeof(int64_t));
    g->cedge = malloc(sizeof(int64_t) * (E ? E : 1));
    if (!g->var_of || !g->chk_of || !g->vstart || !g->cstart || !g->cedge) { graph_free(g); return -1; }
    for (int64_t t = 0; t < E; ++t) {
        if (rows[t] < 0 || rows[t] >= m || cols[t] < 0 || cols[t] >= n) { graph_free(g); return -1; }
        g->vstart[cols[t] + 1]++;
        g->cstart[rows[t] + 1]++;
    }
    for (int32_t j = 0; j < n; ++j) g->vstart[j + 1] += g->vstart[j];
    for (int32_t i = 0; i < m; ++i) g->cstart[i + 1] += g->cstart[i];
    /* stable sort of the COO by column: edge id = slot in column order */
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)(n > m ? n : m) + 1));
    if (!fill) { graph_free(g); return -1; }
    for (int32_t j = 0; j < n; ++j) fill[j] = g->vstart[j];
    for (int64_t t = 0; t < E; ++t) {
        int64_t e = fill[cols[t]]++;
        g->var_of[e] = cols[t];
        g->chk_of[e] = rows[t];
    }
    /* each check's edges in increasing edge id (stable sort of e by check) */
    for (int32_t i = 0; i < m; ++i) fill[i] = g->cstart[i];
    for (int64_t e = 0; e < E; ++e) g->cedge[fill[g->chk_of[e]]++] = e;
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Node rules                                                               */
/* ------------------------------------------------------------------------ */

/* phi(x) = ln((e^x + 1)/(e^x - 1)) for x > 0. */
static double phi(double x) { return log1p(2.0 / expm1(x)); }

/* phi with its argument clamped to [phi(L_MAX), L_MAX]. */
static double phi_hat(double x, double l_max) {
    double lo = phi(l_max);
    if (x < lo) x = lo;
    if (x > l_max) x = l_max;
    return phi(x);
}

/* phi_T: phi on the chords of the log-spaced bucket grid (rule 2). */
static double bucket_edge(uint32_t key) {
    uint32_t bits = key << 17;
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

static double phi_chord(double x) {
    float xf = (float)x;  /* the bucket is chosen on the single-precision value */
    uint32_t bits;
    memcpy(&bits, &xf, sizeof bits);
    uint32_t key = bits >> 17;
    double lo = bucket_edge(key), hi = bucket_edge(key + 1);
    double plo = phi(lo), phi_hi = phi(hi);
    return plo + (x - lo) * (phi_hi - plo) / (hi - lo);
}

static double phi_chord_hat(double x, double l_max) {
    double lo = phi(l_max);
    if (x < lo) x = lo;
    if (x > l_max) x = l_max;
    return phi_chord(x);
}

/* Check rule selection: 0 = sum-product, 1 = min-sum family, 2 = sum-product
 * with tabulated phi, 3 = min-sum with a scale and offset per check degree. */
typedef struct {
    int rule;
    double alpha, beta;
    const double *alpha_d, *beta_d;  /* rule 3: [n_deg], indexed by check degree */
    int32_t n_deg;
    int32_t qformat;  /* stored messages: 0 unrounded, 1 the lattice k * qstep,
                         2 binary16, 3 bfloat16 */
    double qstep;     /* format 1: the lattice step */
    int32_t qlevels;  /* format 1: largest stored |k| */
} orc_rule;

/* r rounded to the nearest value of a binary floating-point format with p
 * significand bits and minimum normal exponent emin (ties to even). */
static double round_to_format(double r, int p, int emin) {
    if (r == 0.0 || !isfinite(r)) return r;
    int e2;
    frexp(r, &e2); /* |r| = m 2^e2, 1/2 <= m < 1: the leading bit has exponent e2 - 1 */
    int e = e2 - 1;
    if (e < emin) e = emin;
    double spacing = ldexp(1.0, e - p + 1);
    return nearbyint(r / spacing) * spacing; /* exact scaling by a power of two */
}

/* The stored value of a message under the rule's storage format. */
static double quantise(double r, const orc_rule *rule) {
    if (rule->qformat == 2) return round_to_format(r, 11, -14);
    if (rule->qformat == 3) return round_to_format(r, 8, -126);
    double k = nearbyint(r / rule->qstep);
    if (k > rule->qlevels) k = rule->qlevels;
    if (k < -rule->qlevels) k = -rule->qlevels;
    return k * rule->qstep;
}

/* Min-sum check rule for one check. */
static void check_update_min_sum(const orc_graph *g, int32_t i, const double *q, double *r, double l_max,
                                 const orc_rule *rule, int *one) {
    int64_t b = g->cstart[i], d = g->cstart[i + 1] - b;
    double alpha = rule->alpha, beta = rule->beta;
    if (rule->rule == 3) {
        int64_t t = d < rule->n_deg ? d : rule->n_deg - 1;
        alpha = rule->alpha_d[t];
        beta = rule->beta_d[t];
    }
    for (int64_t k = 0; k < d; ++k) one[k] = q[g->cedge[b + k]] > 0.0;
    for (int64_t k = 0; k < d; ++k) {
        double m = l_max;
        int parity = 0;
        for (int64_t k2 = 0; k2 < d; ++k2) {
            if (k2 == k) continue;
            double a = fabs(q[g->cedge[b + k2]]);
            if (a < m) m = a;
            parity ^= one[k2];
        }
        double a = alpha * m - beta;
        if (a < 0.0) a = 0.0;
        if (a > l_max) a = l_max;
        r[g->cedge[b + k]] = parity ? a : -a;
    }
}

/* Check-node rule for one check: r[e] for every e in N_i from q[e];
 * `table` selects phi_T for phi. */
static void check_update(const orc_graph *g, int32_t i, const double *q, double *r, double l_max,
                         double *mag, int *one, int table) {
    int64_t b = g->cstart[i], d = g->cstart[i + 1] - b;
    for (int64_t k = 0; k < d; ++k) {
        double qk = q[g->cedge[b + k]];
        mag[k] = table ? phi_chord_hat(fabs(qk), l_max) : phi_hat(fabs(qk), l_max);
        one[k] = qk > 0.0;
    }
    for (int64_t k = 0; k < d; ++k) {
        double s = 0.0;
        int parity = 0;
        for (int64_t k2 = 0; k2 < d; ++k2) {
            if (k2 == k) continue;
            s += mag[k2];
            parity ^= one[k2];
        }
        double a = table ? phi_chord_hat(s, l_max) : phi_hat(s, l_max);
        r[g->cedge[b + k]] = parity ? a : -a;
    }
}

/* One flooding pass of Algorithm 2 for one frame.
 * r_prev == NULL: the first check pass, q = lambda (Algorithm 3).
 * Otherwise q_e = lambda_j + sum over the other edges of j of r_prev.
 * Writes r_next [E], app [n], chat [n] and returns the syndrome weight. */
static int64_t sp_pass(const orc_graph *g, const double *lam, const double *r_prev, double *r_next,
                       double *app, uint8_t *chat, double l_max, const orc_rule *rule, double *q, double *mag,
                       int *one) {
    for (int32_t j = 0; j < g->n; ++j) {
        for (int64_t e = g->vstart[j]; e < g->vstart[j + 1]; ++e) {
            double v = lam[j];
            if (r_prev)
                for (int64_t e2 = g->vstart[j]; e2 < g->vstart[j + 1]; ++e2)
                    if (e2 != e) v += r_prev[e2];
            q[e] = v;
        }
    }
    for (int32_t i = 0; i < g->m; ++i) {
        if (rule && (rule->rule == 1 || rule->rule == 3))
            check_update_min_sum(g, i, q, r_next, l_max, rule, one);
        else
            check_update(g, i, q, r_next, l_max, mag, one, rule && rule->rule == 2);
    }
    if (rule && rule->qformat != 0)
        for (int64_t e = 0; e < g->E; ++e) r_next[e] = quantise(r_next[e], rule);
    for (int32_t j = 0; j < g->n; ++j) {
        double v = lam[j];
        for (int64_t e = g->vstart[j]; e < g->vstart[j + 1]; ++e) v += r_next[e];
        app[j] = v;
        chat[j] = v > 0.0;
    }
    int64_t weight = 0;
    for (int32_t i = 0; i < g->m; ++i) {
        int z = 0;
        for (int64_t k = g->cstart[i]; k < g->cstart[i + 1]; ++k) z ^= chat[g->var_of[g->cedge[k]]];
        weight += z;
    }
    return weight;
}

static int64_t max_check_degree(const orc_graph *g) {
    int64_t dmax = 1;
    for (int32_t i = 0; i < g->m; ++i)
        if (g->cstart[i + 1] - g->cstart[i] > dmax) dmax = g->cstart[i + 1] - g->cstart[i];
    return dmax;
}

/* ------------------------------------------------------------------------ */
/* Public entry points (called through ctypes from oracle.py)               */
/* ------------------------------------------------------------------------ */

/* Nonzero when a rule's parameters are out of range: alpha > 0 and beta >= 0
 * (each table entry too, rule 3, which needs at least one entry); rule 2
 * needs l_max <= 22, since the bucket grid spans [2^-32, 2^5). */
static int rule_invalid(int32_t check_rule, double alpha, double beta, double l_max, const double *alpha_d,
                        const double *beta_d, int32_t n_deg) {
    if (check_rule < 0 || check_rule > 3 || !(alpha > 0.0) || !(beta >= 0.0)) return 1;
    if (check_rule == 2 && !(l_max <= 22.0)) return 1;
    if (check_rule == 3) {
        if (n_deg < 1 || !alpha_d || !beta_d) return 1;
        for (int32_t t = 0; t < n_deg; ++t)
            if (!(alpha_d[t] > 0.0) || !(beta_d[t] >= 0.0) || !isfinite(alpha_d[t]) || !isfinite(beta_d[t]))
                return 1;
    }
    return 0;
}

/* Decode n_frames frames of LLRs lam [F][n] (FP64).
 * Outputs: bits [F][n], iters [F], ok [F]; optional post [F][n] (APP LLRs)
 * and r_out [F][E] (last check-to-bit messages, edge order).
 * Returns 0, or -1 on bad input / allocation failure. */
int orc_decode(int32_t m, int32_t n, int64_t E, const int32_t *rows, const int32_t *cols,
               const double *lam, int32_t n_frames, int32_t max_iter, int32_t early_exit, double l_max,
               uint8_t *bits, int32_t *iters, uint8_t *ok, double *post, double *r_out, int32_t n_threads,
               int32_t check_rule, double alpha, double beta, int32_t qformat, double qstep, int32_t qlevels,
               const double *alpha_by_degree, const double *beta_by_degree, int32_t n_degrees) {
    if (m < 0 || n < 0 || E < 0 || n_frames < 0 || max_iter < 0 || !(l_max > 0.0)) return -1;
    if (rule_invalid(check_rule, alpha, beta, l_max, alpha_by_degree, beta_by_degree, n_degrees)) return -1;
    if (qformat < 0 || qformat > 3 || (qformat == 1 && (!(qstep > 0.0) || qlevels < 1))) return -1;
    orc_rule rule = {check_rule, alpha, beta, alpha_by_degree, beta_by_degree, n_degrees, qformat, qstep, qlevels};
    orc_graph g;
    if (graph_build(m, n, E, rows, cols, &g)) return -1;
    int64_t dmax = max_check_degree(&g);
    int failed = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t f = 0; f < n_frames; ++f) {
        size_t ecount = (size_t)(E ? E : 1);
        double *q = malloc(sizeof(double) * ecount);
        double *ra = malloc(sizeof(double) * ecount);
        double *rb = malloc(sizeof(double) * ecount);
        double *app = malloc(sizeof(double) * ((size_t)n + 1));
        uint8_t *chat = malloc((size_t)n + 1);
        double *mag = malloc(sizeof(double) * (size_t)dmax);
        int *one = malloc(sizeof(int) * (size_t)dmax);
        if (!q || !ra || !rb || !app || !chat || !mag || !one) {
            failed = 1;
        } else {
            const double *lf = lam + (size_t)f * n;
            double *r_cur = ra, *r_new = rb;
            /* first check pass, estimation and syndrome test (before the loop) */
            int64_t w = sp_pass(&g, lf, NULL, r_cur, app, chat, l_max, &rule, q, mag, one);
            int32_t it_done = 0;
            int stopped = early_exit && w == 0;
            for (int32_t it = 1; it <= max_iter && !stopped; ++it) {
                w = sp_pass(&g, lf, r_cur, r_new, app, chat, l_max, &rule, q, mag, one);
                double *t = r_cur; r_cur = r_new; r_new = t;
                it_done = it;
                if (early_exit && w == 0) stopped = 1;
            }
            iters[f] = stopped ? it_done : max_iter;
            ok[f] = w == 0;
            memcpy(bits + (size_t)f * n, chat, (size_t)n);
            if (post) memcpy(post + (size_t)f * n, app, sizeof(double) * (size_t)n);
            if (r_out) memcpy(r_out + (size_t)f * E, r_cur, sizeof(double) * (size_t)E);
        }
        free(q); free(ra); free(rb); free(app); free(chat); free(mag); free(one);
    }
    graph_free(&g);
    return failed ? -1 : 0;
}

/* One pass for every frame, starting from given messages r_prev [F][E]
 * (NULL: the first check pass on q = lambda). Writes r_next [F][E],
 * app [F][n], bits [F][n], syndrome weight [F]. Used to check the CUDA path
 * one iteration at a time from its own state. */
int orc_pass(int32_t m, int32_t n, int64_t E, const int32_t *rows, const int32_t *cols,
             const double *lam, int32_t n_frames, const double *r_prev, double l_max,
             double *r_next, double *app, uint8_t *bits, int64_t *weight, int32_t n_threads,
             int32_t check_rule, double alpha, double beta, int32_t qformat, double qstep, int32_t qlevels,
             const double *alpha_by_degree, const double *beta_by_degree, int32_t n_degrees) {
    if (m < 0 || n < 0 || E < 0 || n_frames < 0 || !(l_max > 0.0)) return -1;
    if (rule_invalid(check_rule, alpha, beta, l_max, alpha_by_degree, beta_by_degree, n_degrees)) return -1;
    if (qformat < 0 || qformat > 3 || (qformat == 1 && (!(qstep > 0.0) || qlevels < 1))) return -1;
    orc_rule rule = {check_rule, alpha, beta, alpha_by_degree, beta_by_degree, n_degrees, qformat, qstep, qlevels};
    orc_graph g;
    if (graph_build(m, n, E, rows, cols, &g)) return -1;
    int64_t dmax = max_check_degree(&g);
    int failed = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t f = 0; f < n_frames; ++f) {
        double *q = malloc(sizeof(double) * (size_t)(E ? E : 1));
        double *mag = malloc(sizeof(double) * (size_t)dmax);
        int *one = malloc(sizeof(int) * (size_t)dmax);
        if (!q || !mag || !one) {
            failed = 1;
        } else {
            weight[f] = sp_pass(&g, lam + (size_t)f * n, r_prev ? r_prev + (size_t)f * E : NULL,
                                r_next + (size_t)f * E, app + (size_t)f * n, bits + (size_t)f * n, l_max, &rule,
                                q, mag, one);
        }
        free(q); free(mag); free(one);
    }
    graph_free(&g);
    return failed ? -1 : 0;
}

/* The stored value of r under storage format qformat (1 needs qstep and
 * qlevels), exported for the pins of the storage formats. */
double orc_store(double r, int32_t qformat, double qstep, int32_t qlevels) {
    orc_rule rule;
    memset(&rule, 0, sizeof(rule));
    rule.qformat = qformat;
    rule.qstep = qstep;
    rule.qlevels = qlevels;
    return qformat == 0 ? r : quantise(r, &rule);
}

/* phi and its tabulated form, exported for the pins of rule 2. */
double orc_phi(double x) { return phi(x); }
double orc_phi_chord(double x) { return phi_chord(x); }

/* Syndrome weights of hard words bits [F][n]: number of unsatisfied checks. */
int orc_syndrome(int32_t m, int32_t n, int64_t E, const int32_t *rows, const int32_t *cols,
                 const uint8_t *bits, int32_t n_frames, int64_t *weight) {
    orc_graph g;
    if (graph_build(m, n, E, rows, cols, &g)) return -1;
    for (int32_t f = 0; f < n_frames; ++f) {
        const uint8_t *b = bits + (size_t)f * n;
        int64_t w = 0;
        for (int32_t i = 0; i < m; ++i) {
            int z = 0;
            for (int64_t k = g.cstart[i]; k < g.cstart[i + 1]; ++k) z ^= b[g.var_of[g.cedge[k]]] & 1;
            w += z;
        }
        weight[f] = w;
    }
    graph_free(&g);
    return 0;
}

/* Address iterators of the paper, Tables 1-2, from the definitions of
 * Section III-B: for edge e (variable-sorted) v, c, t = degree of v,
 * s = first edge of v, u = e - s; for check-sorted slot k, ebar = edge id,
 * vbar, cbar, tbar = degree of cbar, sbar = first slot of cbar, ubar = k - sbar. */
int orc_address_iterators(int32_t m, int32_t n, int64_t E, const int32_t *rows, const int32_t *cols,
                          int32_t *v, int32_t *c, int32_t *t, int32_t *s, int32_t *u, int32_t *ebar,
                          int32_t *vbar, int32_t *cbar, int32_t *tbar, int32_t *sbar, int32_t *ubar) {
    orc_graph g;
    if (graph_build(m, n, E, rows, cols, &g)) return -1;
    for (int64_t e = 0; e < E; ++e) {
        int32_t j = g.var_of[e];
        v[e] = j;
        c[e] = g.chk_of[e];
        t[e] = (int32_t)(g.vstart[j + 1] - g.vstart[j]);
        s[e] = (int32_t)g.vstart[j];
        u[e] = (int32_t)(e - g.vstart[j]);
    }
    for (int32_t i = 0; i < m; ++i) {
        for (int64_t k = g.cstart[i]; k < g.cstart[i + 1]; ++k) {
            int64_t e = g.cedge[k];
            ebar[k] = (int32_t)e;
            vbar[k] = g.var_of[e];
            cbar[k] = i;
            tbar[k] = (int32_t)(g.cstart[i + 1] - g.cstart[i]);
            sbar[k] = (int32_t)g.cstart[i];
            ubar[k] = (int32_t)(k - g.cstart[i]);
        }
    }
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Channel: Philox-4x64-10 and Box-Muller                                   */
/* ------------------------------------------------------------------------ */

/* Philox-4x64 with 10 rounds, from Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): each round multiplies words 0
 * and 2 by two fixed odd constants into 128-bit products, then mixes their
 * halves with words 1 and 3 and the round key; the key is bumped by two
 * Weyl constants between rounds. */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Raw Philox blocks for counters (ctr0 + i, ctr1, 0, 0), i < count: out [count][4]. */
void orc_philox_blocks(uint64_t key0, uint64_t key1, uint64_t ctr0, uint64_t ctr1, int64_t count, uint64_t *out) {
    uint64_t key[2] = {key0, key1};
    for (int64_t i = 0; i < count; ++i) {
        uint64_t ctr[4] = {ctr0 + (uint64_t)i, ctr1, 0, 0};
        orc_philox4x64_10(ctr, key, out + 4 * i);
    }
}

/* BPSK over AWGN, LLR per bit (FP64).
 * Frame f (global index frame_offset + f), bit j: counter (j / 4, frame, 0, 0),
 * key (seed, 0). Block words (w0, w1) give the normals of bits 4q and 4q+1,
 * (w2, w3) those of bits 4q+2 and 4q+3, through Box-Muller on 24-bit uniforms
 *   ua = ((w >> 40) + 1) 2^-24 in (0, 1],  ub = (w >> 40) 2^-24 in [0, 1),
 *   rho = sqrt(-2 ln ua), z0 = rho cos(2 pi ub), z1 = rho sin(2 pi ub).
 * x = 2c - 1 (c = 0 when codewords is NULL), y = x + sigma z, llr = 2y / sigma^2. */
int orc_gen_awgn(uint64_t seed, int64_t frame_offset, int32_t n_frames, int32_t n, double sigma2,
                 const uint8_t *codewords, double *llr) {
    if (n_frames < 0 || n < 0 || !(sigma2 > 0.0)) return -1;
    const double sigma = sqrt(sigma2);
    const double two_pi = 6.283185307179586476925286766559;
    const double inv24 = 1.0 / 16777216.0;
    uint64_t key[2] = {seed, 0};
    for (int32_t f = 0; f < n_frames; ++f) {
        uint64_t frame = (uint64_t)(frame_offset + f);
        for (int32_t q4 = 0; q4 < (n + 3) / 4; ++q4) {
            uint64_t ctr[4] = {(uint64_t)q4, frame, 0, 0}, w[4];
            orc_philox4x64_10(ctr, key, w);
            double z[4];
            for (int pair = 0; pair < 2; ++pair) {
                double ua = ((double)(w[2 * pair] >> 40) + 1.0) * inv24;
                double ub = (double)(w[2 * pair + 1] >> 40) * inv24;
                double rho = sqrt(-2.0 * log(ua));
                z[2 * pair] = rho * cos(two_pi * ub);
                z[2 * pair + 1] = rho * sin(two_pi * ub);
            }
            for (int t = 0; t < 4; ++t) {
                int32_t j = 4 * q4 + t;
                if (j >= n) break;
                double x = codewords ? 2.0 * (double)codewords[(size_t)f * n + j] - 1.0 : -1.0;
                double y = x + sigma * z[t];
                llr[(size_t)f * n + j] = 2.0 * y / sigma2;
            }
        }
    }
    return 0;
}
