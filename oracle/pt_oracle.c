/*
 * pt_oracle.c -- plain, slow, FP64 CPU oracle for the Phylogenetic Topographer
 * (PT) hot path of arXiv 1811.11007.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header or table with the CUDA
 * path: every definition below is written out here from the paper and from the
 * textbook definitions the paper delegates to its likelihood library.
 *
 * What the paper fixes (section "Phylogenetic Topographer"):
 *   - the search loop: visit = optimise all branch lengths, discard below
 *     lmax + T, keep in the good set, update lmax, then for every unvisited NNI
 *     neighbour optimise the branches around the new edge and queue it if its
 *     partially optimised likelihood clears lmax + T;
 *   - NNI neighbourhoods, and a canonical per-topology key so no topology is
 *     visited twice;
 *   - JC69 / GTR with Gamma rate variation (section "Phylogenetic Topographer",
 *     "Maximum Likelihood Estimation of Local Maxima").
 * What the paper leaves to libpll and this oracle writes from textbook
 * definitions: Felsenstein pruning, the discrete-Gamma category rates (mean
 * of each equal-probability category), P(t) = expm(Q r t), Newton iterations
 * on one branch, the sweep order of the full optimisation, and the key (a sum
 * of 128-bit split hashes replacing the paper's sorted Newick strings).
 * Readings where the paper is silent are marked READING below.
 *
 * Parity status: every function here is pinned by a CPU test (closed forms,
 * brute force, library routines, invariants, the (2n-5)!! topology count),
 * except the finite-threshold visited sets and, beyond four taxa, the proposal
 * lengths, which the paper gives no values for ("parity unpinned"; they are
 * pinned only through invariants and the oracle-vs-GPU comparison).  On four
 * taxa the five branches of a proposal are the whole tree, and the proposal
 * is pinned to the likelihood maximum found by a library optimiser.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 128
#define OR_MAXNODE (2 * OR_MAXN - 2)
#define OR_MAXCAT 8
#define OR_LN2 0.6931471805599453094172321
/* per-site rescaling: when every entry of a conditional likelihood vector is
 * below 2^-256 the vector is multiplied by 2^256 (exact) and a counter
 * incremented (READING: per site, not per category). */
#define OR_SCALE_EXP 256

/* ------------------------------------------------------------------------- */
/* Problem: alignment (pattern-compressed), model, optimisation settings.      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n, P, C;
    uint8_t *tips;   /* [n][P], 0..3 = A C G T, 4 = gap / unknown */
    double *w;       /* [P] pattern weights */
    double pi[4];
    double Q[16];    /* normalised GTR rate matrix, row-major */
    double rates[OR_MAXCAT];
    double tmin, tmax, newton_tol, sweep_tol;
    int newton_maxit, full_max_sweeps, prop_max_sweeps;
    int prop_mode;   /* 0 = five branches around the NNI edge, 1 = central only, 2 = every branch */
    double prior_rate; /* 0: maximum likelihood; > 0: MAP under an Exponential(prior_rate) prior per branch */
    double alpha;      /* Gamma shape of the model (the rates above are its category means) */
    int reopt_alpha;   /* 1: every visit re-optimises the Gamma shape with the branch lengths */
    /* counters (diagnostics for tests) */
    long n_newton_evals, n_newton_nonconv;
} or_problem;

/* ------------------------------------------------------------------------- */
/* Regularised incomplete gamma P(a, x) and the discrete Gamma rates.           */
/* ------------------------------------------------------------------------- */
/* P(a,x) by its power series  e^-x x^a / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k))
 * for x < a + 1, otherwise 1 - Q(a,x) with Q from the Legendre continued
 * fraction evaluated by the modified Lentz method. */
double or_gamma_p(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double lpre = -x + a * log(x) - lgamma(a);
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term, ap = a;
        for (int k = 0; k < 100000; ++k) {
            ap += 1.0;
            term *= x / ap;
            sum += term;
            if (fabs(term) < fabs(sum) * 1e-17) break;
        }
        return sum * exp(lpre);
    }
    /* Q(a,x) = e^-x x^a / Gamma(a) * 1/(x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(x+5-a- ...))) */
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 100000; ++i) {
        double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return 1.0 - exp(lpre) * h;
}

/* Quantile of Gamma(shape alpha, rate alpha) at probability q, by bisection on
 * P(alpha, alpha x) (plain and monotone; 200 halvings exhaust FP64). */
static double or_gamma_quantile(double alpha, double q)
{
    double lo = 0.0, hi = 1.0;
    while (or_gamma_p(alpha, alpha * hi) < q) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (or_gamma_p(alpha, alpha * mid) < q) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Discrete Gamma with C equal-probability categories, each represented by its
 * conditional mean (READING: the mean method, not the median).  With the
 * category bounds b_k = F^-1(k/C) of Gamma(alpha, rate alpha), the mean of
 * category k is C * [P(alpha+1, alpha b_{k+1}) - P(alpha+1, alpha b_k)],
 * because x f_alpha(x) is the Gamma(alpha+1, rate alpha) density.  The rates
 * are finally renormalised to mean exactly 1. */
int or_gamma_rates(double alpha, int C, double *rates)
{
    if (C < 1 || C > OR_MAXCAT) return -1;
    if (C == 1) { rates[0] = 1.0; return 0; }
    if (!(alpha > 0.0)) return -1;
    double prev = 0.0, sum = 0.0;
    for (int k = 0; k < C; ++k) {
        double upper;
        if (k == C - 1) upper = 1.0;
        else upper = or_gamma_p(alpha + 1.0, alpha * or_gamma_quantile(alpha, (double)(k + 1) / C));
        rates[k] = C * (upper - prev);
        prev = upper;
        sum += rates[k];
    }
    for (int k = 0; k < C; ++k) rates[k] *= C / sum;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* GTR rate matrix and P(t) = expm(Q t).                                        */
/* ------------------------------------------------------------------------- */
/* Q_ij = s_ij pi_j (i != j), rows sum to zero, scaled so that the expected
 * number of substitutions per unit time  -sum_i pi_i Q_ii  equals 1.
 * Exchangeabilities in the order AC AG AT CG CT GT. */
int or_gtr_q(const double exch[6], const double freqs[4], double Q[16])
{
    double s[4][4] = {{0}};
    s[0][1] = s[1][0] = exch[0];
    s[0][2] = s[2][0] = exch[1];
    s[0][3] = s[3][0] = exch[2];
    s[1][2] = s[2][1] = exch[3];
    s[1][3] = s[3][1] = exch[4];
    s[2][3] = s[3][2] = exch[5];
    for (int i = 0; i < 4; ++i) if (!(freqs[i] > 0.0)) return -1;
    for (int i = 0; i < 6; ++i) if (!(exch[i] > 0.0)) return -1;
    double mu = 0.0;
    for (int i = 0; i < 4; ++i) {
        double row = 0.0;
        for (int j = 0; j < 4; ++j) {
            if (i == j) continue;
            Q[i * 4 + j] = s[i][j] * freqs[j];
            row += Q[i * 4 + j];
        }
        Q[i * 4 + i] = -row;
        mu += freqs[i] * row;
    }
    for (int i = 0; i < 16; ++i) Q[i] /= mu;
    return 0;
}

static void mat4_mul(const double *A, const double *B, double *R)
{
    double T[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc += A[i * 4 + k] * B[k * 4 + j];
            T[i * 4 + j] = acc;
        }
    memcpy(R, T, sizeof T);
}

/* expm(Q * s) by scaling and squaring of a truncated Taylor series: halve
 * until the 1-norm is below 1/2, sum 24 Taylor terms, square back. */
void or_expm(const double Q[16], double s, double E[16])
{
    double A[16], norm = 0.0;
    for (int i = 0; i < 16; ++i) A[i] = Q[i] * s;
    for (int j = 0; j < 4; ++j) {
        double col = 0.0;
        for (int i = 0; i < 4; ++i) col += fabs(A[i * 4 + j]);
        if (col > norm) norm = col;
    }
    int sq = 0;
    while (norm > 0.5) { norm *= 0.5; ++sq; }
    double scale = ldexp(1.0, -sq);
    for (int i = 0; i < 16; ++i) A[i] *= scale;
    double term[16], sum[16];
    for (int i = 0; i < 16; ++i) term[i] = sum[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int k = 1; k <= 24; ++k) {
        mat4_mul(term, A, term);
        for (int i = 0; i < 16; ++i) { term[i] /= k; sum[i] += term[i]; }
    }
    for (int k = 0; k < sq; ++k) mat4_mul(sum, sum, sum);
    memcpy(E, sum, sizeof sum);
}

/* ------------------------------------------------------------------------- */
/* Problem construction.                                                        */
/* ------------------------------------------------------------------------- */
or_problem *or_problem_new(int n, int P, int C, const uint8_t *tips, const double *w,
                           const double exch[6], const double freqs[4], double alpha)
{
    if (n < 3 || n > OR_MAXN || P < 0 || C < 1 || C > OR_MAXCAT) return NULL;
    or_problem *pb = (or_problem *)calloc(1, sizeof *pb);
    pb->n = n; pb->P = P; pb->C = C;
    pb->tips = (uint8_t *)malloc((size_t)n * (P ? P : 1));
    pb->w = (double *)malloc(sizeof(double) * (P ? P : 1));
    memcpy(pb->tips, tips, (size_t)n * P);
    memcpy(pb->w, w, sizeof(double) * P);
    for (int i = 0; i < 4; ++i) pb->pi[i] = freqs[i];
    pb->alpha = alpha;
    if (or_gtr_q(exch, freqs, pb->Q) || or_gamma_rates(alpha, C, pb->rates)) {
        free(pb->tips); free(pb->w); free(pb);
        return NULL;
    }
    pb->tmin = 1e-6; pb->tmax = 100.0;
    pb->newton_tol = 1e-8; pb->newton_maxit = 50;
    pb->sweep_tol = 1e-6; pb->full_max_sweeps = 64; pb->prop_max_sweeps = 8;
    pb->prop_mode = 0;
    pb->prior_rate = 0.0;
    return pb;
}

void or_problem_free(or_problem *pb)
{
    if (!pb) return;
    free(pb->tips); free(pb->w); free(pb);
}

/* MAP objective ("Phylogenetic Topographer", its optional exponential branch
 * length prior): every branch length gets an Exponential(rate) prior, so a
 * topology's score is lnL + sum over its 2n-3 branches of (ln rate - rate t);
 * rate 0 restores maximum likelihood (score = lnL). */
void or_problem_prior(or_problem *pb, double rate) { pb->prior_rate = rate; }

/* Model re-optimisation ("Phylogenetic Topographer": optimising the shape of
 * the Gamma rate heterogeneity for each visited topology): on = 1 makes every
 * visit (full optimisation of a start or a kept neighbour) optimise the shape
 * jointly with the branch lengths; proposals keep the model's shape. */
void or_problem_reopt(or_problem *pb, int on) { pb->reopt_alpha = on; }

void or_problem_settings(or_problem *pb, double tmin, double tmax, double newton_tol, int newton_maxit,
                         double sweep_tol, int full_max_sweeps, int prop_max_sweeps, int prop_mode)
{
    pb->tmin = tmin; pb->tmax = tmax; pb->newton_tol = newton_tol; pb->newton_maxit = newton_maxit;
    pb->sweep_tol = sweep_tol; pb->full_max_sweeps = full_max_sweeps;
    pb->prop_max_sweeps = prop_max_sweeps; pb->prop_mode = prop_mode;
}

void or_problem_model(const or_problem *pb, double *Q, double *rates)
{
    memcpy(Q, pb->Q, sizeof pb->Q);
    memcpy(rates, pb->rates, sizeof(double) * pb->C);
}

long or_problem_counter(const or_problem *pb, int which)
{
    return which == 0 ? pb->n_newton_evals : pb->n_newton_nonconv;
}

/* ------------------------------------------------------------------------- */
/* Unrooted binary trees: leaves 0..n-1, inner nodes n..2n-3, 2n-3 edges.        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n, nnode;
    int deg[OR_MAXNODE];
    int adj[OR_MAXNODE][3];
    double len[OR_MAXNODE][3]; /* len[v][k] = length of edge (v, adj[v][k]) */
} or_tree;

static int tree_find(const or_tree *t, int v, int u)
{
    for (int k = 0; k < t->deg[v]; ++k) if (t->adj[v][k] == u) return k;
    return -1;
}

static double tree_len(const or_tree *t, int u, int v) { return t->len[u][tree_find(t, u, v)]; }

static void tree_set_len(or_tree *t, int u, int v, double x)
{
    t->len[u][tree_find(t, u, v)] = x;
    t->len[v][tree_find(t, v, u)] = x;
}

/* Builds the adjacency form and checks that the edge list is a binary tree
 * on leaves 0..n-1 (leaves degree 1, inner nodes degree 3, connected). */
static int tree_from_edges(int n, const int32_t *edges, const double *lengths, or_tree *t)
{
    if (n < 3 || n > OR_MAXN) return -1;
    t->n = n; t->nnode = 2 * n - 2;
    for (int v = 0; v < t->nnode; ++v) t->deg[v] = 0;
    for (int e = 0; e < 2 * n - 3; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= t->nnode || b >= t->nnode || a == b) return -1;
        if (t->deg[a] >= 3 || t->deg[b] >= 3) return -1;
        double x = lengths ? lengths[e] : 0.1;
        t->adj[a][t->deg[a]] = b; t->len[a][t->deg[a]++] = x;
        t->adj[b][t->deg[b]] = a; t->len[b][t->deg[b]++] = x;
    }
    for (int v = 0; v < t->nnode; ++v) if (t->deg[v] != (v < n ? 1 : 3)) return -1;
    /* connectivity by a DFS from leaf 0 */
    int seen[OR_MAXNODE] = {0}, stack[OR_MAXNODE], sp = 0, cnt = 0;
    stack[sp++] = 0; seen[0] = 1;
    while (sp) {
        int v = stack[--sp]; ++cnt;
        for (int k = 0; k < t->deg[v]; ++k)
            if (!seen[t->adj[v][k]]) { seen[t->adj[v][k]] = 1; stack[sp++] = t->adj[v][k]; }
    }
    return cnt == t->nnode ? 0 : -1;
}

static void tree_to_edges(const or_tree *t, int32_t *edges, double *lengths)
{
    int e = 0;
    for (int v = 0; v < t->nnode; ++v)
        for (int k = 0; k < 3 && k < t->deg[v]; ++k) {
            int u = t->adj[v][k];
            if (u > v) {
                edges[2 * e] = v; edges[2 * e + 1] = u;
                if (lengths) lengths[e] = t->len[v][k];
                ++e;
            }
        }
}

/* Leaf set of the subtree at v seen from `from` (two 64-bit words). */
static void subtree_bits(const or_tree *t, int v, int from, uint64_t b[2])
{
    if (v < t->n) { b[0] = b[1] = 0; b[v >> 6] |= 1ull << (v & 63); return; }
    b[0] = b[1] = 0;
    for (int k = 0; k < 3; ++k) {
        int c = t->adj[v][k];
        if (c == from) continue;
        uint64_t cb[2];
        subtree_bits(t, c, v, cb);
        b[0] |= cb[0]; b[1] |= cb[1];
    }
}

static int min_taxon(const uint64_t b[2])
{
    if (b[0]) return __builtin_ctzll(b[0]);
    return 64 + __builtin_ctzll(b[1]);
}

/* ------------------------------------------------------------------------- */
/* Felsenstein pruning (per site, per category), FP64 with per-site scaling.   */
/* ------------------------------------------------------------------------- */
/* Conditional likelihood vector of the subtree hanging at v away from `from`:
 * out[p][r][i] = Pr(data below v at site p | state i at v, rate category r).
 * Leaves give a one-hot vector (all ones for code 4).  Inner nodes take the
 * product over their two children c of  sum_j P_r(t_vc)[i][j] out_c[p][r][j]. */
static void clv(const or_problem *pb, const or_tree *t, int v, int from, double *out, int *scl)
{
    const int P = pb->P, C = pb->C, S = 4 * C;
    if (v < t->n) {
        for (int p = 0; p < P; ++p) {
            int code = pb->tips[(size_t)v * P + p];
            for (int r = 0; r < C; ++r)
                for (int i = 0; i < 4; ++i)
                    out[(size_t)p * S + r * 4 + i] = (code >= 4 || code == i) ? 1.0 : 0.0;
            scl[p] = 0;
        }
        return;
    }
    for (int p = 0; p < P * S; ++p) out[p] = 1.0;
    for (int p = 0; p < P; ++p) scl[p] = 0;
    double *cv = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1) * S);
    int *cs = (int *)malloc(sizeof(int) * (P ? P : 1));
    for (int k = 0; k < 3; ++k) {
        int c = t->adj[v][k];
        if (c == from) continue;
        clv(pb, t, c, v, cv, cs);
        double Pm[OR_MAXCAT][16];
        for (int r = 0; r < C; ++r) or_expm(pb->Q, pb->rates[r] * t->len[v][k], Pm[r]);
        for (int p = 0; p < P; ++p) {
            for (int r = 0; r < C; ++r)
                for (int i = 0; i < 4; ++i) {
                    double acc = 0.0;
                    for (int j = 0; j < 4; ++j) acc += Pm[r][i * 4 + j] * cv[(size_t)p * S + r * 4 + j];
                    out[(size_t)p * S + r * 4 + i] *= acc;
                }
            scl[p] += cs[p];
        }
    }
    for (int p = 0; p < P; ++p) {
        double mx = 0.0;
        for (int q = 0; q < S; ++q) if (out[(size_t)p * S + q] > mx) mx = out[(size_t)p * S + q];
        if (mx < ldexp(1.0, -OR_SCALE_EXP)) {
            for (int q = 0; q < S; ++q) out[(size_t)p * S + q] = ldexp(out[(size_t)p * S + q], OR_SCALE_EXP);
            scl[p] += 1;
        }
    }
    free(cv); free(cs);
}

/* Log-likelihood with the tree rooted at inner node `root`:
 * L_p = sum_r (1/C) sum_i pi_i prod_{children c} sum_j P_r(t)[i][j] clv_c[p][r][j]
 * and lnL = sum_p w_p ln L_p (scaling counters undone).  Per-site values are
 * written to site_lnl when it is not NULL. */
static double lnl_rooted(const or_problem *pb, const or_tree *t, int root, double *site_lnl)
{
    const int P = pb->P, C = pb->C, S = 4 * C;
    double *X = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1) * S);
    int *sx = (int *)malloc(sizeof(int) * (P ? P : 1));
    clv(pb, t, root, -1, X, sx);  /* from = -1: all three neighbours are children */
    double total = 0.0;
    for (int p = 0; p < P; ++p) {
        double L = 0.0;
        for (int r = 0; r < C; ++r)
            for (int i = 0; i < 4; ++i) L += pb->pi[i] * X[(size_t)p * S + r * 4 + i];
        L /= C;
        double lp = log(L) - sx[p] * OR_SCALE_EXP * OR_LN2;
        if (site_lnl) site_lnl[p] = lp;
        total += pb->w[p] * lp;
    }
    free(X); free(sx);
    return total;
}

/* ------------------------------------------------------------------------- */
/* One branch: lnL(t), d lnL/dt, d2 lnL/dt2 given the two subtree vectors.      */
/* ------------------------------------------------------------------------- */
/* L_p(t) = sum_r (1/C) sum_ij pi_i X[p][r][i] P_r(t)[i][j] Y[p][r][j], with
 * dP_r/dt = r Q P_r and d2P_r/dt2 = r^2 Q^2 P_r.  Then
 *   f  = sum_p w_p ln L_p,  d1 = sum_p w_p L'_p/L_p,
 *   d2 = sum_p w_p (L''_p/L_p - (L'_p/L_p)^2). */
static void branch_eval(or_problem *pb, const double *X, const int *sx, const double *Y, const int *sy,
                        double t, double *f, double *d1, double *d2)
{
    const int P = pb->P, C = pb->C, S = 4 * C;
    double Pm[OR_MAXCAT][16], D1[OR_MAXCAT][16], D2[OR_MAXCAT][16], Q2[16];
    mat4_mul(pb->Q, pb->Q, Q2);
    for (int r = 0; r < C; ++r) {
        double rr = pb->rates[r];
        or_expm(pb->Q, rr * t, Pm[r]);
        mat4_mul(pb->Q, Pm[r], D1[r]);
        mat4_mul(Q2, Pm[r], D2[r]);
        for (int q = 0; q < 16; ++q) { D1[r][q] *= rr; D2[r][q] *= rr * rr; }
    }
    double F = 0.0, G = 0.0, H = 0.0;
    for (int p = 0; p < P; ++p) {
        double L = 0.0, L1 = 0.0, L2 = 0.0;
        for (int r = 0; r < C; ++r)
            for (int i = 0; i < 4; ++i) {
                double xi = pb->pi[i] * X[(size_t)p * S + r * 4 + i];
                for (int j = 0; j < 4; ++j) {
                    double yj = Y[(size_t)p * S + r * 4 + j];
                    L += xi * Pm[r][i * 4 + j] * yj;
                    L1 += xi * D1[r][i * 4 + j] * yj;
                    L2 += xi * D2[r][i * 4 + j] * yj;
                }
            }
        L /= C; L1 /= C; L2 /= C;
        double a = L1 / L, b = L2 / L;
        F += pb->w[p] * (log(L) - (sx[p] + sy[p]) * OR_SCALE_EXP * OR_LN2);
        G += pb->w[p] * a;
        H += pb->w[p] * (b - a * a);
    }
    *f = F; *d1 = G; *d2 = H;
    pb->n_newton_evals++;
}

/* Safeguarded Newton on one branch length (READING: the paper gives no rule).
 * The bracket [lo, hi] starts as [tmin, tmax]; after each evaluation the side
 * the derivative points away from is moved to t.  The Newton point
 * t - d1/d2 is taken when d2 < 0 and it falls strictly inside the bracket;
 * otherwise the bracket's geometric midpoint sqrt(lo*hi).  Stops when the
 * step is at most newton_tol, when d1 is exactly zero, or after newton_maxit
 * evaluations. */
static double newton_branch(or_problem *pb, const double *X, const int *sx, const double *Y, const int *sy,
                            double t0)
{
    double lo = pb->tmin, hi = pb->tmax;
    double t = t0 < lo ? lo : (t0 > hi ? hi : t0);
    for (int it = 0; it < pb->newton_maxit; ++it) {
        double f, d1, d2;
        branch_eval(pb, X, sx, Y, sy, t, &f, &d1, &d2);
        d1 -= pb->prior_rate;    /* the prior's ln rate - rate t has slope -rate */
        if (d1 == 0.0) return t; /* flat (e.g. a branch to an all-gap leaf) */
        if (d1 > 0.0) lo = t; else hi = t;
        double tn;
        if (d2 < 0.0 && (tn = t - d1 / d2) > lo && tn < hi) {
            /* Newton step accepted */
        } else {
            tn = sqrt(lo * hi);
        }
        if (fabs(tn - t) <= pb->newton_tol) return tn;
        t = tn;
    }
    pb->n_newton_nonconv++;
    return t;
}

/* Newton on edge (u, v) of tree t, with the two subtree vectors recomputed
 * from scratch by pruning.  Returns |change of the length|. */
static double optimise_edge(or_problem *pb, or_tree *t, int u, int v)
{
    const int P = pb->P, S = 4 * pb->C;
    size_t nb = (size_t)(P ? P : 1);
    double *X = (double *)malloc(sizeof(double) * nb * S), *Y = (double *)malloc(sizeof(double) * nb * S);
    int *sx = (int *)malloc(sizeof(int) * nb), *sy = (int *)malloc(sizeof(int) * nb);
    clv(pb, t, u, v, X, sx);
    clv(pb, t, v, u, Y, sy);
    double t0 = tree_len(t, u, v);
    double tn = newton_branch(pb, X, sx, Y, sy, t0);
    tree_set_len(t, u, v, tn);
    free(X); free(Y); free(sx); free(sy);
    return fabs(tn - t0);
}

static double tree_lnl(const or_problem *pb, const or_tree *t)
{
    return lnl_rooted(pb, t, t->n, NULL); /* node n is always an inner node */
}

/* The objective of a topology at its lengths: lnL, plus the log prior
 * density of the lengths under the MAP objective. */
static double tree_score(const or_problem *pb, const or_tree *t)
{
    double f = tree_lnl(pb, t);
    if (pb->prior_rate > 0.0) {
        double sum = 0.0;
        for (int u = 0; u < t->nnode; ++u)
            for (int j = 0; j < t->deg[u]; ++j)
                if (t->adj[u][j] > u) sum += t->len[u][j]; /* each edge once */
        f += (2 * t->n - 3) * log(pb->prior_rate) - pb->prior_rate * sum;
    }
    return f;
}

/* ------------------------------------------------------------------------- */
/* Full optimisation: sweeps over all 2n-3 edges (section "Phylogenetic         */
/* Topographer", step 2 of the loop; "full branch optimization").               */
/* ------------------------------------------------------------------------- */
/* READING: the sweep visits edges in pre-order from leaf 0: first the edge at
 * leaf 0, then, below each inner node, its two child subtrees in increasing
 * order of their smallest taxon.  Sweeps stop after the first sweep in which
 * no branch length moved by more than sweep_tol, or after full_max_sweeps
 * sweeps; the result is the exact lnL at the final lengths.  (A rule on the
 * lengths rather than on lnL gains: the lengths converge to within 1e-9 in
 * FP32 partials too, while lnL gains below ~1e-5 nats do not resolve there.) */
static int order_edges(const or_tree *t, int p, int q, int (*out)[2], int k)
{
    out[k][0] = p; out[k][1] = q; ++k;
    if (q < t->n) return k;
    int ch[2], nc = 0;
    for (int j = 0; j < 3; ++j) if (t->adj[q][j] != p) ch[nc++] = t->adj[q][j];
    uint64_t b0[2], b1[2];
    subtree_bits(t, ch[0], q, b0);
    subtree_bits(t, ch[1], q, b1);
    if (min_taxon(b1) < min_taxon(b0)) { int x = ch[0]; ch[0] = ch[1]; ch[1] = x; }
    k = order_edges(t, q, ch[0], out, k);
    k = order_edges(t, q, ch[1], out, k);
    return k;
}

static double full_optimise(or_problem *pb, or_tree *t, int *sweeps_out)
{
    int order[2 * OR_MAXN][2];
    int ne = order_edges(t, 0, t->adj[0][0], order, 0);
    int s;
    for (s = 0; s < pb->full_max_sweeps; ++s) {
        double moved = 0.0;
        for (int e = 0; e < ne; ++e) {
            double d = optimise_edge(pb, t, order[e][0], order[e][1]);
            if (d > moved) moved = d;
        }
        if (moved <= pb->sweep_tol) { ++s; break; }
    }
    if (sweeps_out) *sweeps_out = s;
    return tree_score(pb, t);
}

/* READING (the paper gives no procedure): the shape is searched on u = ln alpha
 * in [ln 0.02, ln 100] by golden-section search with a fixed 40 steps (final
 * bracket ~4e-8 wide; its midpoint is the new shape), at fixed branch
 * lengths, maximising lnL; then the lengths are fully re-optimised at the new
 * shape.  Shape search and length optimisation alternate until the shape
 * moves by at most 1e-6 in ln alpha (at most 16 alternations).  The visit's
 * score is the objective at the final shape and lengths. */
#define OR_ALPHA_LO 0.02
#define OR_ALPHA_HI 100.0
#define OR_GOLDEN_STEPS 40

static void set_alpha(or_problem *pb, double alpha)
{
    or_gamma_rates(alpha, pb->C, pb->rates);
}

static double golden_alpha(or_problem *pb, const or_tree *t)
{
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    double a = log(OR_ALPHA_LO), b = log(OR_ALPHA_HI);
    double x1 = b - g * (b - a), x2 = a + g * (b - a);
    set_alpha(pb, exp(x1));
    double f1 = tree_lnl(pb, t);
    set_alpha(pb, exp(x2));
    double f2 = tree_lnl(pb, t);
    for (int it = 0; it < OR_GOLDEN_STEPS; ++it) {
        if (f1 >= f2) {
            b = x2; x2 = x1; f2 = f1;
            x1 = b - g * (b - a);
            set_alpha(pb, exp(x1));
            f1 = tree_lnl(pb, t);
        } else {
            a = x1; x1 = x2; f1 = f2;
            x2 = a + g * (b - a);
            set_alpha(pb, exp(x2));
            f2 = tree_lnl(pb, t);
        }
    }
    return exp(0.5 * (a + b));
}

/* Full optimisation of lengths and (C > 1 and reopt_alpha) the Gamma shape.
 * alpha_out (may be NULL) receives the final shape; the problem's rates are
 * the model's again on return. */
static double visit_optimise(or_problem *pb, or_tree *t, double *alpha_out)
{
    double alpha = pb->alpha;
    if (!pb->reopt_alpha || pb->C == 1) {
        if (alpha_out) *alpha_out = alpha;
        return full_optimise(pb, t, NULL);
    }
    double f = full_optimise(pb, t, NULL);
    for (int alt = 0; alt < 16; ++alt) {
        double a2 = golden_alpha(pb, t);
        set_alpha(pb, a2);
        f = full_optimise(pb, t, NULL);
        int done = fabs(log(a2) - log(alpha)) <= 1e-6;
        alpha = a2;
        if (done) break;
    }
    set_alpha(pb, pb->alpha);
    if (alpha_out) *alpha_out = alpha;
    return f;
}

/* ------------------------------------------------------------------------- */
/* Split-set key (replaces the paper's sorted-Newick key).                      */
/* ------------------------------------------------------------------------- */
/* SplitMix64 output function (Steele, Lea and Flood 2014). */
uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* 128-bit hash of a split bitset (lo = taxa 0..63, hi = taxa 64..127):
 *   h.lo = mix64(lo ^ mix64(hi + 0x9e3779b97f4a7c15))
 *   h.hi = mix64(hi ^ mix64(lo + 0xd1b54a32d192ed03)) */
void or_split_hash(uint64_t lo, uint64_t hi, uint64_t h[2])
{
    h[0] = or_mix64(lo ^ or_mix64(hi + 0x9e3779b97f4a7c15ull));
    h[1] = or_mix64(hi ^ or_mix64(lo + 0xd1b54a32d192ed03ull));
}

static void add128(uint64_t a[2], const uint64_t b[2])
{
    uint64_t lo = a[0] + b[0];
    a[1] = a[1] + b[1] + (lo < a[0]);
    a[0] = lo;
}

static void sub128(uint64_t a[2], const uint64_t b[2])
{
    uint64_t lo = a[0] - b[0];
    a[1] = a[1] - b[1] - (a[0] < b[0]);
    a[0] = lo;
}

static int cmp128(const uint64_t a[2], const uint64_t b[2])
{
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return 0;
}

/* Non-trivial splits of the tree, each as the side without taxon 0, sorted
 * ascending as 128-bit integers (hi word first). Returns the count (n-3). */
static int tree_splits(const or_tree *t, uint64_t (*sp)[2])
{
    int m = 0;
    for (int v = t->n; v < t->nnode; ++v)
        for (int k = 0; k < 3; ++k) {
            int u = t->adj[v][k];
            if (u < t->n || u < v) continue; /* internal edge (v,u) once */
            uint64_t b[2];
            subtree_bits(t, u, v, b);
            if (b[0] & 1ull) { b[0] = ~b[0]; b[1] = ~b[1];
                /* complement within the n taxa */
                if (t->n < 64) { b[0] &= (1ull << t->n) - 1; b[1] = 0; }
                else if (t->n < 128) { b[1] &= (1ull << (t->n - 64)) - 1; }
            }
            sp[m][0] = b[0]; sp[m][1] = b[1]; ++m;
        }
    /* insertion sort */
    for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && cmp128(sp[j], sp[j - 1]) < 0; --j) {
            uint64_t x0 = sp[j][0], x1 = sp[j][1];
            sp[j][0] = sp[j - 1][0]; sp[j][1] = sp[j - 1][1];
            sp[j - 1][0] = x0; sp[j - 1][1] = x1;
        }
    return m;
}

/* key = sum over non-trivial splits of H(split) mod 2^128; a zero sum is
 * reported as 1 (zero marks an empty slot). */
static void key_of_splits(uint64_t (*sp)[2], int m, uint64_t key[2])
{
    key[0] = key[1] = 0;
    for (int i = 0; i < m; ++i) {
        uint64_t h[2];
        or_split_hash(sp[i][0], sp[i][1], h);
        add128(key, h);
    }
    if (!key[0] && !key[1]) key[0] = 1;
}

static void tree_key(const or_tree *t, uint64_t key[2])
{
    uint64_t sp[OR_MAXN][2];
    int m = tree_splits(t, sp);
    key_of_splits(sp, m, key);
}

/* ------------------------------------------------------------------------- */
/* NNI (section "Phylogenetic Topographer": neighbours by nearest-neighbour      */
/* interchange).                                                                */
/* ------------------------------------------------------------------------- */
/* Quartet around internal edge (u, v): u is the end whose far side holds
 * taxon 0; A = u's neighbour towards taxon 0, B = u's other neighbour; C, D =
 * v's other neighbours with min-taxon(C) < min-taxon(D).  Swap 0 exchanges B
 * and C, swap 1 exchanges B and D; every branch keeps its length. */
typedef struct { int u, v, a, b, c, d; uint64_t split[2]; } or_quartet;

static int quartets(const or_tree *t, or_quartet *qs)
{
    int m = 0;
    for (int x = t->n; x < t->nnode; ++x)
        for (int k = 0; k < 3; ++k) {
            int y = t->adj[x][k];
            if (y < t->n || y < x) continue;
            uint64_t bx[2];
            subtree_bits(t, x, y, bx); /* side of x away from y */
            int u = (bx[0] & 1ull) ? x : y, v = (u == x) ? y : x;
            or_quartet q; q.u = u; q.v = v;
            int on[2], no = 0;
            for (int j = 0; j < 3; ++j) if (t->adj[u][j] != v) on[no++] = t->adj[u][j];
            uint64_t b0[2];
            subtree_bits(t, on[0], u, b0);
            if (b0[0] & 1ull) { q.a = on[0]; q.b = on[1]; } else { q.a = on[1]; q.b = on[0]; }
            no = 0;
            for (int j = 0; j < 3; ++j) if (t->adj[v][j] != u) on[no++] = t->adj[v][j];
            uint64_t c0[2], c1[2];
            subtree_bits(t, on[0], v, c0);
            subtree_bits(t, on[1], v, c1);
            if (min_taxon(c0) < min_taxon(c1)) { q.c = on[0]; q.d = on[1]; } else { q.c = on[1]; q.d = on[0]; }
            subtree_bits(t, v, u, q.split); /* C u D: the side without taxon 0 */
            qs[m++] = q;
        }
    /* canonical edge order: ascending split */
    for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && cmp128(qs[j].split, qs[j - 1].split) < 0; --j) {
            or_quartet x = qs[j]; qs[j] = qs[j - 1]; qs[j - 1] = x;
        }
    return m;
}

/* Replaces neighbour `old` of node x by `nw`, keeping the slot's length. */
static void relink(or_tree *t, int x, int old, int nw)
{
    int k = tree_find(t, x, old);
    t->adj[x][k] = nw;
}

static void apply_nni(const or_tree *t, const or_quartet *q, int swap, or_tree *out)
{
    *out = *t;
    int s = swap == 0 ? q->c : q->d; /* the v-side subtree that moves to u */
    double tb = tree_len(t, q->u, q->b), ts = tree_len(t, q->v, s);
    /* b: u -> v ; s: v -> u */
    relink(out, q->u, q->b, s);
    relink(out, q->v, s, q->b);
    relink(out, q->b, q->u, q->v);
    relink(out, s, q->v, q->u);
    tree_set_len(out, q->v, q->b, tb);
    tree_set_len(out, q->u, s, ts);
}

/* Proposal optimisation of a neighbour: sweeps over the five branches the
 * NNI touches in the order central, A, B, C, D (prop_mode 0), or the central
 * branch only (prop_mode 1, the paper's radius-0 default).  Stop rule as for
 * the full optimisation (no length moved by more than sweep_tol), capped at
 * prop_max_sweeps; the result is the exact lnL at the final lengths.
 * prop_mode 2 is the paper's radius -1: the full optimisation of the
 * neighbour from its inherited lengths. */
static double propose_optimise(or_problem *pb, or_tree *nt, const or_quartet *q, int swap)
{
    if (pb->prop_mode == 2) return full_optimise(pb, nt, NULL);
    int s = swap == 0 ? q->c : q->d, o = swap == 0 ? q->d : q->c;
    /* after the swap: u holds a and s, v holds b and o */
    int br[5][2];
    br[0][0] = q->u; br[0][1] = q->v;
    br[1][0] = q->u; br[1][1] = q->a;
    br[2][0] = q->v; br[2][1] = q->b;
    /* C and D by label: c is attached to u if swap 0 else to v */
    br[3][0] = (q->c == s) ? q->u : q->v; br[3][1] = q->c;
    br[4][0] = (q->d == s) ? q->u : q->v; br[4][1] = q->d;
    (void)o;
    int nb = pb->prop_mode == 1 ? 1 : 5;
    for (int sw = 0; sw < pb->prop_max_sweeps; ++sw) {
        double moved = 0.0;
        for (int i = 0; i < nb; ++i) {
            double d = optimise_edge(pb, nt, br[i][0], br[i][1]);
            if (d > moved) moved = d;
        }
        if (moved <= pb->sweep_tol) break;
    }
    return tree_score(pb, nt);
}

/* ------------------------------------------------------------------------- */
/* Exported single-tree entry points (used by the tests).                      */
/* ------------------------------------------------------------------------- */
int or_loglik(const or_problem *pb, int n, const int32_t *edges, const double *lengths, int root,
              double *site_lnl, double *lnl)
{
    or_tree t;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    if (root < n || root >= t.nnode) root = n;
    *lnl = lnl_rooted(pb, &t, root, site_lnl);
    return 0;
}

/* lnL, d1, d2 with respect to the length of edge e (index into `edges`). */
int or_edge_derivs(or_problem *pb, int n, const int32_t *edges, const double *lengths, int e,
                   double *f, double *d1, double *d2)
{
    or_tree t;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    int u = edges[2 * e], v = edges[2 * e + 1];
    const int P = pb->P, S = 4 * pb->C;
    size_t nb = (size_t)(P ? P : 1);
    double *X = (double *)malloc(sizeof(double) * nb * S), *Y = (double *)malloc(sizeof(double) * nb * S);
    int *sx = (int *)malloc(sizeof(int) * nb), *sy = (int *)malloc(sizeof(int) * nb);
    clv(pb, &t, u, v, X, sx);
    clv(pb, &t, v, u, Y, sy);
    branch_eval(pb, X, sx, Y, sy, tree_len(&t, u, v), f, d1, d2);
    free(X); free(Y); free(sx); free(sy);
    return 0;
}

/* Full optimisation from the given lengths; lengths are overwritten in the
 * caller's edge order. */
int or_full_optimise(or_problem *pb, int n, const int32_t *edges, double *lengths, double *lnl, int *sweeps)
{
    or_tree t;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    *lnl = full_optimise(pb, &t, sweeps);
    for (int e = 0; e < 2 * n - 3; ++e) lengths[e] = tree_len(&t, edges[2 * e], edges[2 * e + 1]);
    return 0;
}

/* A visit: full optimisation, with the Gamma shape too when reopt_alpha is on. */
int or_visit_optimise(or_problem *pb, int n, const int32_t *edges, double *lengths, double *lnl, double *alpha)
{
    or_tree t;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    *lnl = visit_optimise(pb, &t, alpha);
    for (int e = 0; e < 2 * n - 3; ++e) lengths[e] = tree_len(&t, edges[2 * e], edges[2 * e + 1]);
    return 0;
}

int or_tree_key(int n, const int32_t *edges, uint64_t key[2])
{
    or_tree t;
    if (tree_from_edges(n, edges, NULL, &t)) return -1;
    tree_key(&t, key);
    return 0;
}

/* Sorted non-trivial splits, [n-3][2] words. */
int or_tree_splits(int n, const int32_t *edges, uint64_t *splits)
{
    or_tree t;
    if (tree_from_edges(n, edges, NULL, &t)) return -1;
    return tree_splits(&t, (uint64_t(*)[2])splits);
}

/* All 2(n-3) NNI neighbours, in canonical order (edge by ascending split,
 * then swap 0, 1).  Writes their edge lists / inherited lengths, keys, and
 * the edge index + swap of each. */
int or_nni_neighbours(int n, const int32_t *edges, const double *lengths, int32_t *nb_edges,
                      double *nb_lengths, uint64_t *nb_keys)
{
    or_tree t;
    if (tree_from_edges(n, edges, lengths, &t)) return -1;
    or_quartet qs[OR_MAXN];
    int m = quartets(&t, qs), k = 0;
    for (int i = 0; i < m; ++i)
        for (int s = 0; s < 2; ++s, ++k) {
            or_tree nt;
            apply_nni(&t, &qs[i], s, &nt);
            tree_to_edges(&nt, nb_edges + (size_t)k * 2 * (2 * n - 3), nb_lengths + (size_t)k * (2 * n - 3));
            tree_key(&nt, nb_keys + 2 * k);
        }
    return k;
}

/* Proposal optimisation of neighbour k (ordering as or_nni_neighbours) of a
 * tree: writes the neighbour's edges, its optimised lengths and lnL. */
int or_propose(or_problem *pb, int n, const int32_t *edges, const double *lengths, int k,
               int32_t *nb_edges, double *nb_lengths, double *lnl)
{
    or_tree t, nt;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    or_quartet qs[OR_MAXN];
    int m = quartets(&t, qs);
    if (k < 0 || k >= 2 * m) return -1;
    apply_nni(&t, &qs[k / 2], k % 2, &nt);
    *lnl = propose_optimise(pb, &nt, &qs[k / 2], k % 2);
    tree_to_edges(&nt, nb_edges, nb_lengths);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Visited table (plain open addressing with growth) + exact split sets.       */
/* ------------------------------------------------------------------------- */
enum { OR_REJECTED = 1, OR_GOOD = 2, OR_BAD = 3 };

typedef struct {
    uint64_t key[2];
    int status;
    double lnl;       /* proposal lnL for rejected ones, full lnL otherwise */
    double plnl;      /* proposal lnL (NaN for starts) */
    double alpha;     /* Gamma shape: the visit's (visited trees), the parent's (proposals) */
    int round;
    uint64_t ppkey[2], psplit[2]; /* the proposer that won this key's round: parent key, */
    int pswap;                    /* split of the edge it rearranged, swap (-1: not proposed) */
    uint64_t *splits; /* exact split set, for the injectivity check */
    int32_t *edges; double *lengths;
} or_entry;

typedef struct {
    or_entry *e; size_t cap, cnt;
    int n; int collision;
} or_set;

static size_t set_slot(const or_set *s, const uint64_t k[2])
{
    return (size_t)(or_mix64(k[0] ^ or_mix64(k[1])) & (s->cap - 1));
}

static or_entry *set_find(const or_set *s, const uint64_t k[2])
{
    for (size_t i = set_slot(s, k);; i = (i + 1) & (s->cap - 1)) {
        if (!s->e[i].status) return NULL;
        if (s->e[i].key[0] == k[0] && s->e[i].key[1] == k[1]) return &s->e[i];
    }
}

static or_entry *set_insert(or_set *s, const uint64_t k[2]);
static void set_grow(or_set *s)
{
    or_entry *old = s->e; size_t oc = s->cap;
    s->cap = oc ? oc * 2 : 1024;
    s->e = (or_entry *)calloc(s->cap, sizeof(or_entry));
    s->cnt = 0;
    for (size_t i = 0; i < oc; ++i)
        if (old[i].status) { or_entry *d = set_insert(s, old[i].key); *d = old[i]; }
    free(old);
}

static or_entry *set_insert(or_set *s, const uint64_t k[2])
{
    if (2 * (s->cnt + 1) > s->cap) set_grow(s);
    size_t i = set_slot(s, k);
    while (s->e[i].status) i = (i + 1) & (s->cap - 1);
    s->e[i].key[0] = k[0]; s->e[i].key[1] = k[1];
    s->e[i].status = -1; /* placeholder, set by caller */
    s->cnt++;
    return &s->e[i];
}

static void entry_fill(or_entry *e, const or_tree *t, int status, double lnl, double plnl, int round)
{
    int n = t->n;
    e->status = status; e->lnl = lnl; e->plnl = plnl; e->round = round;
    e->pswap = -1; e->ppkey[0] = e->ppkey[1] = e->psplit[0] = e->psplit[1] = 0;
    e->splits = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (n > 3 ? n - 3 : 1));
    tree_splits(t, (uint64_t(*)[2])e->splits);
    e->edges = (int32_t *)malloc(sizeof(int32_t) * 2 * (2 * n - 3));
    e->lengths = (double *)malloc(sizeof(double) * (2 * n - 3));
    tree_to_edges(t, e->edges, e->lengths);
}

static int entry_same_splits(const or_entry *e, const or_tree *t)
{
    uint64_t sp[OR_MAXN][2];
    int m = tree_splits(t, sp);
    return memcmp(sp, e->splits, sizeof(uint64_t) * 2 * m) == 0;
}

/* ------------------------------------------------------------------------- */
/* Round-synchronous PT search (loop of section "Phylogenetic Topographer").    */
/* ------------------------------------------------------------------------- */
/* READING (the paper's multithreaded loop is order-dependent; this is its
 * order-independent, round-by-round form):
 *  round 0: fully optimise every start; the first start of each key enters
 *     the visited set; lmax = best lnL; a start is GOOD iff lnL >= lmax - T;
 *     the frontier is the GOOD starts.
 *  round k: every frontier tree proposes its 2(n-3) NNI neighbours; keys
 *     already visited are skipped; among equal keys of this round the
 *     proposer with the smallest (parent key, edge split, swap) wins; the
 *     winner's neighbour is proposal-optimised to l', entered as visited,
 *     and kept iff l' >= lmax - T (lmax as at the start of the round).  Every
 *     kept neighbour is fully optimised to l; lmax = max(lmax, max l); it is
 *     GOOD iff l >= lmax - T (updated lmax), else BAD.  The GOOD ones are the
 *     next frontier.  A neighbour scored once is never re-scored.
 * The search stops when the frontier is empty or after max_rounds rounds. */
typedef struct {
    or_set vis;
    or_tree *front; int nfront;
    double lmax, T;
    int round;
    long n_scored, n_kept, n_good;
} or_search;

typedef struct { uint64_t pkey[2], split[2]; int swap; int parent; int qi; uint64_t nkey[2]; } or_cand;

static int cand_cmp_key(const void *a, const void *b)
{
    const or_cand *x = (const or_cand *)a, *y = (const or_cand *)b;
    int c = cmp128(x->nkey, y->nkey);
    if (c) return c;
    c = cmp128(x->pkey, y->pkey);
    if (c) return c;
    c = cmp128(x->split, y->split);
    if (c) return c;
    return x->swap - y->swap;
}

static int tree_cmp_key(const void *a, const void *b)
{
    uint64_t ka[2], kb[2];
    tree_key((const or_tree *)a, ka);
    tree_key((const or_tree *)b, kb);
    return cmp128(ka, kb);
}

or_search *or_search_new(or_problem *pb, int n_start, const int32_t *edges, const double *lengths, double T)
{
    int n = pb->n, ne = 2 * n - 3;
    or_search *s = (or_search *)calloc(1, sizeof *s);
    s->T = T; s->lmax = -INFINITY;
    s->vis.n = n;
    set_grow(&s->vis);
    or_tree *ts = (or_tree *)malloc(sizeof(or_tree) * (n_start ? n_start : 1));
    double *l = (double *)malloc(sizeof(double) * (n_start ? n_start : 1));
    int *keep = (int *)calloc(n_start ? n_start : 1, sizeof(int));
    for (int i = 0; i < n_start; ++i) {
        if (tree_from_edges(n, edges + (size_t)i * 2 * ne, lengths + (size_t)i * ne, &ts[i])) {
            free(ts); free(l); free(keep); free(s->vis.e); free(s); return NULL;
        }
        uint64_t k[2];
        tree_key(&ts[i], k);
        if (set_find(&s->vis, k)) continue;
        double al;
        l[i] = visit_optimise(pb, &ts[i], &al);
        or_entry *e = set_insert(&s->vis, k);
        entry_fill(e, &ts[i], OR_BAD, l[i], NAN, 0);
        e->alpha = al;
        keep[i] = 1;
        if (l[i] > s->lmax) s->lmax = l[i];
    }
    s->front = (or_tree *)malloc(sizeof(or_tree) * (n_start ? n_start : 1));
    for (int i = 0; i < n_start; ++i) {
        if (!keep[i]) continue;
        uint64_t k[2];
        tree_key(&ts[i], k);
        or_entry *e = set_find(&s->vis, k);
        if (l[i] >= s->lmax - T) { e->status = OR_GOOD; s->front[s->nfront++] = ts[i]; s->n_good++; }
    }
    qsort(s->front, s->nfront, sizeof(or_tree), tree_cmp_key);
    free(ts); free(l); free(keep);
    return s;
}

/* A search positioned just before a round on a given frontier: the trees are
 * entered as visited GOOD topologies with their given lengths (not
 * re-optimised) and lmax is taken as given.  The next or_search_round is then
 * one PT round on that frontier. */
or_search *or_search_from_frontier(or_problem *pb, int nf, const int32_t *edges, const double *lengths, double lmax,
                                   double T)
{
    int n = pb->n, ne = 2 * n - 3;
    or_search *s = (or_search *)calloc(1, sizeof *s);
    s->T = T; s->lmax = lmax;
    s->vis.n = n;
    set_grow(&s->vis);
    s->front = (or_tree *)malloc(sizeof(or_tree) * (size_t)(nf > 0 ? nf : 1));
    for (int i = 0; i < nf; ++i) {
        or_tree t;
        if (tree_from_edges(n, edges + (size_t)i * 2 * ne, lengths + (size_t)i * ne, &t)) {
            free(s->front); free(s->vis.e); free(s); return NULL;
        }
        uint64_t k[2];
        tree_key(&t, k);
        if (set_find(&s->vis, k)) continue;
        or_entry *e = set_insert(&s->vis, k);
        entry_fill(e, &t, OR_GOOD, NAN, NAN, 0);
        e->alpha = pb->alpha;  /* given without a shape: the model's */
        s->front[s->nfront++] = t;
    }
    qsort(s->front, s->nfront, sizeof(or_tree), tree_cmp_key);
    return s;
}

/* One round; returns the new frontier size. */
int or_search_round(or_problem *pb, or_search *s)
{
    int n = pb->n, m = 2 * (n - 3);
    double lmax0 = s->lmax, T = s->T;
    s->round++;
    or_cand *cs = (or_cand *)malloc(sizeof(or_cand) * ((size_t)s->nfront * m + 1));
    or_quartet *qall = (or_quartet *)malloc(sizeof(or_quartet) * ((size_t)s->nfront * (n - 3) + 1));
    int nc = 0;
    for (int f = 0; f < s->nfront; ++f) {
        uint64_t pk[2];
        tree_key(&s->front[f], pk);
        or_quartet *qs = qall + (size_t)f * (n - 3);
        int nq = quartets(&s->front[f], qs);
        for (int i = 0; i < nq; ++i)
            for (int sw = 0; sw < 2; ++sw) {
                or_tree nt;
                apply_nni(&s->front[f], &qs[i], sw, &nt);
                or_cand c;
                tree_key(&nt, c.nkey);
                if (set_find(&s->vis, c.nkey)) continue; /* visited in an earlier round */
                memcpy(c.pkey, pk, sizeof pk);
                memcpy(c.split, qs[i].split, sizeof c.split);
                c.swap = sw; c.parent = f; c.qi = i;
                cs[nc++] = c;
            }
    }
    qsort(cs, nc, sizeof(or_cand), cand_cmp_key);
    or_tree *kept = (or_tree *)malloc(sizeof(or_tree) * (size_t)(nc > 0 ? nc : 1));
    double *kl = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    int nk = 0;
    for (int i = 0; i < nc; ++i) {
        if (i > 0 && cmp128(cs[i].nkey, cs[i - 1].nkey) == 0) continue; /* not the min proposer */
        or_tree nt;
        const or_quartet *q = &qall[(size_t)cs[i].parent * (n - 3) + cs[i].qi];
        apply_nni(&s->front[cs[i].parent], q, cs[i].swap, &nt);
        /* READING: with shape re-optimisation a proposal is scored with its parent's shape
         * (the one its visit found), the shape its inherited lengths were optimised at */
        const or_entry *pe = set_find(&s->vis, cs[i].pkey);
        const double ap = pb->reopt_alpha && pe ? pe->alpha : pb->alpha;
        if (ap != pb->alpha) set_alpha(pb, ap);
        double lp = propose_optimise(pb, &nt, q, cs[i].swap);
        if (ap != pb->alpha) set_alpha(pb, pb->alpha);
        s->n_scored++;
        or_entry *e = set_insert(&s->vis, cs[i].nkey);
        int keepit = lp >= lmax0 - T;
        entry_fill(e, &nt, OR_REJECTED, lp, lp, s->round);
        e->alpha = ap;
        memcpy(e->ppkey, cs[i].pkey, sizeof e->ppkey);
        memcpy(e->psplit, cs[i].split, sizeof e->psplit);
        e->pswap = cs[i].swap;
        if (keepit) { kept[nk] = nt; kl[nk] = lp; ++nk; }
    }
    double lmax = lmax0;
    double *fl = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    double *fa = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    for (int i = 0; i < nk; ++i) {
        fl[i] = visit_optimise(pb, &kept[i], &fa[i]);
        if (fl[i] > lmax) lmax = fl[i];
    }
    s->lmax = lmax;
    s->n_kept += nk;
    int nf = 0;
    or_tree *nfront = (or_tree *)malloc(sizeof(or_tree) * (size_t)(nk > 0 ? nk : 1));
    for (int i = 0; i < nk; ++i) {
        uint64_t k[2];
        tree_key(&kept[i], k);
        or_entry *e = set_find(&s->vis, k);
        if (!entry_same_splits(e, &kept[i])) s->vis.collision = 1;
        free(e->edges); free(e->lengths);
        e->edges = (int32_t *)malloc(sizeof(int32_t) * 2 * (2 * n - 3));
        e->lengths = (double *)malloc(sizeof(double) * (2 * n - 3));
        tree_to_edges(&kept[i], e->edges, e->lengths);
        e->lnl = fl[i];
        e->alpha = fa[i];
        if (fl[i] >= lmax - T) { e->status = OR_GOOD; nfront[nf++] = kept[i]; s->n_good++; }
        else e->status = OR_BAD;
    }
    qsort(nfront, nf, sizeof(or_tree), tree_cmp_key);
    free(s->front);
    s->front = nfront; s->nfront = nf;
    free(cs); free(qall); free(kept); free(kl); free(fl); free(fa);
    return nf;
}

int or_search_run(or_problem *pb, or_search *s, int max_rounds)
{
    int r = 0;
    while (s->nfront > 0 && r < max_rounds) { or_search_round(pb, s); ++r; }
    return r;
}

double or_search_lmax(const or_search *s) { return s->lmax; }
int or_search_frontier(const or_search *s) { return s->nfront; }
size_t or_search_count(const or_search *s) { return s->vis.cnt; }
int or_search_collision(const or_search *s) { return s->vis.collision; }
long or_search_stat(const or_search *s, int which)
{
    return which == 0 ? s->n_scored : which == 1 ? s->n_kept : which == 2 ? s->n_good : s->round;
}

/* Frontier trees (edges + lengths), sorted by key. */
int or_search_frontier_trees(const or_search *s, int32_t *edges, double *lengths)
{
    int n = s->vis.n, ne = 2 * n - 3;
    for (int i = 0; i < s->nfront; ++i)
        tree_to_edges(&s->front[i], edges + (size_t)i * 2 * ne, lengths + (size_t)i * ne);
    return s->nfront;
}

/* Dump: keys [cnt][2], status, lnL, proposal lnL, round; optionally the
 * stored trees (edges [cnt][2n-3][2], lengths [cnt][2n-3]). */
size_t or_search_dump(const or_search *s, uint64_t *keys, int32_t *status, double *lnl, double *plnl,
                      int32_t *round, int32_t *edges, double *lengths)
{
    int n = s->vis.n, ne = 2 * n - 3;
    size_t k = 0;
    for (size_t i = 0; i < s->vis.cap; ++i) {
        const or_entry *e = &s->vis.e[i];
        if (!e->status) continue;
        keys[2 * k] = e->key[0]; keys[2 * k + 1] = e->key[1];
        status[k] = e->status; lnl[k] = e->lnl; plnl[k] = e->plnl; round[k] = e->round;
        if (edges) memcpy(edges + (size_t)k * 2 * ne, e->edges, sizeof(int32_t) * 2 * ne);
        if (lengths) memcpy(lengths + (size_t)k * ne, e->lengths, sizeof(double) * ne);
        ++k;
    }
    return k;
}

/* The winning proposer of every entry, in or_search_dump's order: parent key
 * [cnt][2], split of the rearranged edge [cnt][2] (both low word first) and
 * swap (-1 for trees that were not proposed: starts, given frontiers). */
size_t or_search_proposers(const or_search *s, uint64_t *pkey, uint64_t *split, int32_t *swap)
{
    size_t k = 0;
    for (size_t i = 0; i < s->vis.cap; ++i) {
        const or_entry *e = &s->vis.e[i];
        if (!e->status) continue;
        pkey[2 * k] = e->ppkey[0]; pkey[2 * k + 1] = e->ppkey[1];
        split[2 * k] = e->psplit[0]; split[2 * k + 1] = e->psplit[1];
        swap[k] = e->pswap;
        ++k;
    }
    return k;
}

void or_search_free(or_search *s)
{
    if (!s) return;
    for (size_t i = 0; i < s->vis.cap; ++i)
        if (s->vis.e[i].status) { free(s->vis.e[i].splits); free(s->vis.e[i].edges); free(s->vis.e[i].lengths); }
    free(s->vis.e); free(s->front); free(s);
}

/* ------------------------------------------------------------------------- */
/* Hill-climb from a start tree (stands in for the paper's RAxML starts).      */
/* ------------------------------------------------------------------------- */
/* Fully optimise; then repeatedly score every NNI neighbour by the proposal
 * optimisation, fully optimise the best (ties: smallest key), and move there
 * if its lnL beats the current one by more than 1e-6; stop otherwise or
 * after max_moves moves.  Edges/lengths are overwritten with the result. */
int or_hill_climb(or_problem *pb, int n, int32_t *edges, double *lengths, int max_moves, double *lnl)
{
    or_tree t;
    if (n != pb->n || tree_from_edges(n, edges, lengths, &t)) return -1;
    double cur = full_optimise(pb, &t, NULL);
    int moves = 0;
    for (; moves < max_moves; ++moves) {
        or_quartet qs[OR_MAXN];
        int nq = quartets(&t, qs);
        double best = -INFINITY; uint64_t bkey[2] = {0, 0}; or_tree bt;
        for (int i = 0; i < nq; ++i)
            for (int sw = 0; sw < 2; ++sw) {
                or_tree nt;
                apply_nni(&t, &qs[i], sw, &nt);
                double lp = propose_optimise(pb, &nt, &qs[i], sw);
                uint64_t k[2];
                tree_key(&nt, k);
                if (lp > best || (lp == best && cmp128(k, bkey) < 0)) {
                    best = lp; bkey[0] = k[0]; bkey[1] = k[1]; bt = nt;
                }
            }
        if (nq == 0) break;
        double fl = full_optimise(pb, &bt, NULL);
        if (!(fl > cur + 1e-6)) break;
        t = bt; cur = fl;
    }
    tree_to_edges(&t, edges, lengths);
    *lnl = cur;
    return moves;
}
