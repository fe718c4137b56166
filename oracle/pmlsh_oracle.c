/*
 * PM-LSH oracle: a plain, slow, FP64 CPU restatement of the PM-LSH query
 * algorithms (Zheng et al., "PM-LSH: a fast and accurate in-memory framework
 * for high-dimensional approximate NN and closest pair search").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Arithmetic conventions (fixed so that a reader can check them by eye):
 *   - every floating-point quantity is FP64; FP32 inputs are widened first;
 *   - sums run sequentially in index order, multiply and add are separate
 *     operations (the file is compiled with -ffp-contract=off);
 *   - ties are broken by the smaller point id (pairs: by (i, j), i < j).
 *
 * Functions and the passage each follows:
 *   orc_splitmix64 ........ SplitMix64 output function (Steele, Lea, Flood,
 *                           OOPSLA 2014), used as a counter-based generator
 *   orc_gen_projection .... Sec. 3.2, Eq. 3: entries of each a_j i.i.d. N(0,1)
 *                           (2-stable), drawn with the Box-Muller transform
 *   orc_chi2_sf/isf ....... Lemma 3 (upper quantile of chi^2(m))
 *   orc_params ............ Eq. 9 and Lemma 5 (beta = 2 alpha2)
 *   orc_budget ............ Algorithm 2 budget |C| >= beta n + k
 *   orc_project ........... Eq. 3, o' = [a_1.o, ..., a_m.o]
 *   orc_rmin_auto ......... Sec. 5.2 "Selecting the radius r of a range query"
 *   orc_knn ............... Algorithm 2, (c,k)-ANN
 *   orc_rcbc .............. Algorithm 1, (r,c)-BC
 *   orc_exact_knn ......... Definition 2 with c = 1 (brute force ground truth)
 *   orc_exact_kcp ......... Definition 4 with c = 1 (nested-loop join, NLJ)
 *   orc_cp_bnb ............ Algorithm 3 (branch and bound): the T pairs nearest
 *                           in the projected space, verified, top k
 *   orc_cp_radius_filter .. Algorithm 4 with FindLCA (Algorithm 5) on a given
 *                           hierarchy of leaves
 *   orc_node_ball ......... node ball (e.RO, e.r) of Sec. 4.1 for the given
 *                           hierarchy
 *   orc_distance_sample ... Sec. 4.2, distance distribution F(x) =
 *                           Pr[||o_i, o_j|| <= x], estimated from sampled
 *                           pairs in the projected space
 *   orc_cost_model ........ Sec. 4.2, node access probability Pr[e] and the
 *                           computation cost CC(range(q, r_q)) of the PM-tree
 *                           cost model, on given node entries
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Counter-based generator: SplitMix64 output function applied to
 * seed + (i+1) * golden-gamma.  Value i of stream `seed`.                   */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sec. 3.2 / Eq. 3: A[j][i], j < m, i < d, row-major, i.i.d. N(0,1).
 * Value pairs (2p, 2p+1) of the stream give u1 in (0,1], u2 in [0,1);
 * Box-Muller gives rad*cos(2 pi u2) then rad*sin(2 pi u2).                  */
void orc_gen_projection(uint64_t seed, int m, int d, double *A)
{
    const double two_pi = 6.283185307179586476925286766559;
    int64_t total = (int64_t)m * d;
    for (int64_t e = 0; e < total; e += 2) {
        uint64_t p = (uint64_t)(e / 2);
        double u1 = ((double)(orc_splitmix64(seed, 2 * p) >> 11) + 1.0) * 0x1.0p-53;
        double u2 = (double)(orc_splitmix64(seed, 2 * p + 1) >> 11) * 0x1.0p-53;
        double rad = sqrt(-2.0 * log(u1));
        A[e] = rad * cos(two_pi * u2);
        if (e + 1 < total) A[e + 1] = rad * sin(two_pi * u2);
    }
}

/* ------------------------------------------------------------------------ */
/* chi^2(m) tail.  Pr[chi^2(m) > x] = Q(m/2, x/2), Q the regularized upper
 * incomplete gamma function.  For y < a+1 the power series of the lower
 * function P(a,y) = y^a e^-y / Gamma(a+1) * sum_n y^n / ((a+1)...(a+n))
 * converges fast; otherwise Q is evaluated from its continued fraction
 * Q(a,y) = y^a e^-y / Gamma(a) * 1/(y+1-a- 1(1-a)/(y+3-a- 2(2-a)/(y+5-a- ...)))
 * with the modified Lentz method.                                           */
static double lower_series(double a, double y)
{
    double term = 1.0 / a, sum = term;
    for (int n = 1; n < 100000; n++) {
        term = term * y / (a + n);
        sum = sum + term;
        if (fabs(term) < fabs(sum) * 1e-17) break;
    }
    return sum * exp(-y + a * log(y) - lgamma(a));
}

static double upper_cfrac(double a, double y)
{
    const double tiny = 1e-300;
    double b = y + 1.0 - a;
    double cc = 1.0 / tiny;
    double dd = 1.0 / b;
    double h = dd;
    for (int i = 1; i < 100000; i++) {
        double an = -i * (i - a);
        b = b + 2.0;
        dd = an * dd + b;
        if (fabs(dd) < tiny) dd = tiny;
        cc = b + an / cc;
        if (fabs(cc) < tiny) cc = tiny;
        dd = 1.0 / dd;
        double delta = dd * cc;
        h = h * delta;
        if (fabs(delta - 1.0) < 1e-17) break;
    }
    return exp(-y + a * log(y) - lgamma(a)) * h;
}

/* Pr[chi^2(m) > x]  (Lemma 1 / Lemma 3). */
double orc_chi2_sf(double x, int m)
{
    if (x <= 0.0) return 1.0;
    double a = 0.5 * m, y = 0.5 * x;
    if (y < a + 1.0) return 1.0 - lower_series(a, y);
    return upper_cfrac(a, y);
}

/* Lemma 3: the upper quantile chi^2_alpha(m), i.e. the x with
 * Pr[chi^2(m) > x] = alpha, found by bisection to adjacent doubles.         */
double orc_chi2_isf(double alpha, int m)
{
    if (!(alpha > 0.0 && alpha < 1.0) || m < 1) return NAN;
    double lo = 0.0, hi = (double)m + 1.0;
    while (orc_chi2_sf(hi, m) > alpha) hi = hi * 2.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_chi2_sf(mid, m) > alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Eq. 9: t^2 = chi^2_{alpha1}(m) and t^2 = c^2 chi^2_{1-alpha2}(m).
 * The second line says Pr[chi^2(m) > t^2/c^2] = 1 - alpha2, hence
 * alpha2 = Pr[chi^2(m) <= t^2/c^2].  Lemma 5 sets beta = 2 alpha2.          */
void orc_params(int m, double c, double alpha1, double *t, double *alpha2, double *beta_eq9)
{
    double t2 = orc_chi2_isf(alpha1, m);
    double a2 = 1.0 - orc_chi2_sf(t2 / (c * c), m);
    if (t) *t = sqrt(t2);
    if (alpha2) *alpha2 = a2;
    if (beta_eq9) *beta_eq9 = 2.0 * a2;
}

/* Algorithm 2 stops once |C| >= beta n + k; with |C| an integer that is
 * |C| >= ceil(beta n) + k.  The 1e-9 absorbs representation error of beta n. */
int64_t orc_budget(int64_t n, double beta, int64_t k)
{
    return (int64_t)ceil(beta * (double)n - 1e-9) + k;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3: o'[j] = a_j . o, with the FP32 matrix A32 [m][d] and FP32 points. */
void orc_project(const float *X, int64_t n, int d, const float *A32, int m, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        const float *x = X + p * (int64_t)d;
        for (int j = 0; j < m; j++) {
            const float *a = A32 + (int64_t)j * d;
            double s = 0.0;
            for (int i = 0; i < d; i++) s = s + (double)a[i] * (double)x[i];
            out[p * m + j] = s;
        }
    }
}

/* ||o1, o2|| in the original space (Sec. 2, Euclidean distance). */
static double dist64(const float *x, const float *y, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; i++) {
        double diff = (double)x[i] - (double)y[i];
        s = s + diff * diff;
    }
    return sqrt(s);
}

/* ||o1', o2'|| in the projected space (Sec. 3.2, r' = sqrt(sum rho_i^2)). */
static double pdist64(const double *a, const double *b, int m)
{
    double s = 0.0;
    for (int j = 0; j < m; j++) {
        double diff = a[j] - b[j];
        s = s + diff * diff;
    }
    return sqrt(s);
}

double orc_dist(const float *x, const float *y, int d) { return dist64(x, y, d); }
double orc_pdist(const double *a, const double *b, int m) { return pdist64(a, b, m); }

/* ------------------------------------------------------------------------ */
typedef struct { double key; int64_t id; } keyed;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

static int cmp_i64(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return (a > b) - (a < b);
}

static int cmp_double(const void *pa, const void *pb)
{
    double a = *(const double *)pa, b = *(const double *)pb;
    return (a > b) - (a < b);
}

/* Sec. 5.2, selection of r_min.  F is the distance distribution of the data
 * set; the paper takes r with n F(r) = beta n + k and an r_min slightly
 * below it.  Reading used here: F is the empirical CDF of `npairs` sampled
 * point pairs (indices from the counter generator stream `seed`), and the
 * lower quantile rstar at p = min(1, (beta n + k)/n), and r_min = rstar / c (one growth
 * step below rstar).  If rstar is 0 the smallest positive sample is used, and 1.0
 * if every sample is 0.                                                     */
double orc_rmin_auto(const float *X, int64_t n, int d, double beta, int64_t k, double c,
                     uint64_t seed, int64_t npairs)
{
    if (n < 2 || npairs < 1) return 1.0;
    double *v = (double *)malloc(sizeof(double) * (size_t)npairs);
    for (int64_t s = 0; s < npairs; s++) {
        int64_t i = (int64_t)(orc_splitmix64(seed, 2 * (uint64_t)s) % (uint64_t)n);
        int64_t j = (int64_t)(orc_splitmix64(seed, 2 * (uint64_t)s + 1) % (uint64_t)n);
        if (j == i) j = (j + 1) % n;
        v[s] = dist64(X + i * (int64_t)d, X + j * (int64_t)d, d);
    }
    qsort(v, (size_t)npairs, sizeof(double), cmp_double);
    double p = (beta * (double)n + (double)k) / (double)n;
    if (p > 1.0) p = 1.0;
    int64_t rank = (int64_t)ceil(p * (double)npairs - 1e-9);
    if (rank < 1) rank = 1;
    if (rank > npairs) rank = npairs;
    double rstar = v[rank - 1];
    if (!(rstar > 0.0)) {
        rstar = 0.0;
        for (int64_t s = 0; s < npairs; s++) if (v[s] > 0.0) { rstar = v[s]; break; }
        if (!(rstar > 0.0)) { free(v); return 1.0; }
    }
    free(v);
    return rstar / c;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, (c,k)-ANN, for queries Q [nq][d].
 *
 * Inputs follow the algorithm's parameter list: r_min (per query), beta via
 * the budget B = ceil(beta n) + k, n, t, c, k.  Oproj [n][m] is the data set
 * in the projected space (orc_project) and A32 the projection.
 *
 * Readings taken where the listing is open:
 *   - the inner "while |C| < beta n + k: add a node of B(q', t r)" depends on
 *     the tree's visiting order; here C_i is the range set S_i = {o :
 *     ||o', q'|| <= t r_i} (closed ball) and, when |S_i| >= B, the B members
 *     of S_i with the smallest (||o', q'||, id) -- then stop rule 2 returns;
 *   - stop rule 1 (|{p in C : ||p,q|| <= c r}| >= k) sits at the loop top,
 *     after r <- c r, as printed (stop_rule = 0, "literal"); stop_rule = 1
 *     tests it right after the range query with the same r (the form of
 *     Algorithm 1 and of the proof of Theorem 1);
 *   - once S_i holds every point the candidate set can no longer change, so
 *     the top-k is returned at once (reported as rule 3); the literal loop
 *     would return the same top-k after more radius growth.
 *
 * Outputs per query: the k ids and FP64 distances sorted by (dist, id), the
 * number of range queries run, the rule that stopped (1, 2 or 3), |C| and
 * the final r.                                                              */
static void knn_one(const float *X, const double *Oproj, int64_t n, int d, int m,
                    const float *q, const double *qp, int64_t k, double c, double t,
                    int64_t B, double rmin, int stop_rule,
                    double *pd, double *dist, keyed *buf,
                    int64_t *ids_out, double *d_out, int32_t *rounds_out, int32_t *rule_out,
                    int64_t *ncand_out, double *r_out)
{
    for (int64_t p = 0; p < n; p++) {
        pd[p] = pdist64(Oproj + p * m, qp, m);
        dist[p] = -1.0; /* not verified yet */
    }
    int64_t csize = 0;  /* |C| */
    double r = rmin;
    int rounds = 0, rule = 0;
    for (;;) {
        if (stop_rule == 0 && csize > 0) {
            int64_t cnt = 0;
            for (int64_t p = 0; p < n; p++)
                if (dist[p] >= 0.0 && dist[p] <= c * r) cnt++;
            if (cnt >= k) { rule = 1; break; }
        }
        double R = t * r;
        int64_t ssize = 0;
        for (int64_t p = 0; p < n; p++)
            if (pd[p] <= R) buf[ssize++] = (keyed){pd[p], p};
        rounds++;
        if (ssize >= B) {
            qsort(buf, (size_t)ssize, sizeof(keyed), cmp_keyed);
            for (int64_t e = 0; e < B; e++) {
                int64_t p = buf[e].id;
                if (dist[p] < 0.0) dist[p] = dist64(X + p * (int64_t)d, q, d);
            }
            for (int64_t e = B; e < ssize; e++) dist[buf[e].id] = -1.0;
            csize = B;
            rule = 2;
            break;
        }
        for (int64_t e = 0; e < ssize; e++) {
            int64_t p = buf[e].id;
            if (dist[p] < 0.0) dist[p] = dist64(X + p * (int64_t)d, q, d);
        }
        csize = ssize;
        if (ssize == n) { rule = 3; break; }
        if (stop_rule == 1) {
            int64_t cnt = 0;
            for (int64_t p = 0; p < n; p++)
                if (dist[p] >= 0.0 && dist[p] <= c * r) cnt++;
            if (cnt >= k) { rule = 1; break; }
        }
        r = c * r;
    }
    int64_t nc = 0;
    for (int64_t p = 0; p < n; p++)
        if (dist[p] >= 0.0) buf[nc++] = (keyed){dist[p], p};
    qsort(buf, (size_t)nc, sizeof(keyed), cmp_keyed);
    for (int64_t e = 0; e < k; e++) {
        ids_out[e] = e < nc ? buf[e].id : -1;
        d_out[e] = e < nc ? buf[e].key : INFINITY;
    }
    *rounds_out = rounds;
    *rule_out = rule;
    *ncand_out = csize;
    *r_out = r;
}

int orc_knn(const float *X, const double *Oproj, int64_t n, int d, const float *A32, int m,
            const float *Q, int64_t nq, int64_t k, double c, double t, int64_t B,
            const double *rmin, int stop_rule,
            int64_t *out_ids, double *out_dists, int32_t *out_rounds, int32_t *out_rule,
            int64_t *out_ncand, double *out_r)
{
    if (k < 1 || k > n || !(c > 1.0) || m < 1 || d < 1 || B < k) return 1;
    int bad = 0;
#pragma omp parallel
    {
        double *pd = (double *)malloc(sizeof(double) * (size_t)n);
        double *dist = (double *)malloc(sizeof(double) * (size_t)n);
        keyed *buf = (keyed *)malloc(sizeof(keyed) * (size_t)n);
        double qp[64];
        if (!pd || !dist || !buf || m > 64) bad = 1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; qi++) {
            if (bad) continue;
            const float *q = Q + qi * (int64_t)d;
            for (int j = 0; j < m; j++) {
                const float *a = A32 + (int64_t)j * d;
                double s = 0.0;
                for (int i = 0; i < d; i++) s = s + (double)a[i] * (double)q[i];
                qp[j] = s;
            }
            knn_one(X, Oproj, n, d, m, q, qp, k, c, t, B, rmin[qi], stop_rule, pd, dist, buf,
                    out_ids + qi * k, out_dists + qi * k, out_rounds + qi, out_rule + qi,
                    out_ncand + qi, out_r + qi);
        }
        free(pd); free(dist); free(buf);
    }
    return bad ? 2 : 0;
}

/* Algorithm 1, (r,c)-BC for one radius r: C = range(q', t r); if
 * |C| >= beta n + 1 (Bbc = ceil(beta n) + 1) or some p in C has
 * ||p,q|| <= c r, return the point of C closest to q (ties by id), else -1. */
int orc_rcbc(const float *X, const double *Oproj, int64_t n, int d, const float *A32, int m,
             const float *Q, int64_t nq, double r, double c, double t, int64_t Bbc,
             int64_t *out_id, double *out_dist, int64_t *out_ncand)
{
    for (int64_t qi = 0; qi < nq; qi++) {
        const float *q = Q + qi * (int64_t)d;
        double qp[64];
        if (m > 64) return 1;
        for (int j = 0; j < m; j++) {
            const float *a = A32 + (int64_t)j * d;
            double s = 0.0;
            for (int i = 0; i < d; i++) s = s + (double)a[i] * (double)q[i];
            qp[j] = s;
        }
        double R = t * r, best = INFINITY;
        int64_t bestid = -1, cs = 0, within = 0;
        for (int64_t p = 0; p < n; p++) {
            if (pdist64(Oproj + p * m, qp, m) <= R) {
                cs++;
                double dd = dist64(X + p * (int64_t)d, q, d);
                if (dd <= c * r) within++;
                if (dd < best || (dd == best && p < bestid)) { best = dd; bestid = p; }
            }
        }
        out_ncand[qi] = cs;
        if (cs >= Bbc || within >= 1) { out_id[qi] = bestid; out_dist[qi] = best; }
        else { out_id[qi] = -1; out_dist[qi] = INFINITY; }
    }
    return 0;
}

/* Definition 2 with c = 1: exact k nearest neighbours by linear scan. */
int orc_exact_knn(const float *X, int64_t n, int d, const float *Q, int64_t nq, int64_t k,
                  int64_t *out_ids, double *out_dists)
{
    if (k < 1 || k > n) return 1;
#pragma omp parallel
    {
        keyed *buf = (keyed *)malloc(sizeof(keyed) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t qi = 0; qi < nq; qi++) {
            const float *q = Q + qi * (int64_t)d;
            for (int64_t p = 0; p < n; p++) buf[p] = (keyed){dist64(X + p * (int64_t)d, q, d), p};
            qsort(buf, (size_t)n, sizeof(keyed), cmp_keyed);
            for (int64_t e = 0; e < k; e++) {
                out_ids[qi * k + e] = buf[e].id;
                out_dists[qi * k + e] = buf[e].key;
            }
        }
        free(buf);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Closest pairs.  A pair is kept as (dist, i, j) with i < j (original ids). */
typedef struct { double key; int64_t i, j; } keyed_pair;

static int cmp_pair(const void *pa, const void *pb)
{
    const keyed_pair *a = (const keyed_pair *)pa, *b = (const keyed_pair *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->i != b->i) return (a->i > b->i) - (a->i < b->i);
    return (a->j > b->j) - (a->j < b->j);
}

/* Running top-k of pairs, kept sorted by (dist, i, j). */
typedef struct { keyed_pair *v; int64_t n, k; } topk_pairs;

static void topk_push(topk_pairs *t, keyed_pair e)
{
    if (t->n == t->k && cmp_pair(&e, &t->v[t->k - 1]) >= 0) return;
    int64_t pos = t->n < t->k ? t->n : t->k - 1;
    if (t->n < t->k) t->n++;
    while (pos > 0 && cmp_pair(&e, &t->v[pos - 1]) < 0) { t->v[pos] = t->v[pos - 1]; pos--; }
    t->v[pos] = e;
}

static keyed_pair make_pair(double key, int64_t a, int64_t b)
{
    keyed_pair e;
    e.key = key;
    e.i = a < b ? a : b;
    e.j = a < b ? b : a;
    return e;
}

/* Sec. 6.1, Algorithm 3 (branch and bound), its result stated directly:
 * C = the T pairs with the smallest projected distance ||o1',o2'|| (ties by
 * (i, j)).  The best-first search over node pairs ends with exactly these
 * pairs: Mindist(e1, e2) bounds every pair under (e1, e2) from below, so a
 * node pair is left out only when none of its pairs can beat the T-th
 * distance.  Each pair of C is verified by its original distance and the k
 * smallest by (distance, i, j) are returned.  Reading: |C| = T (the text of
 * Sec. 6.1 and its example keep T pairs after the self-joins; the first
 * line of the listing prints k).  T larger than n(n-1)/2 means every pair. */
int orc_cp_bnb(const float *X, const double *Oproj, int64_t n, int d, int m, int64_t T, int64_t k,
               int64_t *out_pairs, double *out_dists)
{
    const int64_t P = n * (n - 1) / 2;
    if (n < 2 || k < 1 || T < k || k > P) return 1;
    if (T > P) T = P;
    topk_pairs c = {(keyed_pair *)malloc(sizeof(keyed_pair) * (size_t)T), 0, T};
    topk_pairs r = {(keyed_pair *)malloc(sizeof(keyed_pair) * (size_t)k), 0, k};
    if (!c.v || !r.v) { free(c.v); free(r.v); return 2; }
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++)
            topk_push(&c, make_pair(pdist64(Oproj + a * (int64_t)m, Oproj + b * (int64_t)m, m), a, b));
    for (int64_t e = 0; e < c.n; e++) {
        const int64_t i = c.v[e].i, j = c.v[e].j;
        topk_push(&r, make_pair(dist64(X + i * (int64_t)d, X + j * (int64_t)d, d), i, j));
    }
    for (int64_t e = 0; e < k; e++) {
        out_pairs[2 * e] = r.v[e].i;
        out_pairs[2 * e + 1] = r.v[e].j;
        out_dists[e] = r.v[e].key;
    }
    free(c.v);
    free(r.v);
    return 0;
}

/* Definition 4 with c = 1: exact k closest pairs (nested-loop join). */
int orc_exact_kcp(const float *X, int64_t n, int d, int64_t k, int64_t *out_pairs, double *out_dists)
{
    if (n < 2 || k < 1 || k > n * (n - 1) / 2) return 1;
    topk_pairs t = {(keyed_pair *)malloc(sizeof(keyed_pair) * (size_t)k), 0, k};
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++)
            topk_push(&t, make_pair(dist64(X + a * (int64_t)d, X + b * (int64_t)d, d), a, b));
    for (int64_t e = 0; e < k; e++) {
        out_pairs[2 * e] = t.v[e].i;
        out_pairs[2 * e + 1] = t.v[e].j;
        out_dists[e] = t.v[e].key;
    }
    free(t.v);
    return 0;
}

/* Node ball of Sec. 4.1 (e.RO, e.r) for the points at positions [lo, hi)
 * of `perm`: RO is the midpoint of the FP64 bounding box of the projected
 * points (any centre gives a valid covering ball; this one does not depend on
 * the order in which points are visited) and r the largest distance from RO. */
void orc_node_ball(const double *Oproj, int m, const int32_t *perm, int64_t lo, int64_t hi,
                   double *ro, double *rad)
{
    double mn[64], mx[64];
    for (int j = 0; j < m; j++) { mn[j] = INFINITY; mx[j] = -INFINITY; }
    for (int64_t e = lo; e < hi; e++) {
        const double *o = Oproj + (int64_t)perm[e] * m;
        for (int j = 0; j < m; j++) {
            if (o[j] < mn[j]) mn[j] = o[j];
            if (o[j] > mx[j]) mx[j] = o[j];
        }
    }
    for (int j = 0; j < m; j++) ro[j] = 0.5 * (mn[j] + mx[j]);
    double r = 0.0;
    for (int64_t e = lo; e < hi; e++) {
        double v = pdist64(Oproj + (int64_t)perm[e] * m, ro, m);
        if (v > r) r = v;
    }
    *rad = r;
}

/* Algorithm 5, FindLCA(e, R, A): an inner node with e.r < R is appended to
 * A; otherwise its children are visited.  Leaf nodes are never appended.    */
static void find_lca(int64_t e, double R, const int32_t *left, const int32_t *right,
                     const double *nrad, int64_t *A, int64_t *na)
{
    if (left[e] < 0) return; /* not an inner node */
    if (nrad[e] < R) { A[(*na)++] = e; return; }
    find_lca(left[e], R, left, right, nrad, A, na);
    find_lca(right[e], R, left, right, nrad, A, na);
}

static const double *g_sort_rad;
static int cmp_node(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (g_sort_rad[a] < g_sort_rad[b]) return -1;
    if (g_sort_rad[a] > g_sort_rad[b]) return 1;
    return (a > b) - (a < b);
}

/* Algorithm 4, radius filtering, on a given hierarchy.
 *
 * Hierarchy (data, not recomputed): perm [n] lists point ids in leaf order,
 * leaf_off [L+1] gives each leaf's positions, and nodes 0..nn-1 (node 0 the
 * root) have a leaf range [nlo, nhi) and children (nleft, nright), -1 for a
 * leaf node.  Node balls come from orc_node_ball.
 *
 * Steps: self-join every leaf and verify every pair (count = their number,
 * ub = k-th smallest distance, +inf if fewer than k); R = gamma t ub;
 * A = FindLCA(root, R) sorted by (radius, node id); for each node, the
 * candidate pairs are the pairs of its subtree that lie in different leaves
 * with ||o1', o2'|| < t ub (ub as it stands when the node starts); if count
 * plus their number exceeds T, only the T + 1 - count smallest by
 * (||o1',o2'||, i, j) are kept; they are verified and count grows; after the
 * node ub becomes the current k-th distance; the loop ends once count > T.
 * (Reading: ub is frozen inside a node, which makes the result independent
 * of the order in which a node's pairs are visited.)
 * Returns the k closest verified pairs sorted by (dist, i, j).              */
int orc_cp_radius_filter(const float *X, const double *Oproj, int64_t n, int d, int m,
                         const int32_t *perm, const int64_t *leaf_off, int64_t L,
                         const int64_t *nlo, const int64_t *nhi, const int32_t *nleft,
                         const int32_t *nright, int64_t nn,
                         int64_t k, double t, double gamma, int64_t T,
                         int64_t *out_pairs, double *out_dists, int64_t *out_count,
                         double *out_ub_self, int64_t *out_nodes, int64_t *out_nodes_done)
{
    if (n < 2 || k < 1 || k > n * (n - 1) / 2 || m > 64) return 1;
    topk_pairs tk = {(keyed_pair *)malloc(sizeof(keyed_pair) * (size_t)k), 0, k};
    int64_t count = 0;
    /* self-join of each leaf */
    for (int64_t l = 0; l < L; l++)
        for (int64_t a = leaf_off[l]; a < leaf_off[l + 1]; a++)
            for (int64_t b = a + 1; b < leaf_off[l + 1]; b++) {
                int64_t ia = perm[a], ib = perm[b];
                topk_push(&tk, make_pair(dist64(X + ia * (int64_t)d, X + ib * (int64_t)d, d), ia, ib));
                count++;
            }
    double ub = tk.n == k ? tk.v[k - 1].key : INFINITY;
    *out_ub_self = ub;
    double R = gamma * t * ub;
    /* node balls */
    double *nrad = (double *)malloc(sizeof(double) * (size_t)nn);
    double ro[64];
    for (int64_t e = 0; e < nn; e++)
        orc_node_ball(Oproj, m, perm, leaf_off[nlo[e]], leaf_off[nhi[e]], ro, &nrad[e]);
    int64_t *A = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t na = 0;
    find_lca(0, R, nleft, nright, nrad, A, &na);
    g_sort_rad = nrad;
    qsort(A, (size_t)na, sizeof(int64_t), cmp_node);
    *out_nodes = na;
    int64_t done = 0;
    /* leaf index of each position */
    int64_t *leaf_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t l = 0; l < L; l++)
        for (int64_t a = leaf_off[l]; a < leaf_off[l + 1]; a++) leaf_of[a] = l;
    for (int64_t ai = 0; ai < na && count <= T; ai++) {
        int64_t e = A[ai];
        int64_t lo = leaf_off[nlo[e]], hi = leaf_off[nhi[e]];
        double thr = t * ub;
        int64_t cap = 1024, nc = 0;
        keyed_pair *cand = (keyed_pair *)malloc(sizeof(keyed_pair) * (size_t)cap);
        for (int64_t a = lo; a < hi; a++)
            for (int64_t b = a + 1; b < hi; b++) {
                if (leaf_of[a] == leaf_of[b]) continue;
                int64_t ia = perm[a], ib = perm[b];
                double pdv = pdist64(Oproj + ia * m, Oproj + ib * m, m);
                if (pdv < thr) {
                    if (nc == cap) { cap *= 2; cand = (keyed_pair *)realloc(cand, sizeof(keyed_pair) * (size_t)cap); }
                    cand[nc++] = make_pair(pdv, ia, ib);
                }
            }
        int64_t keep = nc;
        if (count + nc > T) {
            keep = T + 1 - count;
            qsort(cand, (size_t)nc, sizeof(keyed_pair), cmp_pair);
        }
        for (int64_t c2 = 0; c2 < keep; c2++) {
            int64_t ia = cand[c2].i, ib = cand[c2].j;
            topk_push(&tk, make_pair(dist64(X + ia * (int64_t)d, X + ib * (int64_t)d, d), ia, ib));
        }
        count += keep;
        free(cand);
        ub = tk.n == k ? tk.v[k - 1].key : INFINITY;
        done++;
    }
    *out_nodes_done = done;
    *out_count = count;
    for (int64_t e = 0; e < k; e++) {
        out_pairs[2 * e] = e < tk.n ? tk.v[e].i : -1;
        out_pairs[2 * e + 1] = e < tk.n ? tk.v[e].j : -1;
        out_dists[e] = e < tk.n ? tk.v[e].key : INFINITY;
    }
    free(leaf_of); free(A); free(nrad); free(tk.v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Setting of gamma for radius filtering (Sec. 6.3, "Determining the Setting
 * of gamma"; Sec. 7.1 fixes Pr(gamma) = 0.85).                              */

/* The sample of Sec. 6.3 and Sec. 7.2 ("we randomly sample n' points"):
 * n' = min(nprime, n) distinct ids drawn by a partial Fisher-Yates shuffle of
 * 0..n-1 whose i-th step swaps entry i with entry i + (v_i mod (n - i)), v_i
 * value i of the counter-based SplitMix64 stream `seed`; the first n' entries,
 * sorted ascending, are the sample.  Returns n'.                            */
int64_t orc_gamma_sample(int64_t n, int64_t nprime, uint64_t seed, int64_t *ids)
{
    if (n < 1 || nprime < 1) return 0;
    int64_t np = nprime < n ? nprime : n;
    int64_t *all = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; i++) all[i] = i;
    if (np < n)
        for (int64_t i = 0; i < np; i++) {
            int64_t j = i + (int64_t)(orc_splitmix64(seed, (uint64_t)i) % (uint64_t)(n - i));
            int64_t t = all[i]; all[i] = all[j]; all[j] = t;
        }
    for (int64_t i = 0; i < np; i++) ids[i] = all[i];
    free(all);
    qsort(ids, (size_t)np, sizeof(int64_t), cmp_i64);
    return np;
}

/* gamma of Sec. 6.3 over the pairs of a point set with a given hierarchy (the
 * PM-tree built on the sample; data, not recomputed).  For each pair of
 * points, the ratio R / ||o1', o2'|| with R the radius (orc_node_ball) of
 * their lowest common node: descending from the root while both points lie
 * in the same child; two points of one leaf have that leaf as their lowest
 * common node.  For coincident projections the ratio is 0 when R = 0 (the
 * node is found for every positive filter radius) and +inf otherwise.
 * gamma is the lower empirical quantile at probability pr of the
 * n (n - 1) / 2 ratios: the smallest ratio with at least pr of the ratios at
 * or below it (rank ceil(pr N - 1e-9), at least 1).  Oproj is indexed by
 * point id, perm maps positions to ids as in orc_cp_radius_filter.
 * Returns 0, or 1 for fewer than 2 points or pr outside (0, 1].           */
int orc_gamma_calibrate(const double *Oproj, int64_t n, int m, const int32_t *perm,
                        const int64_t *leaf_off, int64_t L, const int64_t *nlo, const int64_t *nhi,
                        const int32_t *nleft, const int32_t *nright, int64_t nn, double pr, double *gamma)
{
    if (n < 2 || !(pr > 0.0 && pr <= 1.0) || m > 64 || nn < 1) return 1;
    double *nrad = (double *)malloc(sizeof(double) * (size_t)nn);
    double ro[64];
    for (int64_t e = 0; e < nn; e++)
        orc_node_ball(Oproj, m, perm, leaf_off[nlo[e]], leaf_off[nhi[e]], ro, &nrad[e]);
    int64_t *leaf_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t l = 0; l < L; l++)
        for (int64_t a = leaf_off[l]; a < leaf_off[l + 1]; a++) leaf_of[a] = l;
    const int64_t N = n * (n - 1) / 2;
    double *ratio = (double *)malloc(sizeof(double) * (size_t)N);
    int64_t c = 0;
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++) {
            const int64_t la = leaf_of[a], lb = leaf_of[b];
            int64_t e = 0;
            while (nleft[e] >= 0) {
                const int64_t x = nleft[e], y = nright[e];
                if (la >= nlo[x] && la < nhi[x] && lb >= nlo[x] && lb < nhi[x]) e = x;
                else if (la >= nlo[y] && la < nhi[y] && lb >= nlo[y] && lb < nhi[y]) e = y;
                else break;
            }
            const double R = nrad[e];
            const double dv = pdist64(Oproj + (int64_t)perm[a] * m, Oproj + (int64_t)perm[b] * m, m);
            ratio[c++] = dv > 0.0 ? R / dv : (R > 0.0 ? INFINITY : 0.0);
        }
    qsort(ratio, (size_t)N, sizeof(double), cmp_double);
    int64_t rank = (int64_t)ceil(pr * (double)N - 1e-9);
    if (rank < 1) rank = 1;
    if (rank > N) rank = N;
    *gamma = ratio[rank - 1];
    free(ratio); free(leaf_of); free(nrad);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cost model of the PM-tree (Sec. 4.2)                                      */

/* F(x) = Pr[||o_i, o_j|| <= x] over pairs of D, in the projected space where
 * the tree lives.  Reading used here: `npairs` pairs drawn from the counter
 * generator stream `seed` exactly as orc_rmin_auto draws them (i from counter
 * 2s, j from 2s + 1, both mod n, j = i moved to i + 1 mod n), the FP64
 * projected distance of each, sorted ascending.  The estimate of F is the
 * empirical CDF of this sample.                                             */
void orc_distance_sample(const double *Oproj, int64_t n, int m, uint64_t seed, int64_t npairs,
                         double *out_sorted)
{
    for (int64_t s = 0; s < npairs; s++) {
        int64_t i = (int64_t)(orc_splitmix64(seed, 2 * (uint64_t)s) % (uint64_t)n);
        int64_t j = (int64_t)(orc_splitmix64(seed, 2 * (uint64_t)s + 1) % (uint64_t)n);
        if (j == i) j = (j + 1) % n;
        out_sorted[s] = pdist64(Oproj + i * (int64_t)m, Oproj + j * (int64_t)m, m);
    }
    qsort(out_sorted, (size_t)npairs, sizeof(double), cmp_double);
}

/* Empirical CDF: the fraction of the sorted sample F[0..nF) that is <= x.   */
static double ecdf(const double *F, int64_t nF, double x)
{
    int64_t lo = 0, hi = nF;   /* first index with F[idx] > x */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (F[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return (double)lo / (double)nF;
}

/* A node e is accessed by range(q, r_q) iff ||q, e.RO|| <= e.r + r_q and,
 * for every pivot p_i, ||q, p_i|| - r_q <= e.HR[i].max and
 * ||q, p_i|| + r_q >= e.HR[i].min.  With F standing for the distribution of
 * each of those query distances:
 *   Pr[e] = F(e.r + r_q) * prod_i (F(e.HR[i].max + r_q) - F(e.HR[i].min - r_q)),
 *   CC    = sum_e N(e) Pr[e].
 * Nodes are given by their entry counts N(e) [nn], radii [nn] and rings
 * hr_min, hr_max [nn][s].  Returns CC; *expected_nodes = sum_e Pr[e].        */
double orc_cost_model(const double *F, int64_t nF, int64_t nn, const int64_t *count, const double *radius,
                      int s, const double *hr_min, const double *hr_max, double rq, double *expected_nodes)
{
    double cc = 0.0, en = 0.0;
    for (int64_t e = 0; e < nn; e++) {
        double pr = ecdf(F, nF, radius[e] + rq);
        for (int i = 0; i < s; i++) {
            double hi = ecdf(F, nF, hr_max[e * s + i] + rq);
            double lo = ecdf(F, nF, hr_min[e * s + i] - rq);
            pr = pr * (hi - lo);
        }
        cc = cc + (double)count[e] * pr;
        en = en + pr;
    }
    if (expected_nodes) *expected_nodes = en;
    return cc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
