/*
 * pmlsh.h -- C ABI of the GB300 PM-LSH library (libpmlsh.so).
 *
 * PM-LSH (Zheng, Zhao, Weng, Hung, Liu, Jensen) answers (c,k)-approximate
 * nearest-neighbour queries (Definition 2) and (c,k)-approximate closest-pair
 * queries (Definition 4) over a data set D of n points in R^d by projecting
 * every point onto m Gaussian directions (Sec. 3.2, Eq. 3), running range
 * queries in the projected space whose radius t*r comes from a chi-square
 * confidence interval (Lemma 3, Eq. 9) and grows by c per round
 * (Algorithm 2), and verifying candidates by their exact distance.
 *
 * Conventions shared by every entry point
 *   - Status codes only: no call aborts, throws across the ABI or traps on
 *     the device.  On failure the call returns a code != PMLSH_OK and
 *     pmlsh_last_error() describes it (thread-local string).
 *   - Pointers may be host or device memory; the library asks the CUDA
 *     runtime which kind each one is.  The caller owns every buffer it
 *     passes; the library copies what it keeps.  Results written to host
 *     buffers are complete when the call returns; results written to device
 *     buffers are complete when `stream` reaches the end of the work the
 *     call enqueued (the call still synchronises internally once per round
 *     of Algorithm 2 to read small per-query decisions).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Distances are Euclidean (not squared).  Results are sorted by
 *     ascending distance, ties by smaller id; closest pairs are (i, j) with
 *     i < j and ties by (i, j).
 *   - Floating-point decisions (range membership, the budget cut, the k-th
 *     neighbour, the stop rules) are taken on FP32 values with a proven
 *     error bound and re-taken in FP64 wherever the FP32 value lies inside
 *     that bound, so they equal the decisions of an FP64 evaluation of the
 *     same formulas (sequential sums, separate multiply and add).
 *   - Not thread-safe per index, except through the pmlsh_serve_* API.
 */
#ifndef PMLSH_H
#define PMLSH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMLSH_OK = 0,
    PMLSH_EINVAL = 1,     /* an argument is out of range or NULL */
    PMLSH_ENOMEM = 2,     /* device or host allocation failed */
    PMLSH_ETIMEOUT = 3,   /* a bounded wait expired */
    PMLSH_ECUDA = 4,      /* a CUDA runtime call failed */
    PMLSH_ECANCELED = 5,  /* request cancelled or server stopped */
    PMLSH_EINTERNAL = 6   /* an internal capacity was exceeded */
} pmlsh_status;

typedef struct pmlsh_index pmlsh_index;   /* opaque */

/* ------------------------------------------------------------ parameters */

/* Eq. 9 (Sec. 5.3) and Lemma 5: t = sqrt(chi^2_{alpha1}(m)) (upper
 * quantile, Lemma 3), alpha2 = Pr[chi^2(m) <= t^2 / c^2], beta = 2 alpha2.
 * Requires 1 <= m <= 16, c > 1, 0 < alpha1 < 1.  Any output may be NULL. */
pmlsh_status pmlsh_params(int m, double c, double alpha1,
                          double *t, double *alpha2, double *beta_eq9);

/* Algorithm 2 budget: the smallest integer B with B >= beta n + k,
 * computed as ceil(beta n - 1e-9) + k. */
int64_t pmlsh_budget(int64_t n, double beta, int64_t k);

/* ------------------------------------------------------------------ build */

typedef struct {
    int m;              /* number of projections (Eq. 3), 1..16; default 15 */
    int s;              /* number of global pivots (Sec. 4.1), 0..8; default 5 */
    int leaf_size;      /* leaf capacity M (points per leaf), 16..1024;
                           default 256; 0 = autotuned: the index is built
                           for M = 128, 256 and 512, pmlsh_knn with the
                           default options is timed on up to 1,024 rows of X
                           (an even stride) as queries, and the fastest index
                           is kept (pmlsh_index_info reports its M);
                           -1 = chosen by the cost model of Sec. 4.2: of
                           the same candidates, the index with the fewest
                           modelled distance computations per query,
                           L + CC(range(q, t r_min)) (pmlsh_cost_model, F
                           from 65,536 pairs of stream seed + 6, t and r_min
                           for the default query options) */
    int cp_leaf_size;   /* unused by pmlsh_build; see pmlsh_cp_opts */
    uint64_t seed;      /* the projection uses stream seed+2 of the
                           counter-based SplitMix64 generator with the
                           Box-Muller transform; the r_min sample uses seed+3 */
    const float *proj;  /* optional caller projection A, row-major [m][d]
                           FP32, host or device; NULL = draw from `seed` */
    int64_t rmin_pairs; /* pairs sampled for the distance distribution F of
                           Sec. 5.2 (r_min rule); 0 = default 10000 */
    int bf16_shadow;    /* 1 (default) = also keep the tensor-core operand of
                           the projected points (BF16 hi/lo split, 100 bytes
                           per point) that PMLSH_BF16_TENSOR needs and the BF16
                           residual rows (2 bytes per coordinate plus 4 per
                           point) that PMLSH_BF16_VERIFY needs */
} pmlsh_build_opts;

/* Fills `o` with the defaults above. */
void pmlsh_build_opts_default(pmlsh_build_opts *o);

/* Builds an index over X [n][d] (row-major FP32, host or device).
 *   Projects every point (Eq. 3) in FP64 and FP32, partitions the projected
 *   points into leaves of at most M points by recursive bisection, records
 *   each leaf's ball (centre, radius) and pivot rings (the PM-tree node
 *   entries of Sec. 4.1) and a binary hierarchy of leaves (used by
 *   pmlsh_closest_pair), samples the distance distribution for r_min and
 *   keeps a permuted device copy of X.  X is not referenced afterwards.
 * Errors: EINVAL (NULL pointers, n < 1, d < 1, m outside 1..16, s outside
 *   0..8, leaf_size outside 0, -1 or 16..1024, n >= 2^31), ENOMEM, ECUDA.
 * On success *out owns device memory until pmlsh_free(*out). */
pmlsh_status pmlsh_build(const float *X, int64_t n, int d,
                         const pmlsh_build_opts *opts, void *stream,
                         pmlsh_index **out);

void pmlsh_free(pmlsh_index *index);

/* Index facts: n, d, m, leaf count, leaf size, node count. Any may be NULL. */
pmlsh_status pmlsh_index_info(const pmlsh_index *index, int64_t *n, int *d,
                              int *m, int64_t *leaves, int *leaf_size,
                              int64_t *nodes);

/* Copies the projection actually used, [m][d] FP32, to host memory. */
pmlsh_status pmlsh_get_projection(const pmlsh_index *index, float *A_host);

/* Copies the FP64 projected coordinates [n][m], in original id order, to
 * host memory (Eq. 3). */
pmlsh_status pmlsh_get_projected(const pmlsh_index *index, double *O_host);

/* Exports the leaf hierarchy to host buffers (sizes from pmlsh_index_info):
 *   perm [n] int32       point id at each leaf-order position
 *   leaf_off [L+1]       leaf l holds positions [leaf_off[l], leaf_off[l+1])
 *   node_lo, node_hi [N] node e covers leaves [node_lo[e], node_hi[e])
 *   node_left, node_right [N] children, -1 for a leaf node; node 0 = root.
 * Any pointer may be NULL to skip that array. */
pmlsh_status pmlsh_export_layout(const pmlsh_index *index, int32_t *perm,
                                 int64_t *leaf_off, int64_t *node_lo,
                                 int64_t *node_hi, int32_t *node_left,
                                 int32_t *node_right);

/* Exports the PM-tree entry of every leaf (Sec. 4.1: e.RO, e.r, e.HR[i]) as
 * the index uses it in the Eq. 5 test, to host buffers (L from
 * pmlsh_index_info, m the projection count):
 *   s                    number of pivots
 *   centre [L][m]        routing object RO (FP32)
 *   radius [L]           covering radius r (FP32, rounded up so that it
 *                        covers the FP32 coordinates of the leaf's points)
 *   ring_min, ring_max [L][s]  HR[i].min / HR[i].max, widened by 1e-5
 *   pivots [s][m]        the pivots p_i.
 * Any pointer may be NULL.  EINVAL (NULL index), ECUDA. */
pmlsh_status pmlsh_export_leaf_entries(const pmlsh_index *index, int *s,
                                       float *centre, float *radius,
                                       float *ring_min, float *ring_max,
                                       float *pivots);

/* ------------------------------------------------------------- cost model */

/* Sec. 4.2 (cost model of the PM-tree): a sample of the distance
 * distribution F(x) = Pr[||o_i, o_j|| <= x] of the indexed points in the
 * projected space.  Pair s has ids i = v_{2s} mod n and j = v_{2s+1} mod n,
 * v the counter-based SplitMix64 stream `seed` (j = i is moved to
 * i + 1 mod n); each distance is the FP64 Euclidean distance of the FP64
 * projected coordinates (sequential sum, correctly rounded square root).
 * out_sorted [npairs] FP64 (host or device, caller-owned) receives the
 * distances in ascending order; its empirical CDF is the estimate of F.
 * EINVAL (n < 2, npairs outside 1..2^28), ENOMEM, ECUDA. */
pmlsh_status pmlsh_distance_sample(const pmlsh_index *index, int64_t npairs,
                                   uint64_t seed, double *out_sorted,
                                   void *stream);

/* Sec. 4.2: for each radius rq[r] (projected space, >= 0), the cost model's
 *   Pr[e] = F(e.r + rq) * prod_i (F(e.HR[i].max + rq) - F(e.HR[i].min - rq))
 * over the index's leaves e (their entries as pmlsh_export_leaf_entries
 * gives them, widened to FP64), and
 *   out_cc[r]    = CC(range(q, rq)) = sum_e N(e) Pr[e]   (N(e): leaf size),
 *   out_nodes[r] = sum_e Pr[e]                           (expected leaves).
 * F is the empirical CDF (fraction of entries <= x) of F_sorted [nF] FP64,
 * ascending and finite, e.g. from pmlsh_distance_sample.  F_sorted, rq [nr]
 * and the outputs [nr] may be host or device (caller-owned); either output
 * may be NULL.  The leaves are summed on the device in a fixed order.
 * EINVAL (F not ascending or not finite, nF outside 1..2^28, nr outside
 * 0..65535, rq < 0 or NaN), ENOMEM, ECUDA. */
pmlsh_status pmlsh_cost_model(const pmlsh_index *index, const double *F_sorted,
                              int64_t nF, const double *rq, int64_t nr,
                              double *out_cc, double *out_nodes, void *stream);

/* Projects the rows of Q [nq][d] (FP32, host or device) onto the index's m
 * directions (Eq. 3, the first step of Algorithm 2): out64 [nq][m] holds the
 * FP64 coordinates (sequential sums over d, the same arithmetic as the
 * build-time projection of the data set), out32 [nq][m] the same values
 * rounded to FP32.  Outputs may be host or device memory; either may be
 * NULL.  Uses (and may grow) the index's scratch buffers, so calls on one
 * index must not overlap.  Errors: EINVAL, ENOMEM, ECUDA. */
pmlsh_status pmlsh_project(pmlsh_index *index, const float *Q, int64_t nq,
                           double *out64, float *out32, void *stream);

/* pmlsh_project without any device allocation, for callers that cannot let
 * a library call cudaMalloc: a process whose device memory is owned by its
 * own caching allocator (a library cudaMalloc could fail or fragment that
 * reservation), or a latency-critical loop where cudaMalloc's implicit
 * device-wide synchronisation would stall other streams.  The paper has no
 * counterpart; this is a deployment convenience.
 *   The query rows are staged in a 16 MiB array of device memory that is
 *   part of the library image (every GPU that loads the library holds it
 *   until the process exits), so nq * (d rounded up to a multiple of 32)
 *   must not exceed 4,194,304; larger batches are rejected with EINVAL.
 *   With lazy module loading (the CUDA default) the driver reserves the
 *   array when the first call on a device looks up its address, so that
 *   first call can fail with ECUDA if the device is full; a process whose
 *   own allocator reserves the device should make one warm-up call at
 *   start-up, before that reservation.
 *   Outputs (out64 [nq][m] FP64, out32 [nq][m] FP32, either may be NULL)
 *   must be device memory; Q may be host or device memory.  Results are
 *   identical to pmlsh_project's.
 *   The first call on each device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents: calls
 *   that overlap on the GPU (other streams, other threads) race and must be
 *   serialised by the caller.
 *   No cudaMalloc, cudaFree or allocating routine is called.
 * Errors: EINVAL (NULL pointers, size beyond the limit, host outputs),
 *   ECUDA. */
pmlsh_status pmlsh_project_noalloc(const pmlsh_index *index, const float *Q,
                                   int64_t nq, double *out64, float *out32,
                                   void *stream);

/* ------------------------------------------------------- (c,k)-ANN query */

/* Precision modes (bits; PMLSH_BF16_RERANK = both) */
enum { PMLSH_FP32_PLAIN = 0, PMLSH_BF16_TENSOR = 1, PMLSH_BF16_VERIFY = 2, PMLSH_BF16_RERANK = 3 };
enum { PMLSH_STOP_LITERAL = 0, PMLSH_STOP_BC_CONSISTENT = 1 };

typedef struct {
    int k;            /* neighbours per query, 1..min(n, 256) */
    double c;         /* approximation ratio c > 1 (Definition 2) */
    double alpha1;    /* E1 failure probability (Lemma 4); default 1/e */
    double beta;      /* candidate budget fraction, 0 < beta <= 1;
                         default 0.2809 (Sec. 7.1) */
    double r_min;     /* first radius; <= 0: the Sec. 5.2 rule (r* with
                         F(rstar) = (beta n + k)/n on the sampled distance
                         distribution, r_min = rstar / c) */
    int precision;    /* bit set.  PMLSH_BF16_TENSOR: the range rounds count
                         projected distances on the tensor cores (q'.o' from a
                         three-product BF16 split, FP32 accumulate; every
                         pair whose decision that value cannot settle is
                         recomputed exactly), else on the CUDA cores.
                         PMLSH_BF16_VERIFY: verification's first pass reads
                         BF16 residual rows (each row minus its leaf's
                         original-space centre, rounded to BF16) and bounds
                         every candidate's distance from below and above;
                         the candidates whose lower bound can reach the k-th
                         upper bound are reranked from the FP32 rows, then
                         FP64 where FP32 cannot decide; a query whose bounds
                         cannot settle that set is verified again without
                         the first pass.  PMLSH_FP32_PLAIN (0): neither.
                         Every mode returns the same ids, distances and
                         statistics |C|, rounds, stop rule (n_verified and
                         leaves_visited describe the work done).  Both BF16
                         bits need an index built with bf16_shadow = 1 (else
                         PMLSH_EINVAL) */
    double t;         /* projected radius factor of Lemma 4; <= 0: t from
                         alpha1 by Eq. 9 (t = sqrt(chi^2_{alpha1}(m))) */
    int stop_rule;    /* PMLSH_STOP_LITERAL: stop rule 1 tested at the loop
                         top after r <- c r, as printed in Algorithm 2;
                         PMLSH_STOP_BC_CONSISTENT: tested after the range
                         query with the same r (Algorithm 1's form) */
} pmlsh_knn_opts;

void pmlsh_knn_opts_default(pmlsh_knn_opts *o);

typedef struct {
    int32_t rounds;        /* range queries run */
    int32_t stop_rule;     /* 1: >= k verified within c r; 2: budget
                              |C| >= beta n + k reached; 3: C = D */
    int64_t n_cand;        /* |C| at return */
    double r_final;        /* r at return */
    int32_t fp64_checks;   /* decisions re-taken in FP64 */
    int32_t leaves_visited; /* leaves whose candidates were verified */
    int64_t n_verified;    /* exact distances computed, over all rounds */
    int32_t first_pass_fallbacks; /* rounds whose BF16 first pass (precision
                              PMLSH_BF16_VERIFY) could not settle the rerank
                              set, so that FP32 verification redid them */
    int32_t reserved;
} pmlsh_query_stats;

/* Algorithm 2 for nq queries Q [nq][d] (FP32, host or device).
 * Outputs (host or device): out_ids [nq][k] int64 original ids,
 * out_dists [nq][k] FP32 distances (the FP64 distance rounded to FP32),
 * out_err [nq][k] or NULL: |out_dist - FP64 distance| per result,
 * stats [nq] or NULL.
 * Candidate set reading: C_i is the closed range set {o : ||o',q'|| <=
 * t r_i}; once |C_i| >= B (B = pmlsh_budget(n, beta, k)) C_i keeps the B
 * points with the smallest (||o',q'||, id) and stop rule 2 returns.
 * Errors: EINVAL (NULL pointers, nq < 0, k < 1, k > min(n, 256), c <= 1,
 *   beta outside (0,1], alpha1 outside (0,1)), ENOMEM, ECUDA, EINTERNAL
 *   (more than the internal capacity of points tied within one FP32 error
 *   band; the message says which). nq = 0 returns PMLSH_OK at once. */
pmlsh_status pmlsh_knn(pmlsh_index *index, const float *Q, int64_t nq,
                       const pmlsh_knn_opts *opts, int64_t *out_ids,
                       float *out_dists, float *out_err,
                       pmlsh_query_stats *stats, void *stream);

/* The first radius r_min that pmlsh_knn uses when opts.r_min <= 0 (the rule
 * of Sec. 5.2 on the index's sampled distance distribution: r* with
 * F(r*) = min(1, (beta n + k) / n), its lower empirical quantile, then
 * r_min = r* / c).  Errors: EINVAL (NULL pointers, beta outside (0, 1],
 * k < 1, c <= 1). */
pmlsh_status pmlsh_rmin(const pmlsh_index *index, double beta, int k, double c,
                        double *r_min);

/* Device scratch bytes pmlsh_knn reserves (and keeps in the index) for a
 * batch of nq queries with this k and precision: every buffer whose size
 * the batch fixes.  Not included: the budget selection's key buffers, which
 * grow with the range sets of the queries that reach the budget (8 bytes per
 * point of those sets).  Errors: EINVAL (NULL pointers, nq < 0, k outside
 * 1..256). */
pmlsh_status pmlsh_knn_workspace_bytes(pmlsh_index *index, int64_t nq, int k,
                                       int precision, int64_t *bytes);

/* Algorithm 1, the (r,c)-BC query (Sec. 5.1), for nq queries Q [nq][d]
 * (FP32, host or device) at one radius r > 0.  Per query, C is the closed
 * range set {o : ||o',q'|| <= t r} (no budget cut); if |C| >= beta n + 1
 * (as an integer: pmlsh_budget(n, beta, 1)) or the point of C nearest to q
 * lies within c r, that point is returned, else nothing (id -1, distance
 * +inf).  From `opts` the call uses c, alpha1 (or t), beta and precision;
 * k, r_min and stop_rule are ignored.  Outputs (host or device): out_ids
 * [nq] int64 original ids, out_dists [nq] FP32 (the FP64 distance rounded),
 * stats [nq] or NULL (rounds = 1, stop_rule 2: |C| >= beta n + 1, 1: within
 * c r, 0: nothing; n_cand = |C|).  Ties by smaller id.  Errors: EINVAL (NULL
 * pointers, r <= 0, options as pmlsh_knn), ENOMEM, ECUDA, EINTERNAL. */
pmlsh_status pmlsh_rcbc(pmlsh_index *index, const float *Q, int64_t nq,
                        double r, const pmlsh_knn_opts *opts, int64_t *out_ids,
                        float *out_dists, pmlsh_query_stats *stats,
                        void *stream);

/* ---------------------------------------------------- (c,k)-ACP query */

typedef struct {
    int k;            /* closest pairs to return, 1..min(n(n-1)/2, 1024) */
    double c;         /* approximation ratio c > 1 (Definition 4) */
    double alpha1;    /* Lemma 4; default 1/e; gives t by Eq. 9 when t <= 0 */
    double alpha2;    /* budget fraction: T = ceil(alpha2 n (n-1)) + k when
                         T <= 0; default 0.0024 (Sec. 7.1) */
    int64_t T;        /* candidate-pair budget of Algorithm 4; <= 0: from alpha2 */
    double gamma;     /* radius-filter factor (Sec. 6.3), may be +inf;
                         <= 0 (default): calibrated with Pr(gamma) = 0.85
                         (Sec. 7.1) by pmlsh_gamma_calibrate on 10,000
                         sampled points, stream seed + 7 */
    double t;         /* projected radius factor; <= 0: from alpha1 (Eq. 9) */
} pmlsh_cp_opts;

void pmlsh_cp_opts_default(pmlsh_cp_opts *o);

typedef struct {
    int64_t count;       /* verified pairs (Algorithm 4's count) */
    double ub_self;      /* k-th distance after the leaf self-joins */
    int64_t lca_nodes;   /* nodes returned by FindLCA */
    int64_t nodes_done;  /* of those, nodes examined before count > T */
    int64_t self_pairs;  /* pairs inside leaves */
    int64_t fp64_checks; /* projected-distance decisions re-taken in FP64 */
    double t;            /* t used */
    int64_t T;           /* T used */
    double gamma;        /* gamma used (pmlsh_closest_pair) */
} pmlsh_cp_stats;

/* Algorithm 4 (radius filtering) with FindLCA (Algorithm 5) over the index's
 * leaf hierarchy (pmlsh_export_layout): every pair inside a leaf is verified
 * (count = their number, ub = k-th distance); R = gamma t ub; the maximal
 * inner nodes with ball radius < R (FP64 bounding-box-midpoint balls of the
 * projected points) are taken in ascending (radius, node id); for each, the
 * pairs of its subtree that lie in different leaves and have projected
 * distance < t ub (ub as the node starts) are verified, keeping only the
 * T + 1 - count smallest by (projected distance, i, j) if count would pass
 * T; ub is updated after each node; the loop ends once count > T.
 * Outputs (host or device): out_pairs [k][2] original ids (i < j),
 * out_dists [k] FP32 (FP64 distance rounded), stats or NULL.  Pairs sorted
 * by (distance, i, j); missing entries are -1 / +inf.
 * Errors: EINVAL (k, gamma, alpha), ENOMEM, ECUDA, EINTERNAL (more than 4096
 * pairs tied inside one FP32 error band). */
pmlsh_status pmlsh_closest_pair(pmlsh_index *index, const pmlsh_cp_opts *opts,
                                int64_t *out_pairs, float *out_dists,
                                pmlsh_cp_stats *stats, void *stream);

/* Setting of gamma for radius filtering (Sec. 6.3, "Determining the Setting
 * of gamma"; Sec. 7.1 uses Pr(gamma) = 0.85).  A sample of
 * n' = min(nsample, n) points is drawn (partial Fisher-Yates shuffle of the
 * ids 0..n-1 whose i-th step swaps entry i with entry i + (v_i mod (n - i)),
 * v_i value i of the counter-based SplitMix64 stream `seed`; the first n'
 * ids, ascending) and indexed by the same build as `index` (its projection,
 * pivot count and leaf capacity; the index itself when n' = n).  For every
 * pair of the sample the ratio R / ||o1', o2'|| of its lowest common node's
 * radius (the FP64 ball of pmlsh_closest_pair; the leaf for two points of
 * one leaf) over its FP64 projected distance is formed (0 / 0 -> 0,
 * R / 0 -> +inf), and *gamma receives the lower empirical quantile at `pr`:
 * the smallest ratio with at least pr of the n'(n'-1)/2 ratios at or below
 * it.  Device memory: 8 bytes per pair.  Errors: EINVAL (NULL pointers, pr
 * outside (0, 1], nsample outside 2..32768, n < 2), ENOMEM, ECUDA. */
pmlsh_status pmlsh_gamma_calibrate(pmlsh_index *index, double pr, int64_t nsample,
                                   uint64_t seed, double *gamma, void *stream);

/* Algorithm 3, branch and bound (Sec. 6.1): the T pairs with the smallest
 * projected distance (ties by (i, j); T = opts->T, or ceil(alpha2 n (n-1))
 * + k when T <= 0; at least k, at most n(n-1)/2) are found by a best-first
 * search over leaf pairs in ascending Mindist (the larger of the pivot-ring
 * gap and ||RO1, RO2|| - r1 - r2 of the two leaf entries), starting from
 * every leaf's self-join, stopping at the first leaf pair whose Mindist
 * exceeds the T-th projected distance; they are verified by their original
 * distance and the k nearest are returned.  Leaf pairs are listed in bands of
 * Mindist, the first ending near the T-th distance of a sample of 65,536
 * projected pair distances (stream seed + 8), each later one quadrupling the
 * sample quantile, until a band reaches the T-th distance: the result does
 * not depend on the bands.  From `opts` the call uses k, T and alpha2 (c,
 * alpha1, t and gamma are not used).  Outputs as pmlsh_closest_pair; stats:
 * count = pairs verified (T), lca_nodes = leaf pairs listed, nodes_done =
 * leaf pairs examined, self_pairs, fp64_checks.  Memory grows with T (12 bytes per kept
 * pair plus a batch of up to 2^24 pairs) and with the leaf count L: a listing
 * buffer of 12 bytes per leaf pair, L(L-1)/2, and 16 bytes per listed leaf
 * pair while a band is ordered (on the device by a radix sort for up to
 * 92,682 leaves, on the host beyond).  Errors: EINVAL, ENOMEM,
 * ECUDA, EINTERNAL (more than 4096 pairs tied inside one FP32 error band; a
 * device ordering that fails its check). */
pmlsh_status pmlsh_closest_pair_bnb(pmlsh_index *index, const pmlsh_cp_opts *opts,
                                    int64_t *out_pairs, float *out_dists,
                                    pmlsh_cp_stats *stats, void *stream);

/* ------------------------------------------------------------- serving */

/* Continuous batching over one resident index.  `slots` worker threads, each
 * with its own CUDA stream and scratch buffers, take the oldest waiting
 * request plus every later waiting request with identical query options (up
 * to max_batch_queries rows) and run them as one pmlsh_knn batch, so
 * requests that arrive while others run are admitted as slots and memory
 * free up and their work overlaps on the device.  Each request's results
 * equal pmlsh_knn's on that request alone.
 * Memory admission: a batch starts when the scratch every slot holds, the
 * growth charged to running batches and its own growth (the bytes by
 * which its slot's scratch buffers grow to the sizes pmlsh_knn asks for) fit
 * mem_budget_bytes; when nothing runs, idle slots release their scratch to
 * make room, and a batch that needs more than the budget by itself runs
 * alone.  A slot whose batch left the total above the budget releases its
 * scratch afterwards.  Not counted: the budget selection's key buffers
 * (8 bytes per point in the range sets of queries that reach the budget). */
typedef struct pmlsh_server pmlsh_server;

typedef struct {
    int slots;                  /* concurrent batches (streams); default 3 */
    int64_t max_batch_queries;  /* rows per batch; default 16384 */
    int64_t mem_budget_bytes;   /* device scratch across slots; default 8 GiB */
} pmlsh_serve_opts;

typedef struct {
    int64_t submitted, completed, queries, batches;
    int64_t deferred;     /* times a slot waited for memory */
    int64_t canceled;     /* requests cancelled by pmlsh_serve_stop */
    int64_t queue_depth;  /* requests waiting now */
    double p50_ms, p99_ms, mean_ms;  /* submit -> completion latency */
    double qps;           /* queries / (last completion - first submission) */
    int64_t resident_bytes; /* device scratch the slots hold now, plus the
                               growth charged to running batches */
    int64_t peak_bytes;     /* the largest such total seen */
} pmlsh_server_stats;

void pmlsh_serve_opts_default(pmlsh_serve_opts *o);

/* Starts the worker threads on the current device.  The index must outlive
 * the server.  Errors: EINVAL, ENOMEM. */
pmlsh_status pmlsh_serve_create(pmlsh_index *index, const pmlsh_serve_opts *opts,
                                pmlsh_server **out);

/* Queues Q [nq][d] (host memory, copied before return) with `opts` and
 * returns a ticket.  Errors: EINVAL (options as pmlsh_knn, nq < 1, device
 * pointer), ENOMEM, ECANCELED (server stopping). */
pmlsh_status pmlsh_serve_submit(pmlsh_server *s, const float *Q, int64_t nq,
                                const pmlsh_knn_opts *opts, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: no limit) for the ticket and copies its
 * results to host buffers ids [nq][k], dists [nq][k] and, unless NULL,
 * err [nq][k] (|returned distance - FP64 distance| per result, as
 * pmlsh_knn's out_err).  ETIMEOUT leaves the ticket valid; any other return
 * consumes it.  ECANCELED: cancelled by pmlsh_serve_stop.  The query path's
 * own errors are passed through. */
pmlsh_status pmlsh_serve_wait(pmlsh_server *s, uint64_t ticket, int64_t *ids,
                              float *dists, float *err, int timeout_ms);

/* Stops accepting requests, cancels the ones not yet started (their waits
 * return ECANCELED), lets running batches finish, joins the workers. */
pmlsh_status pmlsh_serve_stop(pmlsh_server *s);

pmlsh_status pmlsh_serve_stats(pmlsh_server *s, pmlsh_server_stats *out);

/* pmlsh_serve_stop, then frees the server. */
pmlsh_status pmlsh_serve_destroy(pmlsh_server *s);

/* ------------------------------------------------------------- profiling */

/* Turns per-kernel timing on (1) or off (0), process-wide.  While on, every
 * kernel launch of the library is bracketed by two CUDA events recorded on
 * the launch's own stream (a few microseconds of overhead per launch). */
pmlsh_status pmlsh_profile(int enable);

/* Writes the timings gathered since the last read as a JSON object
 * {"kernel_name": [launches, total_ms], ...} into buf (cap bytes, host) and
 * clears them; waits for the recorded events.  EINVAL if cap is too small. */
pmlsh_status pmlsh_profile_read(char *buf, int64_t cap);

/* Number of kernel launches the library has issued in this process. */
long long pmlsh_launch_count(void);

/* ------------------------------------------------------------ thread info */

/* Description of the last failure on the calling thread ("" if none). */
const char *pmlsh_last_error(void);

/* Library version string. */
const char *pmlsh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PMLSH_H */
