// Internal declarations of libpmlsh (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pmlsh.h"

// Projected coordinates are padded to 16 lanes (m <= 16); padded lanes are 0
// for points, queries and pivots, so they add nothing to any distance.
#define PM_MP 16
// Leaf metadata, FP32, per leaf: [0,16) centre RO, [16] radius (over FP32
// coordinates, rounded up), [17,24) radial profile (for g = 2 .. 8 an upper
// bound of the ceil(g s / 8)-th largest member radius), [24,32) ring minima,
// [32,40) ring maxima (Sec. 4.1: e.RO, e.r, e.HR[s]).
#define PM_LEAF_STRIDE 40
#define PM_MAX_PIVOTS 8
#define PM_MAX_K 256
#define PM_PCA 16

// Thread-local error reporting.
void pm_set_error(const char *fmt, ...);

struct PmStatus {
    pmlsh_status code = PMLSH_OK;
    bool ok() const { return code == PMLSH_OK; }
};

#define PM_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            pm_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                  \
            return e_ == cudaErrorMemoryAllocation ? PMLSH_ENOMEM : PMLSH_ECUDA; \
        }                                                                      \
    } while (0)

#define PM_TRY(expr)                                                           \
    do {                                                                       \
        pmlsh_status s_ = (expr);                                              \
        if (s_ != PMLSH_OK) return s_;                                         \
    } while (0)

// A grow-only device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    pmlsh_status reserve(size_t b);
    void release();
    template <class T> T *as() const { return (T *)p; }
};

// A grow-only pinned host buffer (device-to-host copies that do not block
// the host until the stream drains).
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    pmlsh_status reserve(size_t b);
    void release();
};

// Per-call scratch buffers of the query path (kept in the index, grown on
// demand, reused across calls).
struct KnnWork {
    DevBuf Qd, qp32, qp64, qnorm, qpiv, order, keys, keys2, vals2, sortTmp;
    DevBuf qstate, thr, blkCnt, blkLeaves, blkMask, cntSure, cntBand, bandQ, bandPos,
        bandIn, bandCnt;
    DevBuf partD, partI, partSeen, bandInQ, outD64, outIds, outErr, dk, flags;
    DevBuf selBuf, selOff, selCnt, selTau;
    DevBuf active, misc, recheck, leafBits, fullBits, cntPart, cntTight, subIdx, subThr, subBits, qpca;
    HostBuf stage;   // per-round decisions read by the host
};

struct pmlsh_index {
    int64_t n = 0;
    int d = 0, ld = 0;      // ld: padded row length (multiple of 32)
    int m = 0, s = 0, M = 0;
    int64_t L = 0;          // leaves
    uint64_t seed = 0;
    // device arrays (leaf order)
    float *X = nullptr;     // [n][ld]
    int32_t *perm = nullptr;  // [n] position -> id
    float *O32 = nullptr;   // [n][16]
    double *O64 = nullptr;  // [n][16]
    float *A32 = nullptr;   // [16][ld]
    int64_t *leafOff = nullptr;  // [L+1]
    float *leafMeta = nullptr;   // [L][PM_LEAF_STRIDE]
    float *piv32 = nullptr;      // [PM_MAX_PIVOTS][16]
    float *leafMu = nullptr;     // [L][ld] original-space leaf centre (FP32)
    float *leafRx = nullptr;     // [L] radius around leafMu (rounded up)
    // principal directions of the leaf centres (orthonormal rows) and the
    // centres' coordinates along them: ||P q - P mu|| <= ||q - mu||
    double *pcaP = nullptr;      // [PM_PCA][ld] FP64
    float *pcaP32 = nullptr;     // the same rounded to FP32
    float *leafPmu = nullptr;    // [L][PM_PCA] P mu (FP64 rounded to FP32)
    double muMax = 0.0;          // max ||mu_l|| (FP64)
    // chunks: consecutive runs of <= 32 points inside a leaf, with their own
    // original-space balls
    int64_t nChunks = 0;
    int64_t *chunkOff = nullptr;   // [C+1] positions
    int32_t *leafChunk = nullptr;  // [L+1] chunk range of each leaf
    float *chunkMu = nullptr;      // [C][ld]
    float *chunkRx = nullptr;      // [C]
    // tensor-core operand of the projected points: leaf-padded rows
    int64_t *bOff = nullptr;       // [L+1] first row of each leaf (multiple of 16)
    uint16_t *Bsplit = nullptr;    // BF16 [rows][48] in the UMMA canonical layout
    float *bNorm = nullptr;        // [rows] ||o'||^2 (FP32 coordinates), NaN on padding rows
    // BF16 residuals of the rows from their leaf centre (first pass of the
    // verification) and per row the bound of what the rounding lost
    uint16_t *Xr = nullptr;        // [n][ld] BF16(fl32(x - mu_leaf))
    float *rowErr = nullptr;       // [n] >= ||x - mu_leaf - r~||
    std::vector<int64_t> bOffH;
    std::vector<int64_t> chunkOffH;
    std::vector<int32_t> leafChunkH;
    // host copies
    std::vector<float> A_host;       // [m][d]
    std::vector<int64_t> leafOffH;   // [L+1]
    std::vector<int32_t> permH;      // [n]
    std::vector<int64_t> nodeLo, nodeHi;
    std::vector<int32_t> nodeLeft, nodeRight;
    // device copy of the hierarchy used to route queries to a leaf:
    // [e] = {left, right, unused, first leaf}; [e] = {w[16], t}: right iff
    // w . q' >= t
    int32_t *treeI = nullptr;   // [N][4]
    float *treeV = nullptr;     // [N][17]
    std::vector<double> distSample;  // sorted sampled distances (r_min rule)
    double maxNorm = 0.0;            // max ||o'|| (FP64 coordinates)
    KnnWork work;
};

// Build helpers (build.cu)
pmlsh_status pm_build_index(pmlsh_index *ix, const float *X, bool x_on_device,
                            const pmlsh_build_opts *o, cudaStream_t st);
void pm_free_index(pmlsh_index *ix);

// FP64 + FP32 projection of rows X [n][ld] (build.cu), original row order;
// outputs [n][ostride] (ostride = 16 for the padded internal layout, or m),
// either output may be NULL.
void pm_launch_project64(const float *X, int64_t n, int ld, int d, int m, const float *A,
                         double *O64, float *O32, unsigned long long *maxNormBits,
                         cudaStream_t st, int ostride = PM_MP);

void pm_launch_project64_noprof(const float *X, int64_t n, int ld, int d, int m, const float *A,
                                double *O64, float *O32, cudaStream_t st, int ostride);

// Original-space refinement of the leaf layout (layout.cu).  For each
// segment [segLo[i], segHi[i]) of positions of permD (at most 1024 points,
// ids into the original-order rows Xo [n][ld]), permD is reordered within the
// segment and res[i] receives the segment's sub-hierarchy: node {begin, end,
// left, right} (offsets from segLo[i]; local node ids, -1 for a leaf; node 0
// is the segment itself), leaf {begin, end, node, first chunk} in position
// order, and chunk end offsets.
struct LrResult {
    std::vector<int4> node, leaf;
    std::vector<int32_t> chunkEnd;
};
pmlsh_status pm_refine_leaves(const float *Xo, int ld, int d, int32_t *permD, const std::vector<int64_t> &segLo,
                              const std::vector<int64_t> &segHi, std::vector<LrResult> &res, cudaStream_t st);

// Query projection (api.cu helper in knn.cu): stages Q into `staging`
// ([nq][ld], device) and projects it.
pmlsh_status pm_project_rows(const pmlsh_index *ix, const float *Q, int64_t nq, float *staging,
                             double *out64, float *out32, int ostride, cudaStream_t st);

// Query path (knn.cu)
// `work`: scratch buffers for this call (NULL: the index's own); calls on
// one index may run concurrently on different streams with different
// workspaces (the index itself is read-only during queries).
// `rcbc`: Algorithm 1 instead of Algorithm 2: one round at r = o->r_min
// with k = 1, no budget cut of the range set, the budget beta n + 1; the
// nearest candidate is kept if |C| >= beta n + 1 or it lies within c r,
// else the result is -1 / +inf (stats: stop_rule 2, 1 or 0).
pmlsh_status pm_knn(pmlsh_index *ix, const float *Q, int64_t nq,
                    const pmlsh_knn_opts *o, int64_t *ids, float *dists,
                    float *err, pmlsh_query_stats *stats, cudaStream_t st,
                    KnnWork *work = nullptr, bool rcbc = false);
void pm_release_work(KnnWork &w);
// Device bytes pm_knn reserves in a workspace for a batch of nq queries with
// this k and precision: every buffer whose size the batch fixes.  Not
// included: the budget selection's key buffers (8 bytes per point in the
// range sets of the queries that reach the budget B in a round).
int64_t pm_knn_work_bytes(const pmlsh_index *ix, int64_t nq, int k, int precision);
// How many bytes the workspace w grows by for such a batch (each buffer
// grows only to the size the batch asks for).
int64_t pm_knn_work_growth(const pmlsh_index *ix, int64_t nq, int k, int precision, const KnnWork &w);
// Device bytes a workspace holds now.
int64_t pm_work_resident(const KnnWork &w);

// Closest pairs (cp.cu)
pmlsh_status pm_closest_pair(pmlsh_index *ix, const pmlsh_cp_opts *o, int64_t *out_pairs, float *out_dists,
                             pmlsh_cp_stats *stats, cudaStream_t st);
// gamma of Sec. 6.3 at probability pr over a sample of nsample points (all
// points when nsample >= n) drawn from stream `seed` (cp.cu).
pmlsh_status pm_gamma_calibrate(pmlsh_index *ix, double pr, int64_t nsample, uint64_t seed, double *gamma,
                                cudaStream_t st);
pmlsh_status pm_closest_pair_bnb(pmlsh_index *ix, const pmlsh_cp_opts *o, int64_t *out_pairs, float *out_dists,
                             pmlsh_cp_stats *stats, cudaStream_t st);

// Cost model of Sec. 4.2 (cost.cu)
// Sorted FP64 projected distances of `npairs` sampled pairs (host vector).
pmlsh_status pm_distance_sample(const pmlsh_index *ix, int64_t npairs, uint64_t seed, std::vector<double> &out,
                                cudaStream_t st);
// CC and sum of Pr[e] over the leaves for each radius rq[r]; F and rq on the
// host, F sorted ascending.
pmlsh_status pm_cost_model(const pmlsh_index *ix, const double *F, int64_t nF, const double *rq, int64_t nr,
                           double *cc, double *nodes, cudaStream_t st);
// The r_min rule of Sec. 5.2 for a query with these options.
double pm_rmin_rule(const pmlsh_index *ix, double beta, int64_t k, double c);

// Parameters (params.cpp)
double pm_chi2_sf(double x, int m);
double pm_chi2_upper_quantile(double alpha, int m);

// Counter-based SplitMix64 (rng.cpp)
uint64_t pm_splitmix64(uint64_t seed, uint64_t i);
// The same generator for device code: value i of stream `seed` is the
// SplitMix64 finaliser of seed + (i + 1) * 0x9E3779B97F4A7C15.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint64_t pm_splitmix64_hd(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
void pm_gaussian_projection(uint64_t seed, int m, int d, float *A);

bool pm_is_device_ptr(const void *p);

// Largest shared memory a block may opt in to on the current device.
int pm_max_smem_optin();
// Raises `func`'s dynamic shared-memory limit to the largest the device
// allows next to its static shared memory.  The limit is one setting per
// function shared by every caller (and every thread), so it is never set to
// a single call's own need.
pmlsh_status pm_allow_max_dyn_smem(const void *func);

// Launch bookkeeping (prof.cpp): counts every launch; brackets it with CUDA
// events while profiling is enabled.
int pm_prof_begin(const char *name, cudaStream_t st);
void pm_prof_end(int token, cudaStream_t st);
#define PM_LAUNCH(name, st, ...)                                               \
    do {                                                                       \
        int tok_ = pm_prof_begin(name, st);                                    \
        __VA_ARGS__;                                                           \
        pm_prof_end(tok_, st);                                                 \
    } while (0)

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
// Squared projected distance in FP32 with a fixed operation order; every
// kernel that classifies a point against a radius uses this one function, so
// all of them see bit-identical values.
__device__ __forceinline__ float pm_pd2_32(const float *a, const float *b)
{
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PM_MP; j++) {
        float t = __fsub_rn(a[j], b[j]);
        s = __fmaf_rn(t, t, s);
    }
    return s;
}

// FP32 -> FP64 widening by integer operations (exact: every FP32 value is an
// FP64 value); subnormals, infinities and NaNs take the conversion
// instruction.
__device__ __forceinline__ double pm_f2d_exact(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (e == 0u && (u & 0x7FFFFFu) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// FP64 distance of two FP64 coordinate vectors: sequential sum, separate
// multiply and add, correctly rounded square root.
__device__ __forceinline__ double pm_pdist64(const double *a, const double *b, int m)
{
    double s = 0.0;
    for (int j = 0; j < m; j++) {
        double t = __dsub_rn(a[j], b[j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return __dsqrt_rn(s);
}

// FP64 Euclidean distance of two FP32 rows of length d, same arithmetic.
__device__ __forceinline__ double pm_dist64(const float *x, const float *y, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; i++) {
        double t = __dsub_rn((double)x[i], (double)y[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return __dsqrt_rn(s);
}
#endif
