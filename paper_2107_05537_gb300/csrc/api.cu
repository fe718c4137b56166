// C ABI of libpmlsh: argument validation, pointer-kind detection, handles,
// thread-local error text.  Every entry point returns a status code; nothing
// throws across the boundary.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include "pmlsh_impl.h"

static thread_local char g_err[1024] = "";

void pm_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

bool pm_is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

pmlsh_status pm_allow_max_dyn_smem(const void *func)
{
    cudaFuncAttributes fa;
    PM_CUDA(cudaFuncGetAttributes(&fa, func));
    const int v = pm_max_smem_optin() - (int)fa.sharedSizeBytes;
    PM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
    return PMLSH_OK;
}

int pm_max_smem_optin()
{
    int dev = 0, v = 48 * 1024;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        v = 48 * 1024;
    }
    return v;
}

#define PM_CHECK(cond, ...)                                                    \
    do {                                                                       \
        if (!(cond)) {                                                         \
            pm_set_error(__VA_ARGS__);                                         \
            return PMLSH_EINVAL;                                               \
        }                                                                      \
    } while (0)

extern "C" {

const char *pmlsh_last_error(void) { return g_err; }

const char *pmlsh_version(void) { return "pmlsh-gb300 0.1 (sm_103a)"; }

pmlsh_status pmlsh_params(int m, double c, double alpha1, double *t, double *alpha2, double *beta_eq9)
{
    PM_CHECK(m >= 1 && m <= PM_MP, "m must be in 1..16 (got %d)", m);
    PM_CHECK(c > 1.0, "c must be > 1 (got %g)", c);
    PM_CHECK(alpha1 > 0.0 && alpha1 < 1.0, "alpha1 must be in (0,1) (got %g)", alpha1);
    // Eq. 9: t^2 = chi^2_{alpha1}(m); t^2 / c^2 = chi^2_{1-alpha2}(m), i.e.
    // Pr[chi^2(m) > t^2/c^2] = 1 - alpha2.  Lemma 5: beta = 2 alpha2.
    double t2 = pm_chi2_upper_quantile(alpha1, m);
    double a2 = 1.0 - pm_chi2_sf(t2 / (c * c), m);
    if (t) *t = std::sqrt(t2);
    if (alpha2) *alpha2 = a2;
    if (beta_eq9) *beta_eq9 = 2.0 * a2;
    return PMLSH_OK;
}

int64_t pmlsh_budget(int64_t n, double beta, int64_t k)
{
    return (int64_t)std::ceil(beta * (double)n - 1e-9) + k;
}

void pmlsh_build_opts_default(pmlsh_build_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->m = 15;
    o->s = 5;
    o->leaf_size = 256;
    o->cp_leaf_size = 16;
    o->seed = 0;
    o->proj = nullptr;
    o->rmin_pairs = 10000;
    o->bf16_shadow = 1;
}

void pmlsh_knn_opts_default(pmlsh_knn_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k = 10;
    o->c = 1.5;
    o->alpha1 = 0.36787944117144233;  // 1/e (Sec. 5.3)
    o->beta = 0.2809;                 // Sec. 7.1
    o->r_min = 0.0;
    o->precision = PMLSH_FP32_PLAIN;
    o->t = 0.0;
    o->stop_rule = PMLSH_STOP_LITERAL;
}

namespace {

// One index over X with the options as given (leaf_size 16..1024).
pmlsh_status build_one(const float *X, int64_t n, int d, const pmlsh_build_opts &o, cudaStream_t st,
                       pmlsh_index **out)
{
    pmlsh_index *ix = new (std::nothrow) pmlsh_index();
    if (!ix) {
        pm_set_error("host allocation failed");
        return PMLSH_ENOMEM;
    }
    ix->n = n;
    ix->d = d;
    ix->ld = (d + 31) / 32 * 32;
    ix->m = o.m;
    ix->s = std::min<int64_t>(o.s, (n + o.leaf_size - 1) / o.leaf_size);
    ix->M = o.leaf_size;
    ix->seed = o.seed;
    pmlsh_status s = pm_build_index(ix, X, pm_is_device_ptr(X), &o, st);
    if (s != PMLSH_OK) {
        pm_free_index(ix);
        delete ix;
        return s;
    }
    *out = ix;
    return PMLSH_OK;
}

// Leaf-size autotuner: builds the index for each candidate capacity, times
// pmlsh_knn with the default options (k = 10, c = 1.5, beta = 0.2809, no
// statistics) on up to 1,024 rows of X taken at an even stride as queries
// (best of two runs after one warm-up), and keeps the fastest index.
pmlsh_status build_autotuned(const float *X, int64_t n, int d, pmlsh_build_opts o, cudaStream_t st,
                             pmlsh_index **out)
{
    static const int cand[] = {128, 256, 512};
    const int64_t nq = std::min<int64_t>(n, 1024);
    const int64_t stride = n / nq;
    std::vector<float> Qs((size_t)nq * d);
    PM_CUDA(cudaMemcpy2DAsync(Qs.data(), (size_t)d * sizeof(float), X, (size_t)stride * d * sizeof(float),
                              (size_t)d * sizeof(float), (size_t)nq,
                              pm_is_device_ptr(X) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    int64_t *ids = nullptr;
    float *dd = nullptr;
    PM_CUDA(cudaMalloc(&ids, (size_t)nq * 10 * sizeof(int64_t)));
    if (cudaMalloc(&dd, (size_t)nq * 10 * sizeof(float)) != cudaSuccess) {
        cudaFree(ids);
        pm_set_error("device allocation failed");
        return PMLSH_ENOMEM;
    }
    struct Bufs { int64_t *a; float *b; ~Bufs() { cudaFree(a); cudaFree(b); } } bufs{ids, dd};
    pmlsh_knn_opts ko;
    pmlsh_knn_opts_default(&ko);
    ko.k = (int)std::min<int64_t>(10, n);
    pmlsh_index *best = nullptr;
    float bestMs = INFINITY;
    for (int M : cand) {
        if (M > n && best) break;
        o.leaf_size = M;
        pmlsh_index *ix = nullptr;
        pmlsh_status s = build_one(X, n, d, o, st, &ix);
        if (s != PMLSH_OK) {
            if (best) pmlsh_free(best);
            return s;
        }
        float ms = INFINITY;
        for (int rep = 0; rep < 3 && s == PMLSH_OK; rep++) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
            s = pm_knn(ix, Qs.data(), nq, &ko, ids, dd, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float el = INFINITY;
            cudaEventElapsedTime(&el, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rep > 0) ms = std::min(ms, el);
        }
        if (s != PMLSH_OK) {
            pmlsh_free(ix);
            if (best) pmlsh_free(best);
            return s;
        }
        if (ms < bestMs) {
            if (best) pmlsh_free(best);
            best = ix;
            bestMs = ms;
        } else {
            pmlsh_free(ix);
        }
    }
    *out = best;
    return PMLSH_OK;
}

// Leaf-size choice by the cost model of Sec. 4.2: builds the index for each
// candidate capacity and keeps the one with the fewest modelled distance
// computations per query, L (one Eq. 5 test per leaf) + CC(range(q, R)),
// at the first-round radius R = t r_min of a query with the default options
// (k = 10, c = 1.5, alpha1 = 1/e, beta = 0.2809), F estimated from 65,536
// sampled pairs (stream seed + 6).
pmlsh_status build_model_tuned(const float *X, int64_t n, int d, pmlsh_build_opts o, cudaStream_t st,
                               pmlsh_index **out)
{
    static const int cand[] = {128, 256, 512};
    pmlsh_knn_opts ko;
    pmlsh_knn_opts_default(&ko);
    ko.k = (int)std::min<int64_t>(10, n);
    const double t = std::sqrt(pm_chi2_upper_quantile(ko.alpha1, o.m));
    pmlsh_index *best = nullptr;
    double bestW = INFINITY;
    for (int M : cand) {
        if (M > n && best) break;
        o.leaf_size = M;
        pmlsh_index *ix = nullptr;
        pmlsh_status s = build_one(X, n, d, o, st, &ix);
        double W = 0.0;
        if (s == PMLSH_OK && n >= 2) {
            std::vector<double> F;
            s = pm_distance_sample(ix, std::min<int64_t>(65536, n * (n - 1)), o.seed + 6, F, st);
            const double R = t * pm_rmin_rule(ix, ko.beta, ko.k, ko.c);
            double cc = 0.0;
            if (s == PMLSH_OK) s = pm_cost_model(ix, F.data(), (int64_t)F.size(), &R, 1, &cc, nullptr, st);
            W = (double)ix->L + cc;
        }
        if (s != PMLSH_OK) {
            if (ix) pmlsh_free(ix);
            if (best) pmlsh_free(best);
            return s;
        }
        if (W < bestW) {
            if (best) pmlsh_free(best);
            best = ix;
            bestW = W;
        } else {
            pmlsh_free(ix);
        }
    }
    *out = best;
    return PMLSH_OK;
}

}  // namespace

pmlsh_status pmlsh_build(const float *X, int64_t n, int d, const pmlsh_build_opts *opts, void *stream,
                         pmlsh_index **out)
{
    PM_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    PM_CHECK(X != nullptr, "X is NULL");
    PM_CHECK(n >= 1 && n < (int64_t)1 << 31, "n must be in 1..2^31-1 (got %lld)", (long long)n);
    PM_CHECK(d >= 1 && d <= 65536, "d must be in 1..65536 (got %d)", d);
    pmlsh_build_opts o;
    if (opts) o = *opts;
    else pmlsh_build_opts_default(&o);
    PM_CHECK(o.m >= 1 && o.m <= PM_MP, "m must be in 1..16 (got %d)", o.m);
    PM_CHECK(o.s >= 0 && o.s <= PM_MAX_PIVOTS, "s must be in 0..8 (got %d)", o.s);
    PM_CHECK(o.leaf_size == 0 || o.leaf_size == -1 || (o.leaf_size >= 16 && o.leaf_size <= 1024),
             "leaf_size must be 0, -1 or 16..1024 (got %d)", o.leaf_size);
    PM_CHECK(o.rmin_pairs >= 0, "rmin_pairs must be >= 0");
    PM_CHECK(o.bf16_shadow == 0 || o.bf16_shadow == 1, "bf16_shadow must be 0 or 1");
    if (o.leaf_size == 0) return build_autotuned(X, n, d, o, (cudaStream_t)stream, out);
    if (o.leaf_size == -1) return build_model_tuned(X, n, d, o, (cudaStream_t)stream, out);
    return build_one(X, n, d, o, (cudaStream_t)stream, out);
}

void pmlsh_free(pmlsh_index *index)
{
    if (!index) return;
    pm_free_index(index);
    delete index;
}

pmlsh_status pmlsh_index_info(const pmlsh_index *ix, int64_t *n, int *d, int *m, int64_t *leaves,
                              int *leaf_size, int64_t *nodes)
{
    PM_CHECK(ix != nullptr, "index is NULL");
    if (n) *n = ix->n;
    if (d) *d = ix->d;
    if (m) *m = ix->m;
    if (leaves) *leaves = ix->L;
    if (leaf_size) *leaf_size = ix->M;
    if (nodes) *nodes = (int64_t)ix->nodeLo.size();
    return PMLSH_OK;
}

pmlsh_status pmlsh_get_projection(const pmlsh_index *ix, float *A_host)
{
    PM_CHECK(ix && A_host, "NULL argument");
    std::memcpy(A_host, ix->A_host.data(), ix->A_host.size() * sizeof(float));
    return PMLSH_OK;
}

pmlsh_status pmlsh_get_projected(const pmlsh_index *ix, double *O_host)
{
    PM_CHECK(ix && O_host, "NULL argument");
    std::vector<double> tmp((size_t)ix->n * PM_MP);
    PM_CUDA(cudaMemcpy(tmp.data(), ix->O64, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t pos = 0; pos < ix->n; pos++) {
        int64_t id = ix->permH[pos];
        for (int j = 0; j < ix->m; j++) O_host[id * ix->m + j] = tmp[(size_t)pos * PM_MP + j];
    }
    return PMLSH_OK;
}

pmlsh_status pmlsh_export_layout(const pmlsh_index *ix, int32_t *perm, int64_t *leaf_off, int64_t *node_lo,
                                 int64_t *node_hi, int32_t *node_left, int32_t *node_right)
{
    PM_CHECK(ix != nullptr, "index is NULL");
    if (perm) std::memcpy(perm, ix->permH.data(), ix->permH.size() * sizeof(int32_t));
    if (leaf_off) std::memcpy(leaf_off, ix->leafOffH.data(), ix->leafOffH.size() * sizeof(int64_t));
    size_t N = ix->nodeLo.size();
    if (node_lo) std::memcpy(node_lo, ix->nodeLo.data(), N * sizeof(int64_t));
    if (node_hi) std::memcpy(node_hi, ix->nodeHi.data(), N * sizeof(int64_t));
    if (node_left) std::memcpy(node_left, ix->nodeLeft.data(), N * sizeof(int32_t));
    if (node_right) std::memcpy(node_right, ix->nodeRight.data(), N * sizeof(int32_t));
    return PMLSH_OK;
}

pmlsh_status pmlsh_knn(pmlsh_index *ix, const float *Q, int64_t nq, const pmlsh_knn_opts *opts,
                       int64_t *out_ids, float *out_dists, float *out_err, pmlsh_query_stats *stats,
                       void *stream)
{
    PM_CHECK(ix != nullptr, "index is NULL");
    PM_CHECK(opts != nullptr, "opts is NULL");
    PM_CHECK(nq >= 0, "nq must be >= 0");
    if (nq == 0) return PMLSH_OK;
    PM_CHECK(Q && out_ids && out_dists, "NULL argument");
    const pmlsh_knn_opts &o = *opts;
    PM_CHECK(o.k >= 1 && o.k <= PM_MAX_K && o.k <= ix->n, "k must be in 1..min(n, %d) (got %d)",
             PM_MAX_K, o.k);
    PM_CHECK(o.c > 1.0 && std::isfinite(o.c), "c must be > 1 (got %g)", o.c);
    PM_CHECK(o.alpha1 > 0.0 && o.alpha1 < 1.0, "alpha1 must be in (0,1)");
    PM_CHECK(o.beta > 0.0 && o.beta <= 1.0, "beta must be in (0,1]");
    PM_CHECK(std::isfinite(o.r_min), "r_min must be finite");
    PM_CHECK(std::isfinite(o.t), "t must be finite");
    PM_CHECK(o.stop_rule == PMLSH_STOP_LITERAL || o.stop_rule == PMLSH_STOP_BC_CONSISTENT,
             "unknown stop_rule %d", o.stop_rule);
    PM_CHECK(o.precision >= 0 && o.precision <= PMLSH_BF16_RERANK, "unknown precision mode %d", o.precision);
    PM_CHECK(o.precision == PMLSH_FP32_PLAIN || (ix->Bsplit != nullptr && ix->Xr != nullptr),
             "BF16 precision modes need an index built with bf16_shadow = 1");
    return pm_knn(ix, Q, nq, &o, out_ids, out_dists, out_err, stats, (cudaStream_t)stream);
}

pmlsh_status pmlsh_rcbc(pmlsh_index *ix, const float *Q, int64_t nq, double r, const pmlsh_knn_opts *opts,
                        int64_t *out_ids, float *out_dists, pmlsh_query_stats *stats, void *stream)
{
    PM_CHECK(ix != nullptr, "index is NULL");
    PM_CHECK(opts != nullptr, "opts is NULL");
    PM_CHECK(nq >= 0, "nq must be >= 0");
    if (nq == 0) return PMLSH_OK;
    PM_CHECK(Q && out_ids && out_dists, "NULL argument");
    PM_CHECK(r > 0.0 && std::isfinite(r), "r must be > 0 and finite (got %g)", r);
    pmlsh_knn_opts o = *opts;
    PM_CHECK(o.c > 1.0 && std::isfinite(o.c), "c must be > 1 (got %g)", o.c);
    PM_CHECK(o.alpha1 > 0.0 && o.alpha1 < 1.0, "alpha1 must be in (0,1)");
    PM_CHECK(o.beta > 0.0 && o.beta <= 1.0, "beta must be in (0,1]");
    PM_CHECK(std::isfinite(o.t), "t must be finite");
    PM_CHECK(o.precision >= 0 && o.precision <= PMLSH_BF16_RERANK, "unknown precision mode %d", o.precision);
    PM_CHECK(o.precision == PMLSH_FP32_PLAIN || (ix->Bsplit != nullptr && ix->Xr != nullptr),
             "BF16 precision modes need an index built with bf16_shadow = 1");
    o.k = 1;
    o.r_min = r;
    o.stop_rule = PMLSH_STOP_LITERAL;
    return pm_knn(ix, Q, nq, &o, out_ids, out_dists, nullptr, stats, (cudaStream_t)stream, nullptr, true);
}

void pmlsh_cp_opts_default(pmlsh_cp_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k = 10;
    o->c = 1.5;
    o->alpha1 = 0.36787944117144233;
    o->alpha2 = 0.0024;   // Sec. 7.1
    o->T = 0;
    o->gamma = 0.0;
    o->t = 0.0;
}

pmlsh_status pmlsh_closest_pair(pmlsh_index *ix, const pmlsh_cp_opts *opts, int64_t *out_pairs, float *out_dists,
                                pmlsh_cp_stats *stats, void *stream)
{
    PM_CHECK(ix && opts && out_pairs && out_dists, "NULL argument");
    const pmlsh_cp_opts &o = *opts;
    const int64_t npairs = ix->n * (ix->n - 1) / 2;
    PM_CHECK(ix->n >= 2, "closest pairs need n >= 2");
    PM_CHECK(o.k >= 1 && o.k <= 1024 && o.k <= npairs, "k must be in 1..min(n(n-1)/2, 1024) (got %d)", o.k);
    PM_CHECK(o.c > 1.0, "c must be > 1");
    PM_CHECK(!std::isnan(o.gamma), "gamma must not be NaN (<= 0: calibrated, Sec. 6.3)");
    PM_CHECK(o.t > 0.0 || (o.alpha1 > 0.0 && o.alpha1 < 1.0), "alpha1 must be in (0,1)");
    PM_CHECK(o.T > 0 || (o.alpha2 > 0.0 && o.alpha2 <= 1.0), "alpha2 must be in (0,1]");
    return pm_closest_pair(ix, &o, out_pairs, out_dists, stats, (cudaStream_t)stream);
}

pmlsh_status pmlsh_rmin(const pmlsh_index *ix, double beta, int k, double c, double *r_min)
{
    PM_CHECK(ix && r_min, "NULL argument");
    PM_CHECK(beta > 0.0 && beta <= 1.0 && k >= 1 && c > 1.0, "beta must be in (0,1], k >= 1, c > 1");
    *r_min = pm_rmin_rule(ix, beta, k, c);
    return PMLSH_OK;
}

pmlsh_status pmlsh_knn_workspace_bytes(pmlsh_index *ix, int64_t nq, int k, int precision, int64_t *bytes)
{
    PM_CHECK(ix && bytes, "NULL argument");
    PM_CHECK(nq >= 0 && k >= 1 && k <= PM_MAX_K, "nq must be >= 0 and k in 1..256");
    *bytes = pm_knn_work_bytes(ix, nq, k, precision);
    return PMLSH_OK;
}

pmlsh_status pmlsh_gamma_calibrate(pmlsh_index *ix, double pr, int64_t nsample, uint64_t seed, double *gamma,
                                   void *stream)
{
    PM_CHECK(ix && gamma, "NULL argument");
    PM_CHECK(ix->n >= 2, "gamma calibration needs n >= 2");
    PM_CHECK(pr > 0.0 && pr <= 1.0, "pr must be in (0, 1]");
    PM_CHECK(nsample >= 2 && nsample <= 32768, "nsample must be in 2..32768 (got %lld)", (long long)nsample);
    return pm_gamma_calibrate(ix, pr, nsample, seed, gamma, (cudaStream_t)stream);
}

pmlsh_status pmlsh_closest_pair_bnb(pmlsh_index *ix, const pmlsh_cp_opts *opts, int64_t *out_pairs,
                                    float *out_dists, pmlsh_cp_stats *stats, void *stream)
{
    PM_CHECK(ix && opts && out_pairs && out_dists, "NULL argument");
    const pmlsh_cp_opts &o = *opts;
    const int64_t npairs = ix->n * (ix->n - 1) / 2;
    PM_CHECK(ix->n >= 2, "closest pairs need n >= 2");
    PM_CHECK(o.k >= 1 && o.k <= 1024 && o.k <= npairs, "k must be in 1..min(n(n-1)/2, 1024) (got %d)", o.k);
    PM_CHECK(o.T > 0 || (o.alpha2 > 0.0 && o.alpha2 <= 1.0), "alpha2 must be in (0,1]");
    return pm_closest_pair_bnb(ix, &o, out_pairs, out_dists, stats, (cudaStream_t)stream);
}

pmlsh_status pmlsh_project(pmlsh_index *ix, const float *Q, int64_t nq, double *out64, float *out32,
                           void *stream)
{
    PM_CHECK(ix != nullptr, "index is NULL");
    PM_CHECK(nq >= 0, "nq must be >= 0");
    if (nq == 0) return PMLSH_OK;
    PM_CHECK(Q != nullptr && (out64 || out32), "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const bool d64 = !out64 || pm_is_device_ptr(out64), d32 = !out32 || pm_is_device_ptr(out32);
    KnnWork &w = ix->work;
    PM_TRY(w.Qd.reserve((size_t)nq * ix->ld * sizeof(float)));
    double *o64 = out64;
    float *o32 = out32;
    size_t n64 = out64 ? (size_t)nq * ix->m : 0, n32 = out32 ? (size_t)nq * ix->m : 0;
    if (!d64 || !d32) {
        PM_TRY(w.qp64.reserve(std::max<size_t>(n64, 1) * sizeof(double)));
        PM_TRY(w.qp32.reserve(std::max<size_t>(n32, 1) * sizeof(float)));
        if (out64 && !d64) o64 = w.qp64.as<double>();
        if (out32 && !d32) o32 = w.qp32.as<float>();
    }
    PM_TRY(pm_project_rows(ix, Q, nq, w.Qd.as<float>(), o64, o32, ix->m, st));
    if (out64 && !d64) PM_CUDA(cudaMemcpyAsync(out64, o64, n64 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (out32 && !d32) PM_CUDA(cudaMemcpyAsync(out32, o32, n32 * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d64 || !d32) PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}

}  // extern "C"
