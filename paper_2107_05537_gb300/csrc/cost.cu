// Cost model of the PM-tree (Sec. 4.2) on the flat leaf layout.
//
// F(x) = Pr[||o_i, o_j|| <= x] is the distance distribution of the indexed
// points in the projected space, estimated by the empirical CDF of sampled
// pairs.  A leaf e is accessed by range(q, r_q) iff the Eq. 5 conditions hold
// (||q, e.RO|| <= e.r + r_q and, for each pivot, ||q, p_i|| - r_q <=
// e.HR[i].max and ||q, p_i|| + r_q >= e.HR[i].min); taking F for the
// distribution of each of those query distances,
//   Pr[e] = F(e.r + r_q) * prod_i (F(e.HR[i].max + r_q) - F(e.HR[i].min - r_q)),
//   CC(range(q, r_q)) = sum_e N(e) Pr[e],
// the expected number of points in accessed leaves.  The entries are the
// index's own (FP32 centre, radius and rings, widened to FP64).
#include <algorithm>
#include <cmath>
#include <vector>

#include "pmlsh_impl.h"

namespace {

// position of each id: inv[perm[p]] = p
__global__ void k_inv_perm(const int32_t *__restrict__ perm, int64_t n, int32_t *__restrict__ inv)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t id = perm[p];
    if (id >= 0 && id < n) inv[id] = (int32_t)p;
}

// Pair s: ids i = v_{2s} mod n, j = v_{2s+1} mod n of the counter stream
// `seed` (j = i moved to i + 1 mod n, as the Sec. 5.2 radius rule draws its
// pairs), FP64 projected distance with the sequential sum.
__global__ void k_dist_sample(const double *__restrict__ O64, const int32_t *__restrict__ inv, int64_t n, int m,
                              uint64_t seed, int64_t np, double *__restrict__ out)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int64_t i = (int64_t)(pm_splitmix64_hd(seed, 2 * (uint64_t)s) % (uint64_t)n);
    int64_t j = (int64_t)(pm_splitmix64_hd(seed, 2 * (uint64_t)s + 1) % (uint64_t)n);
    if (j == i) j = (j + 1) % n;
    const int32_t pi = inv[i], pj = inv[j];
    if (pi < 0 || pi >= n || pj < 0 || pj >= n) {
        out[s] = NAN;
        return;
    }
    out[s] = pm_pdist64(O64 + (int64_t)pi * PM_MP, O64 + (int64_t)pj * PM_MP, m);
}

// empirical CDF: the fraction of the sorted sample F[0, nF) that is <= x
__device__ double ecdf(const double *__restrict__ F, int64_t nF, double x)
{
    int64_t lo = 0, hi = nF;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (F[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return (double)lo / (double)nF;
}

constexpr int COST_THREADS = 256;

// One block per radius: Pr[e] for every leaf, CC and sum Pr[e] by a
// fixed-order tree reduction.  out[2 r] = CC, out[2 r + 1] = sum Pr[e].
__global__ void __launch_bounds__(COST_THREADS)
k_cost_model(const float *__restrict__ meta, const int64_t *__restrict__ off, int64_t L, int s,
             const double *__restrict__ F, int64_t nF, const double *__restrict__ rq, double *__restrict__ out)
{
    __shared__ double scc[COST_THREADS], sen[COST_THREADS];
    const double r = rq[blockIdx.x];
    double cc = 0.0, en = 0.0;
    for (int64_t l = threadIdx.x; l < L; l += COST_THREADS) {
        const float *M = meta + l * PM_LEAF_STRIDE;
        double pr = ecdf(F, nF, __dadd_rn((double)M[16], r));
        for (int i = 0; i < s; i++) {
            const double hi = ecdf(F, nF, __dadd_rn((double)M[32 + i], r));
            const double lo = ecdf(F, nF, __dsub_rn((double)M[24 + i], r));
            pr = __dmul_rn(pr, __dsub_rn(hi, lo));
        }
        cc = __dadd_rn(cc, __dmul_rn((double)(off[l + 1] - off[l]), pr));
        en = __dadd_rn(en, pr);
    }
    scc[threadIdx.x] = cc;
    sen[threadIdx.x] = en;
    __syncthreads();
    for (int w = COST_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            scc[threadIdx.x] = __dadd_rn(scc[threadIdx.x], scc[threadIdx.x + w]);
            sen[threadIdx.x] = __dadd_rn(sen[threadIdx.x], sen[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = scc[0];
        out[2 * blockIdx.x + 1] = sen[0];
    }
}

template <class T> struct DevTmp {
    T *p = nullptr;
    ~DevTmp() { cudaFree(p); }
    pmlsh_status alloc(size_t count)
    {
        PM_CUDA(cudaMalloc((void **)&p, std::max<size_t>(1, count) * sizeof(T)));
        return PMLSH_OK;
    }
};

}  // namespace

pmlsh_status pm_distance_sample(const pmlsh_index *ix, int64_t npairs, uint64_t seed, std::vector<double> &out,
                                cudaStream_t st)
{
    const int64_t n = ix->n;
    DevTmp<int32_t> inv;
    DevTmp<double> v;
    PM_TRY(inv.alloc((size_t)n));
    PM_TRY(v.alloc((size_t)npairs));
    PM_CUDA(cudaMemsetAsync(inv.p, 0xff, (size_t)n * sizeof(int32_t), st));
    PM_LAUNCH("k_inv_perm", st, k_inv_perm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ix->perm, n, inv.p));
    PM_LAUNCH("k_dist_sample", st,
              k_dist_sample<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(ix->O64, inv.p, n, ix->m, seed,
                                                                              npairs, v.p));
    PM_CUDA(cudaGetLastError());
    out.resize((size_t)npairs);
    PM_CUDA(cudaMemcpyAsync(out.data(), v.p, (size_t)npairs * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    for (double x : out) {
        if (!(x >= 0.0)) {
            pm_set_error("distance sample: position lookup failed");
            return PMLSH_EINTERNAL;
        }
    }
    std::sort(out.begin(), out.end());
    return PMLSH_OK;
}

pmlsh_status pm_cost_model(const pmlsh_index *ix, const double *F, int64_t nF, const double *rq, int64_t nr,
                           double *cc, double *nodes, cudaStream_t st)
{
    if (nr == 0) return PMLSH_OK;
    DevTmp<double> Fd, rd, od;
    PM_TRY(Fd.alloc((size_t)nF));
    PM_TRY(rd.alloc((size_t)nr));
    PM_TRY(od.alloc((size_t)nr * 2));
    PM_CUDA(cudaMemcpyAsync(Fd.p, F, (size_t)nF * sizeof(double), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(rd.p, rq, (size_t)nr * sizeof(double), cudaMemcpyHostToDevice, st));
    PM_LAUNCH("k_cost_model", st,
              k_cost_model<<<(unsigned)nr, COST_THREADS, 0, st>>>(ix->leafMeta, ix->leafOff, ix->L, ix->s, Fd.p,
                                                                  nF, rd.p, od.p));
    PM_CUDA(cudaGetLastError());
    std::vector<double> o((size_t)nr * 2);
    PM_CUDA(cudaMemcpyAsync(o.data(), od.p, o.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    for (int64_t r = 0; r < nr; r++) {
        if (cc) cc[r] = o[2 * r];
        if (nodes) nodes[r] = o[2 * r + 1];
    }
    return PMLSH_OK;
}

// Sec. 5.2: r* is the lower (beta n + k)/n quantile of the sampled
// original-space distances, r_min = r* / c (the query path uses the same rule).
double pm_rmin_rule(const pmlsh_index *ix, double beta, int64_t k, double c)
{
    const std::vector<double> &v = ix->distSample;
    if (v.empty()) return 1.0;
    const double p = std::min(1.0, (beta * (double)ix->n + (double)k) / (double)ix->n);
    const int64_t N = (int64_t)v.size();
    int64_t rank = (int64_t)std::ceil(p * (double)N - 1e-9);
    rank = std::max<int64_t>(1, std::min<int64_t>(N, rank));
    double rstar = v[rank - 1];
    if (!(rstar > 0.0)) {
        rstar = 0.0;
        for (double x : v) if (x > 0.0) { rstar = x; break; }
    }
    return rstar > 0.0 ? rstar / c : 1.0;
}

extern "C" {

pmlsh_status pmlsh_distance_sample(const pmlsh_index *ix, int64_t npairs, uint64_t seed, double *out_sorted,
                                   void *stream)
{
    if (!ix || !out_sorted) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    if (ix->n < 2 || npairs < 1 || npairs > ((int64_t)1 << 28)) {
        pm_set_error("distance sample needs n >= 2 and 1 <= npairs <= 2^28 (n %lld, npairs %lld)",
                     (long long)ix->n, (long long)npairs);
        return PMLSH_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> v;
    PM_TRY(pm_distance_sample(ix, npairs, seed, v, st));
    const cudaMemcpyKind kind = pm_is_device_ptr(out_sorted) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    PM_CUDA(cudaMemcpyAsync(out_sorted, v.data(), v.size() * sizeof(double), kind, st));
    PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}

pmlsh_status pmlsh_cost_model(const pmlsh_index *ix, const double *F_sorted, int64_t nF, const double *rq,
                              int64_t nr, double *out_cc, double *out_nodes, void *stream)
{
    if (!ix || !F_sorted || (nr > 0 && !rq)) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    if (nF < 1 || nF > ((int64_t)1 << 28) || nr < 0 || nr > 65535) {
        pm_set_error("cost model needs 1 <= nF <= 2^28 and 0 <= nr <= 65535 (nF %lld, nr %lld)",
                     (long long)nF, (long long)nr);
        return PMLSH_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> F((size_t)nF), R((size_t)nr), cc((size_t)nr), en((size_t)nr);
    PM_CUDA(cudaMemcpyAsync(F.data(), F_sorted, F.size() * sizeof(double), cudaMemcpyDefault, st));
    if (nr > 0) PM_CUDA(cudaMemcpyAsync(R.data(), rq, R.size() * sizeof(double), cudaMemcpyDefault, st));
    PM_CUDA(cudaStreamSynchronize(st));
    for (int64_t e = 0; e < nF; e++) {
        if (!std::isfinite(F[e]) || (e > 0 && F[e] < F[e - 1])) {
            pm_set_error("F_sorted must be finite and ascending (entry %lld)", (long long)e);
            return PMLSH_EINVAL;
        }
    }
    for (int64_t r = 0; r < nr; r++) {
        if (!(R[r] >= 0.0)) {
            pm_set_error("rq must be >= 0 (entry %lld)", (long long)r);
            return PMLSH_EINVAL;
        }
    }
    PM_TRY(pm_cost_model(ix, F.data(), nF, R.data(), nr, cc.data(), en.data(), st));
    if (nr > 0 && out_cc)
        PM_CUDA(cudaMemcpyAsync(out_cc, cc.data(), cc.size() * sizeof(double), cudaMemcpyDefault, st));
    if (nr > 0 && out_nodes)
        PM_CUDA(cudaMemcpyAsync(out_nodes, en.data(), en.size() * sizeof(double), cudaMemcpyDefault, st));
    PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}

pmlsh_status pmlsh_export_leaf_entries(const pmlsh_index *ix, int *s, float *centre, float *radius,
                                       float *ring_min, float *ring_max, float *pivots)
{
    if (!ix) {
        pm_set_error("index is NULL");
        return PMLSH_EINVAL;
    }
    const int64_t L = ix->L;
    const int m = ix->m, ns = ix->s;
    if (s) *s = ns;
    std::vector<float> meta((size_t)L * PM_LEAF_STRIDE), piv((size_t)PM_MAX_PIVOTS * PM_MP);
    PM_CUDA(cudaMemcpy(meta.data(), ix->leafMeta, meta.size() * sizeof(float), cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(piv.data(), ix->piv32, piv.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (int64_t l = 0; l < L; l++) {
        const float *M = meta.data() + (size_t)l * PM_LEAF_STRIDE;
        for (int j = 0; j < m && centre; j++) centre[l * m + j] = M[j];
        if (radius) radius[l] = M[16];
        for (int i = 0; i < ns; i++) {
            if (ring_min) ring_min[l * ns + i] = M[24 + i];
            if (ring_max) ring_max[l * ns + i] = M[32 + i];
        }
    }
    for (int i = 0; i < ns && pivots; i++)
        for (int j = 0; j < m; j++) pivots[i * m + j] = piv[(size_t)i * PM_MP + j];
    return PMLSH_OK;
}

}  // extern "C"
