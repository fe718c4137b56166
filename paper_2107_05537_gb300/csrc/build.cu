// Index build: projection (Eq. 3), leaf layout (the flattened stand-in for
// the PM-tree of Sec. 4.1), leaf balls and pivot rings, distance sample for
// the r_min rule of Sec. 5.2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "pmlsh_impl.h"

namespace {

// ---------------------------------------------------------------- kernels

// o'[p][j] = sum_i A[j][i] x[p][i] in FP64, sequential in i.  Products of two
// FP32 values are exact in FP64, so fma(a, x, s) equals the separately
// rounded multiply-then-add.  Rows are staged through shared memory in
// 32-column chunks so that global loads are coalesced.
constexpr int PROJ_PTS = 128;
__global__ void __launch_bounds__(PROJ_PTS)
k_project64(const float *__restrict__ X, int64_t n, int ld, int d, int m,
            const float *__restrict__ A, double *__restrict__ O64,
            float *__restrict__ O32, int ostride, unsigned long long *maxNormBits)
{
    __shared__ float As[PM_MP][33];
    __shared__ float Xs[PROJ_PTS][33];
    const int64_t p0 = (int64_t)blockIdx.x * PROJ_PTS;
    const int64_t p = p0 + threadIdx.x;
    double acc[PM_MP];
#pragma unroll
    for (int j = 0; j < PM_MP; j++) acc[j] = 0.0;
    for (int c0 = 0; c0 < d; c0 += 32) {
        __syncthreads();
        // cooperative, coalesced load of 128 rows x 32 columns (and A's chunk)
        for (int e = threadIdx.x; e < PROJ_PTS * 32; e += blockDim.x) {
            int r = e >> 5, c = e & 31;
            int64_t pp = p0 + r;
            float v = 0.f;
            if (pp < n && c0 + c < ld) v = X[pp * ld + c0 + c];
            Xs[r][c] = v;
        }
        for (int e = threadIdx.x; e < PM_MP * 32; e += blockDim.x) {
            int r = e >> 5, c = e & 31;
            As[r][c] = (c0 + c < ld) ? A[r * ld + c0 + c] : 0.f;
        }
        __syncthreads();
        const int cend = min(32, d - c0);
        for (int c = 0; c < cend; c++) {
            double xv = (double)Xs[threadIdx.x][c];
#pragma unroll
            for (int j = 0; j < PM_MP; j++)
                if (j < m) acc[j] = __fma_rn((double)As[j][c], xv, acc[j]);
        }
    }
    if (p >= n) return;
    double nn = 0.0;
#pragma unroll
    for (int j = 0; j < PM_MP; j++) {
        if (j < ostride) {
            if (O64) O64[p * ostride + j] = acc[j];
            if (O32) O32[p * ostride + j] = __double2float_rn(acc[j]);
        }
        nn = __fma_rn(acc[j], acc[j], nn);
    }
    if (maxNormBits) atomicMax(maxNormBits, (unsigned long long)__double_as_longlong(sqrt(nn)));
}

// Gathers rows into leaf order: dst[pos] = src[perm[pos]].
template <class T>
__global__ void k_gather_rows(const T *__restrict__ src, T *__restrict__ dst,
                              const int32_t *__restrict__ perm, int64_t n, int width)
{
    int64_t total = n * width;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t pos = e / width;
        int c = (int)(e - pos * width);
        dst[e] = src[(int64_t)perm[pos] * width + c];
    }
}

__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Leaf ball: centre = midpoint of the FP64 bounding box, radius = largest
// FP64 distance to it; then a radius that also covers the FP32 copies of
// the coordinates (each coordinate is within 2^-24 relative of its FP64
// value).  One block (256 threads) per leaf.
__global__ void k_leaf_ball(const double *__restrict__ O64, const int64_t *__restrict__ off,
                            int m, double maxNorm, float *__restrict__ meta,
                            double *__restrict__ ro64)
{
    __shared__ double smn[8][PM_MP], smx[8][PM_MP], sro[PM_MP], srad[8];
    const int64_t l = blockIdx.x;
    const int64_t a = off[l], b = off[l + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < PM_MP; j++) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
            double v = O64[e * PM_MP + j];
            mn = fmin(mn, v);
            mx = fmax(mx, v);
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) { smn[warp][j] = mn; smx[warp][j] = mx; }
    }
    __syncthreads();
    if (threadIdx.x < PM_MP) {
        int j = threadIdx.x;
        double mn = smn[0][j], mx = smx[0][j];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            mn = fmin(mn, smn[w][j]);
            mx = fmax(mx, smx[w][j]);
        }
        sro[j] = j < m ? __dmul_rn(0.5, __dadd_rn(mn, mx)) : 0.0;
    }
    __syncthreads();
    double rad = 0.0;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x)
        rad = fmax(rad, pm_pdist64(O64 + e * PM_MP, sro, m));
    rad = warp_max(rad);
    if (lane == 0) srad[warp] = rad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0, rn = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) r = fmax(r, srad[w]);
        for (int j = 0; j < PM_MP; j++) rn = fma(sro[j], sro[j], rn);
        double rr = (r + 0x1.0p-23 * (sqrt(rn) + maxNorm)) * (1.0 + 1e-6);
        float *M = meta + l * PM_LEAF_STRIDE;
        for (int j = 0; j < PM_MP; j++) M[j] = __double2float_rn(sro[j]);
        M[16] = __double2float_ru(rr);
        for (int j = 0; j < PM_MP; j++) ro64[l * PM_MP + j] = sro[j];
    }
}

// Pivot rings e.HR[i] = [min, max] of ||o', p_i|| over the leaf, taken on the
// FP32 coordinates and widened by 1e-5 relative so that they bound the exact
// distances of the FP32 coordinates.
__global__ void k_leaf_rings(const float *__restrict__ O32, const int64_t *__restrict__ off,
                             const float *__restrict__ piv, int s, float *__restrict__ meta)
{
    __shared__ float smn[8][PM_MAX_PIVOTS], smx[8][PM_MAX_PIVOTS];
    const int64_t l = blockIdx.x;
    const int64_t a = off[l], b = off[l + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = 0; i < s; i++) {
        float mn = INFINITY, mx = 0.f;
        for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
            float v = sqrtf(pm_pd2_32(O32 + e * PM_MP, piv + i * PM_MP));
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        for (int o = 16; o; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) { smn[warp][i] = mn; smx[warp][i] = mx; }
    }
    __syncthreads();
    if (threadIdx.x < s) {
        int i = threadIdx.x;
        float mn = smn[0][i], mx = smx[0][i];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            mn = fminf(mn, smn[w][i]);
            mx = fmaxf(mx, smx[w][i]);
        }
        float *M = meta + l * PM_LEAF_STRIDE;
        M[24 + i] = mn * (1.f - 1e-5f);
        M[32 + i] = mx * (1.f + 1e-5f);
    }
}

// FP64 distances of the sampled pairs (r_min rule), original point order.
__global__ void k_sample_dist(const float *__restrict__ X, int ld, int d,
                              const int64_t *__restrict__ pi, const int64_t *__restrict__ pj,
                              int64_t cnt, double *__restrict__ out)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= cnt) return;
    out[s] = pm_dist64(X + pi[s] * ld, X + pj[s] * ld, d);
}

}  // namespace

void pm_launch_project64(const float *X, int64_t n, int ld, int d, int m, const float *A,
                         double *O64, float *O32, unsigned long long *maxNormBits,
                         cudaStream_t st, int ostride)
{
    if (n <= 0) return;
    int grid = (int)((n + PROJ_PTS - 1) / PROJ_PTS);
    PM_LAUNCH("k_project64", st, k_project64<<<grid, PROJ_PTS, 0, st>>>(X, n, ld, d, m, A, O64, O32, ostride, maxNormBits));
}

// The same launch without the profiler's bookkeeping (which may create CUDA
// events); used by the no-allocation entry point.
void pm_launch_project64_noprof(const float *X, int64_t n, int ld, int d, int m, const float *A,
                                double *O64, float *O32, cudaStream_t st, int ostride)
{
    if (n <= 0) return;
    int grid = (int)((n + PROJ_PTS - 1) / PROJ_PTS);
    k_project64<<<grid, PROJ_PTS, 0, st>>>(X, n, ld, d, m, A, O64, O32, ostride, nullptr);
}

namespace {

// ------------------------------------------------------------ host layout

struct Bisect {
    const float *O;   // [n][16] FP32 coordinates, original order
    int m, M;
    std::vector<int32_t> perm;
    std::vector<int64_t> leafOff;
    std::vector<int64_t> nlo, nhi;
    std::vector<int32_t> nl, nr, ndim;
    std::vector<float> nval;

    // Splits positions [lo, hi) of perm; returns the node id.
    int32_t split(int64_t lo, int64_t hi)
    {
        int32_t id = (int32_t)nlo.size();
        nlo.push_back((int64_t)leafOff.size() - 1);
        nhi.push_back(-1);
        nl.push_back(-1);
        nr.push_back(-1);
        ndim.push_back(-1);
        nval.push_back(0.f);
        int64_t size = hi - lo;
        if (size <= M) {
            std::sort(perm.begin() + lo, perm.begin() + hi);
            leafOff.push_back(hi);
            nhi[id] = (int64_t)leafOff.size() - 1;
            return id;
        }
        // split dimension: largest extent of the projected points
        int best = 0;
        float bestExt = -1.f;
        for (int j = 0; j < m; j++) {
            float mn = INFINITY, mx = -INFINITY;
            for (int64_t e = lo; e < hi; e++) {
                float v = O[(int64_t)perm[e] * PM_MP + j];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            if (mx - mn > bestExt) { bestExt = mx - mn; best = j; }
        }
        // balanced: the left part holds ceil(leaves/2) full leaves
        int64_t leaves = (size + M - 1) / M;
        int64_t left = ((leaves + 1) / 2) * M;
        const float *O_ = O;
        const int dim = best;
        std::nth_element(perm.begin() + lo, perm.begin() + lo + left, perm.begin() + hi,
                         [O_, dim](int32_t a, int32_t b) {
                             float va = O_[(int64_t)a * PM_MP + dim], vb = O_[(int64_t)b * PM_MP + dim];
                             return va < vb || (va == vb && a < b);
                         });
        ndim[id] = dim;
        nval[id] = O_[(int64_t)perm[lo + left] * PM_MP + dim];
        int32_t L = split(lo, lo + left);
        int32_t R = split(lo + left, hi);
        nl[id] = L;
        nr[id] = R;
        nhi[id] = (int64_t)leafOff.size() - 1;
        return id;
    }
};

template <class T> pmlsh_status dalloc(T **p, size_t count)
{
    PM_CUDA(cudaMalloc((void **)p, std::max<size_t>(1, count) * sizeof(T)));
    return PMLSH_OK;
}

}  // namespace

void pm_free_index(pmlsh_index *ix)
{
    cudaFree(ix->X);
    cudaFree(ix->perm);
    cudaFree(ix->O32);
    cudaFree(ix->O64);
    cudaFree(ix->A32);
    cudaFree(ix->leafOff);
    cudaFree(ix->leafMeta);
    cudaFree(ix->piv32);
    cudaFree(ix->treeI);
    cudaFree(ix->treeV);
    KnnWork &w = ix->work;
    DevBuf *bufs[] = {&w.Qd, &w.qp32, &w.qp64, &w.qnorm, &w.qpiv, &w.order, &w.keys,
                      &w.keys2, &w.vals2, &w.sortTmp, &w.qstate, &w.thr, &w.blkCnt,
                      &w.blkLeaves, &w.cntSure, &w.cntBand, &w.bandQ, &w.bandPos,
                      &w.bandIn, &w.bandCnt, &w.partD, &w.partI, &w.partSeen, &w.bandInQ,
                      &w.outD64, &w.outIds, &w.outErr, &w.dk, &w.flags, &w.selBuf,
                      &w.selOff, &w.selCnt, &w.selTau, &w.active, &w.misc};
    for (DevBuf *b : bufs) b->release();
}

pmlsh_status DevBuf::reserve(size_t b)
{
    if (b <= bytes) return PMLSH_OK;
    release();
    size_t nb = std::max<size_t>(b, 256);
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
        p = nullptr;
        pm_set_error("cudaMalloc(%zu) failed: %s", nb, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PMLSH_ENOMEM : PMLSH_ECUDA;
    }
    bytes = nb;
    return PMLSH_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

pmlsh_status pm_build_index(pmlsh_index *ix, const float *X, bool x_on_device,
                            const pmlsh_build_opts *o, cudaStream_t st)
{
    const int64_t n = ix->n;
    const int d = ix->d;
    const int ld = ix->ld;
    const int m = ix->m;
    // 1. padded, original-order device copy of X
    float *Xo = nullptr;
    PM_TRY(dalloc(&Xo, (size_t)n * ld));
    struct Guard { float *p; ~Guard() { cudaFree(p); } } g{Xo};
    PM_CUDA(cudaMemsetAsync(Xo, 0, (size_t)n * ld * sizeof(float), st));
    PM_CUDA(cudaMemcpy2DAsync(Xo, ld * sizeof(float), X, d * sizeof(float), d * sizeof(float), n,
                              x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // 2. projection matrix
    ix->A_host.assign((size_t)m * d, 0.f);
    if (o->proj) {
        PM_CUDA(cudaMemcpy(ix->A_host.data(), o->proj, sizeof(float) * m * d,
                           pm_is_device_ptr(o->proj) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    } else {
        pm_gaussian_projection(ix->seed + 2, m, d, ix->A_host.data());
    }
    std::vector<float> Apad((size_t)PM_MP * ld, 0.f);
    for (int j = 0; j < m; j++)
        for (int i = 0; i < d; i++) Apad[(size_t)j * ld + i] = ix->A_host[(size_t)j * d + i];
    PM_TRY(dalloc(&ix->A32, Apad.size()));
    PM_CUDA(cudaMemcpyAsync(ix->A32, Apad.data(), Apad.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    // 3. projection, FP64 and FP32, original order
    double *O64o = nullptr;
    float *O32o = nullptr;
    unsigned long long *mx = nullptr;
    PM_TRY(dalloc(&O64o, (size_t)n * PM_MP));
    struct G2 { double *a; float *b; unsigned long long *c; ~G2() { cudaFree(a); cudaFree(b); cudaFree(c); } } g2{O64o, nullptr, nullptr};
    PM_TRY(dalloc(&O32o, (size_t)n * PM_MP));
    g2.b = O32o;
    PM_TRY(dalloc(&mx, 1));
    g2.c = mx;
    PM_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    {
        pm_launch_project64(Xo, n, ld, d, m, ix->A32, O64o, O32o, mx, st);
        PM_CUDA(cudaGetLastError());
    }
    // 4. distance sample for r_min (Sec. 5.2), stream seed+3, original order
    {
        int64_t np = o->rmin_pairs > 0 ? o->rmin_pairs : 10000;
        ix->distSample.clear();
        if (n >= 2) {
            std::vector<int64_t> pi(np), pj(np);
            for (int64_t s = 0; s < np; s++) {
                int64_t i = (int64_t)(pm_splitmix64(ix->seed + 3, 2 * (uint64_t)s) % (uint64_t)n);
                int64_t j = (int64_t)(pm_splitmix64(ix->seed + 3, 2 * (uint64_t)s + 1) % (uint64_t)n);
                if (j == i) j = (j + 1) % n;
                pi[s] = i;
                pj[s] = j;
            }
            int64_t *dpi = nullptr, *dpj = nullptr;
            double *dout = nullptr;
            PM_TRY(dalloc(&dpi, np));
            struct G3 { int64_t *a, *b; double *c; ~G3() { cudaFree(a); cudaFree(b); cudaFree(c); } } g3{dpi, nullptr, nullptr};
            PM_TRY(dalloc(&dpj, np));
            g3.b = dpj;
            PM_TRY(dalloc(&dout, np));
            g3.c = dout;
            PM_CUDA(cudaMemcpyAsync(dpi, pi.data(), np * 8, cudaMemcpyHostToDevice, st));
            PM_CUDA(cudaMemcpyAsync(dpj, pj.data(), np * 8, cudaMemcpyHostToDevice, st));
            PM_LAUNCH("k_sample_dist", st, k_sample_dist<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(Xo, ld, d, dpi, dpj, np, dout));
            PM_CUDA(cudaGetLastError());
            ix->distSample.resize(np);
            PM_CUDA(cudaMemcpyAsync(ix->distSample.data(), dout, np * 8, cudaMemcpyDeviceToHost, st));
            PM_CUDA(cudaStreamSynchronize(st));
            std::sort(ix->distSample.begin(), ix->distSample.end());
        }
    }
    // 5. leaf layout by recursive bisection of the projected points (host)
    std::vector<float> O32h((size_t)n * PM_MP);
    unsigned long long mxh = 0;
    PM_CUDA(cudaMemcpyAsync(O32h.data(), O32o, O32h.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaMemcpyAsync(&mxh, mx, sizeof(mxh), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    {
        double mn;
        std::memcpy(&mn, &mxh, sizeof(mn));
        ix->maxNorm = mn;
    }
    Bisect bs;
    bs.O = O32h.data();
    bs.m = m;
    bs.M = ix->M;
    bs.perm.resize(n);
    std::iota(bs.perm.begin(), bs.perm.end(), 0);
    bs.leafOff.push_back(0);
    bs.split(0, n);
    ix->permH = std::move(bs.perm);
    ix->leafOffH = std::move(bs.leafOff);
    ix->nodeLo = std::move(bs.nlo);
    ix->nodeHi = std::move(bs.nhi);
    ix->nodeLeft = std::move(bs.nl);
    ix->nodeRight = std::move(bs.nr);
    ix->nodeDim = std::move(bs.ndim);
    ix->nodeVal = std::move(bs.nval);
    {
        size_t N = ix->nodeLo.size();
        std::vector<int32_t> ti(N * 4);
        for (size_t e = 0; e < N; e++) {
            ti[e * 4 + 0] = ix->nodeLeft[e];
            ti[e * 4 + 1] = ix->nodeRight[e];
            ti[e * 4 + 2] = ix->nodeDim[e];
            ti[e * 4 + 3] = (int32_t)ix->nodeLo[e];
        }
        PM_TRY(dalloc(&ix->treeI, ti.size()));
        PM_TRY(dalloc(&ix->treeV, N));
        PM_CUDA(cudaMemcpyAsync(ix->treeI, ti.data(), ti.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaMemcpyAsync(ix->treeV, ix->nodeVal.data(), N * sizeof(float), cudaMemcpyHostToDevice, st));
    }
    ix->L = (int64_t)ix->leafOffH.size() - 1;
    const int64_t L = ix->L;
    // 6. permuted device copies
    PM_TRY(dalloc(&ix->perm, n));
    PM_CUDA(cudaMemcpyAsync(ix->perm, ix->permH.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PM_TRY(dalloc(&ix->leafOff, L + 1));
    PM_CUDA(cudaMemcpyAsync(ix->leafOff, ix->leafOffH.data(), (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_TRY(dalloc(&ix->X, (size_t)n * ld));
    PM_TRY(dalloc(&ix->O32, (size_t)n * PM_MP));
    PM_TRY(dalloc(&ix->O64, (size_t)n * PM_MP));
    PM_LAUNCH("k_gather_rows", st, k_gather_rows<float><<<2048, 256, 0, st>>>(Xo, ix->X, ix->perm, n, ld));
    PM_LAUNCH("k_gather_rows", st, k_gather_rows<float><<<2048, 256, 0, st>>>(O32o, ix->O32, ix->perm, n, PM_MP));
    PM_LAUNCH("k_gather_rows", st, k_gather_rows<double><<<2048, 256, 0, st>>>(O64o, ix->O64, ix->perm, n, PM_MP));
    PM_CUDA(cudaGetLastError());
    // 7. leaf balls, pivots (farthest-first over leaf centres), rings
    PM_TRY(dalloc(&ix->leafMeta, (size_t)L * PM_LEAF_STRIDE));
    PM_CUDA(cudaMemsetAsync(ix->leafMeta, 0, (size_t)L * PM_LEAF_STRIDE * sizeof(float), st));
    double *ro64 = nullptr;
    PM_TRY(dalloc(&ro64, (size_t)L * PM_MP));
    struct G4 { double *a; ~G4() { cudaFree(a); } } g4{ro64};
    PM_LAUNCH("k_leaf_ball", st, k_leaf_ball<<<(unsigned)L, 256, 0, st>>>(ix->O64, ix->leafOff, m, ix->maxNorm, ix->leafMeta, ro64));
    PM_CUDA(cudaGetLastError());
    std::vector<float> meta((size_t)L * PM_LEAF_STRIDE);
    PM_CUDA(cudaMemcpyAsync(meta.data(), ix->leafMeta, meta.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    std::vector<float> piv((size_t)PM_MAX_PIVOTS * PM_MP, 0.f);
    {
        std::vector<double> mind(L, INFINITY);
        int64_t cur = 0;
        for (int i = 0; i < ix->s; i++) {
            for (int j = 0; j < PM_MP; j++) piv[(size_t)i * PM_MP + j] = meta[(size_t)cur * PM_LEAF_STRIDE + j];
            int64_t nxt = 0;
            double best = -1.0;
            for (int64_t l = 0; l < L; l++) {
                double s2 = 0.0;
                for (int j = 0; j < PM_MP; j++) {
                    double t = (double)meta[(size_t)l * PM_LEAF_STRIDE + j] - piv[(size_t)i * PM_MP + j];
                    s2 += t * t;
                }
                mind[l] = std::min(mind[l], s2);
                if (mind[l] > best) { best = mind[l]; nxt = l; }
            }
            cur = nxt;
        }
    }
    PM_TRY(dalloc(&ix->piv32, piv.size()));
    PM_CUDA(cudaMemcpyAsync(ix->piv32, piv.data(), piv.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    if (ix->s > 0) {
        PM_LAUNCH("k_leaf_rings", st, k_leaf_rings<<<(unsigned)L, 256, 0, st>>>(ix->O32, ix->leafOff, ix->piv32, ix->s, ix->leafMeta));
        PM_CUDA(cudaGetLastError());
    }
    PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}
