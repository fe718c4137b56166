// Index build: projection (Eq. 3), leaf layout (the flattened stand-in for
// the PM-tree of Sec. 4.1), leaf balls and pivot rings, distance sample for
// the r_min rule of Sec. 5.2.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>

#include <cuda_bf16.h>

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
// Radial profile of a leaf (meta [17, 24)): for g = 2 .. 8, an upper bound of
// the ceil(g s / 8)-th largest distance of the leaf's s members from its FP32
// centre, with the centre's rounding covered as in the leaf radius.  The
// range count's bounds use it: a member whose radius is below d(q, centre) -
// R lies outside the ball, one whose radius is below R - d(q, centre) inside.
// Leaves above LR_MAXS members take the leaf radius for every rank.
constexpr int LR_MAXS = 2048;
__global__ void k_leaf_radii(const double *__restrict__ O64, const int64_t *__restrict__ off, int m,
                             double maxNorm, const double *__restrict__ ro64, float *__restrict__ meta)
{
    __shared__ float rad[LR_MAXS];
    const int64_t l = blockIdx.x;
    const int64_t a = off[l];
    const int sz = (int)(off[l + 1] - a);
    float *M = meta + l * PM_LEAF_STRIDE;
    if (sz > LR_MAXS) {
        for (int g = 2 + (int)threadIdx.x; g <= 8; g += blockDim.x) M[15 + g] = M[16];
        return;
    }
    const double *c = ro64 + l * PM_MP;
    double cn = 0.0;
    for (int j = 0; j < PM_MP; j++) cn = fma(c[j], c[j], cn);
    const double slack = 0x1.0p-23 * (sqrt(cn) + maxNorm);
    for (int e = threadIdx.x; e < sz; e += blockDim.x)
        rad[e] = __double2float_ru((pm_pdist64(O64 + (a + e) * PM_MP, c, m) + slack) * (1.0 + 1e-6));
    __syncthreads();
    // rank of each member in descending order (ties by position); the
    // members at ranks ceil(g s / 8) give the profile
    for (int e = threadIdx.x; e < sz; e += blockDim.x) {
        const float v = rad[e];
        int rank = 0;
        for (int f = 0; f < sz; f++) {
            const float w = rad[f];
            rank += (w > v || (w == v && f < e)) ? 1 : 0;
        }
        for (int g = 2; g <= 8; g++)
            if (rank + 1 == (g * sz + 7) / 8) M[15 + g] = v;
    }
}

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

// Original-space leaf centre mu (FP32 rounding of the FP64 mean) and a radius
// Rx >= the exact distance of every member to mu (FP64, inflated, rounded up):
// ||x - q|| >= ||q - mu|| - Rx bounds the distance of any member from below.
// One block (256 threads) per leaf.
__global__ void k_leaf_orig(const float *__restrict__ X, const int64_t *__restrict__ off, int ld,
                            float *__restrict__ mu, float *__restrict__ rx)  // also used for chunks
{
    __shared__ double sred[8];
    const int64_t l = blockIdx.x;
    const int64_t a = off[l], b = off[l + 1];
    const double inv = 1.0 / (double)(b - a);
    float *M = mu + l * ld;
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        double s = 0.0;
        for (int64_t p = a; p < b; p++) s += (double)X[p * ld + j];
        M[j] = (float)(s * inv);
    }
    __syncthreads();
    double r = 0.0;
    for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < ld; j++) {
            double t = (double)X[p * ld + j] - (double)M[j];
            s = fma(t, t, s);
        }
        r = fmax(r, sqrt(s));
    }
    r = warp_max(r);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = fmax(r, sred[w]);
        r = fmax(r, sred[0]);
        rx[l] = __double2float_ru(r * (1.0 + 1e-6) + 1e-30);
    }
}

// BF16 residuals of the rows from their leaf's original-space centre, for
// the verification's first pass: r~ = BF16(fl32(x - mu_l)) per coordinate,
// and per row e >= ||x - mu_l - r~|| (FP64 of the FP32 and BF16 values,
// inflated, rounded up), so that x = mu_l + r~ + delta with ||delta|| <= e.
// One block per leaf, one warp per row.
__global__ void k_build_resid(const float *__restrict__ X, const int64_t *__restrict__ off, int ld,
                              const float *__restrict__ mu, uint16_t *__restrict__ Xr, float *__restrict__ rowErr)
{
    const int64_t l = blockIdx.x;
    const int64_t a = off[l], b = off[l + 1];
    const float *M = mu + l * ld;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t p = a + w; p < b; p += nw) {
        double e2 = 0.0;
        for (int j = lane; j < ld; j += 32) {
            const float x = X[p * ld + j], m = M[j];
            const __nv_bfloat16 r = __float2bfloat16_rn(__fsub_rn(x, m));
            Xr[p * ld + j] = __bfloat16_as_ushort(r);
            const double dl = ((double)x - (double)m) - (double)__bfloat162float(r);
            e2 += dl * dl;
        }
        for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        if (lane == 0) rowErr[p] = __double2float_ru(sqrt(e2) * (1.0 + 1e-6) + 1e-30);
    }
}

// Tensor-core operand of the projected points: per point the 48 BF16 values
// [hi(o') | hi(o') | lo(o')] (hi = o' rounded to BF16, lo = the rest rounded),
// stored leaf by leaf (each leaf starts at a row that is a multiple of 16,
// padding rows are zero) in the no-swizzle K-major canonical layout of the
// tcgen05 matrix descriptor: 8-row x 8-element core matrices of 128 bytes,
// row group g, K group kg at byte ((g * 6 + kg) * 8 + row % 8) * 16.  Also
// the FP32 squared norms ||o'||^2 of the FP32 coordinates, same rows (NaN
// on padding rows).
__global__ void k_build_bsplit(const float *__restrict__ O32, const int64_t *__restrict__ off,
                               const int64_t *__restrict__ bOff, int64_t L, uint16_t *__restrict__ B,
                               float *__restrict__ norms)
{
    const int64_t l = blockIdx.x;
    const int64_t p0 = off[l], s = off[l + 1] - p0, r0 = bOff[l];
    for (int64_t r = threadIdx.x; r < s; r += blockDim.x) {
        const float *o = O32 + (p0 + r) * PM_MP;
        const int64_t R = r0 + r, g = R >> 3, i = R & 7;
        double nn = 0.0;
        for (int j = 0; j < PM_MP; j++) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(o[j]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(o[j] - __bfloat162float(hi));
            const uint16_t hb = __bfloat16_as_ushort(hi), lb = __bfloat16_as_ushort(lo);
            const int k0 = j, k1 = 16 + j, k2 = 32 + j;
            B[((g * 6 + (k0 >> 3)) * 8 + i) * 8 + (k0 & 7)] = hb;
            B[((g * 6 + (k1 >> 3)) * 8 + i) * 8 + (k1 & 7)] = hb;
            B[((g * 6 + (k2 >> 3)) * 8 + i) * 8 + (k2 & 7)] = lb;
            nn += (double)o[j] * (double)o[j];
        }
        norms[R] = (float)nn;
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

// Query batches: one thread per (row, direction), the same sequential fma
// over the columns as k_project64, so the coordinates are bit-identical;
// a batch of 10^4 rows then fills the GPU instead of 79 blocks.
__global__ void k_project64_rows(const float *__restrict__ X, int64_t n, int ld, int d, int m,
                                 const float *__restrict__ A, double *__restrict__ O64, float *__restrict__ O32,
                                 int ostride)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * ostride) return;
    const int64_t p = e / ostride;
    const int j = (int)(e % ostride);
    double acc = 0.0;
    if (j < m) {
        // the same sequence of fmas over c = 0 .. d - 1; 16-byte loads, eight
        // columns per step (rows are 16-byte aligned), then the tail
        const float *x = X + p * ld, *a = A + (int64_t)j * ld;
        int c = 0;
        for (; c + 8 <= d; c += 8) {
            const float4 a0 = *(const float4 *)(a + c), a1 = *(const float4 *)(a + c + 4);
            const float4 x0 = *(const float4 *)(x + c), x1 = *(const float4 *)(x + c + 4);
            acc = __fma_rn(pm_f2d_exact(a0.x), pm_f2d_exact(x0.x), acc);
            acc = __fma_rn(pm_f2d_exact(a0.y), pm_f2d_exact(x0.y), acc);
            acc = __fma_rn(pm_f2d_exact(a0.z), pm_f2d_exact(x0.z), acc);
            acc = __fma_rn(pm_f2d_exact(a0.w), pm_f2d_exact(x0.w), acc);
            acc = __fma_rn(pm_f2d_exact(a1.x), pm_f2d_exact(x1.x), acc);
            acc = __fma_rn(pm_f2d_exact(a1.y), pm_f2d_exact(x1.y), acc);
            acc = __fma_rn(pm_f2d_exact(a1.z), pm_f2d_exact(x1.z), acc);
            acc = __fma_rn(pm_f2d_exact(a1.w), pm_f2d_exact(x1.w), acc);
        }
        for (; c < d; c++) acc = __fma_rn(pm_f2d_exact(a[c]), pm_f2d_exact(x[c]), acc);
    }
    if (O64) O64[p * ostride + j] = acc;
    if (O32) O32[p * ostride + j] = __double2float_rn(acc);
}

void pm_launch_project64(const float *X, int64_t n, int ld, int d, int m, const float *A,
                         double *O64, float *O32, unsigned long long *maxNormBits,
                         cudaStream_t st, int ostride)
{
    if (n <= 0) return;
    if (!maxNormBits && n * ostride <= ((int64_t)1 << 22)) {
        const int64_t tot = n * ostride;
        PM_LAUNCH("k_project64_rows", st, k_project64_rows<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, n, ld, d, m, A,
                                                                                                    O64, O32, ostride));
        return;
    }
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
    // projected-space nodes: position range, children, routing hyperplane
    std::vector<int64_t> plo, phi;
    std::vector<int32_t> nl, nr;
    std::vector<float> nw;   // [N][16] split hyperplane normal
    std::vector<float> nt;   // [N] split threshold: right iff w . o' >= t
    std::vector<int32_t> pre;   // [N] index of the node's segment for the refinement, -1 if inner
    std::vector<int64_t> preLo, preHi;
    std::vector<double> key;
    // the final layout (assemble): leaf-index ranges of the nodes, leaves, chunks
    std::vector<int64_t> nlo, nhi;
    std::vector<int64_t> leafOff{0};
    std::vector<int64_t> chunkOff{0};   // chunk c holds positions [chunkOff[c], chunkOff[c+1])
    std::vector<int32_t> leafChunk{0};  // leaf l holds chunks [leafChunk[l], leafChunk[l+1])

    const float *pt(int32_t id) const { return O + (int64_t)id * PM_MP; }

    static double d2(const double *a, const float *b)
    {
        double s = 0.0;
        for (int j = 0; j < PM_MP; j++) {
            double t = a[j] - (double)b[j];
            s += t * t;
        }
        return s;
    }

    // Radius of the bounding-box-centred ball of perm[lo, hi).
    double radius(int64_t lo, int64_t hi) const
    {
        double mn[PM_MP], mx[PM_MP], c[PM_MP];
        for (int j = 0; j < PM_MP; j++) { mn[j] = INFINITY; mx[j] = -INFINITY; }
        for (int64_t e = lo; e < hi; e++)
            for (int j = 0; j < PM_MP; j++) {
                double v = pt(perm[e])[j];
                mn[j] = std::min(mn[j], v);
                mx[j] = std::max(mx[j], v);
            }
        for (int j = 0; j < PM_MP; j++) c[j] = 0.5 * (mn[j] + mx[j]);
        double r = 0.0;
        for (int64_t e = lo; e < hi; e++) r = std::max(r, d2(c, pt(perm[e])));
        return std::sqrt(r);
    }

    // 2-means of perm[lo, hi) started from a farthest pair; returns the
    // hyperplane (w, t) separating the two means.
    void two_means(int64_t lo, int64_t hi, double *w, double &t)
    {
        double c0[PM_MP], a[PM_MP], b[PM_MP];
        for (int j = 0; j < PM_MP; j++) c0[j] = pt(perm[lo])[j];
        int64_t ia = lo;
        double best = -1.0;
        for (int64_t e = lo; e < hi; e++) {
            double v = d2(c0, pt(perm[e]));
            if (v > best) { best = v; ia = e; }
        }
        for (int j = 0; j < PM_MP; j++) a[j] = pt(perm[ia])[j];
        int64_t ib = lo;
        best = -1.0;
        for (int64_t e = lo; e < hi; e++) {
            double v = d2(a, pt(perm[e]));
            if (v > best) { best = v; ib = e; }
        }
        for (int j = 0; j < PM_MP; j++) b[j] = pt(perm[ib])[j];
        for (int it = 0; it < 6; it++) {
            double sa[PM_MP] = {0}, sb[PM_MP] = {0};
            int64_t na = 0, nb = 0;
            for (int64_t e = lo; e < hi; e++) {
                const float *p = pt(perm[e]);
                if (d2(b, p) < d2(a, p)) { nb++; for (int j = 0; j < PM_MP; j++) sb[j] += p[j]; }
                else { na++; for (int j = 0; j < PM_MP; j++) sa[j] += p[j]; }
            }
            if (na == 0 || nb == 0) break;
            bool moved = false;
            for (int j = 0; j < PM_MP; j++) {
                double na_ = sa[j] / na, nb_ = sb[j] / nb;
                moved |= na_ != a[j] || nb_ != b[j];
                a[j] = na_;
                b[j] = nb_;
            }
            if (!moved) break;
        }
        // right side: closer to b  <=>  (b - a) . p >= (|b|^2 - |a|^2) / 2
        double aa = 0.0, bb = 0.0;
        for (int j = 0; j < PM_MP; j++) {
            w[j] = b[j] - a[j];
            aa += a[j] * a[j];
            bb += b[j] * b[j];
        }
        t = 0.5 * (bb - aa);
    }

    int32_t new_node(int64_t lo, int64_t hi)
    {
        int32_t id = (int32_t)plo.size();
        plo.push_back(lo);
        phi.push_back(hi);
        nl.push_back(-1);
        nr.push_back(-1);
        for (int j = 0; j < PM_MP; j++) nw.push_back(0.f);
        nt.push_back(0.f);
        pre.push_back(-1);
        return id;
    }

    // A segment the projected bisection does not split further: refined in
    // the original space afterwards (pm_refine_leaves).
    int32_t pre_leaf(int32_t id, int64_t lo, int64_t hi)
    {
        pre[id] = (int32_t)preLo.size();
        preLo.push_back(lo);
        preHi.push_back(hi);
        return id;
    }

    // Splits perm[lo, hi) by 2-means in the projected space (Sec. 4.1 builds
    // the PM-tree so that node balls are tight; the m_RAD promotion of
    // Sec. 6.3 minimises covering radii).  Segments above M points are always
    // split; smaller ones only when both halves' balls shrink below 0.85 of
    // the parent's (a segment holding separate groups of points), so that a
    // leaf does not straddle groups.  A degenerate 2-means split of a large
    // segment falls back to the median along the same direction.
    int32_t split(int64_t lo, int64_t hi)
    {
        const int32_t id = new_node(lo, hi);
        const int64_t size = hi - lo;
        if (size <= 8) return pre_leaf(id, lo, hi);
        double w[PM_MP], t;
        two_means(lo, hi, w, t);
        for (int64_t e = lo; e < hi; e++) {
            const float *p = pt(perm[e]);
            double s = 0.0;
            for (int j = 0; j < PM_MP; j++) s += w[j] * (double)p[j];
            key[perm[e]] = s;
        }
        const double *K = key.data();
        auto less = [K](int32_t a, int32_t b) { return K[a] < K[b] || (K[a] == K[b] && a < b); };
        int64_t nright = 0;
        for (int64_t e = lo; e < hi; e++) nright += K[perm[e]] >= t;
        int64_t left = size - nright;
        if (size > M) {
            if (left < size / 16 || left > size - size / 16) {
                left = size / 2;
                std::nth_element(perm.begin() + lo, perm.begin() + lo + left, perm.begin() + hi, less);
                t = K[perm[lo + left]];
            } else {
                std::partition(perm.begin() + lo, perm.begin() + hi, [K, t](int32_t a) { return K[a] < t; });
            }
        } else {
            if (left == 0 || left == size) return pre_leaf(id, lo, hi);
            std::vector<int32_t> saved(perm.begin() + lo, perm.begin() + hi);
            std::partition(perm.begin() + lo, perm.begin() + hi, [K, t](int32_t a) { return K[a] < t; });
            double rp = radius(lo, hi), rl = radius(lo, lo + left), rr = radius(lo + left, hi);
            if (!(std::max(rl, rr) < 0.85 * rp)) {
                std::copy(saved.begin(), saved.end(), perm.begin() + lo);
                return pre_leaf(id, lo, hi);
            }
        }
        for (int j = 0; j < PM_MP; j++) nw[(size_t)id * PM_MP + j] = (float)w[j];
        nt[id] = (float)t;
        int32_t L = split(lo, lo + left);
        int32_t R = split(lo + left, hi);
        nl[id] = L;
        nr[id] = R;
        return id;
    }

    // The hierarchy after the original-space refinement: the refined
    // segments' sub-trees replace their nodes (refinement splits route
    // queries right: w = 0, t = 0), leaves and chunks in position order, and
    // every node's leaf-index range.
    void assemble(const std::vector<LrResult> &res)
    {
        const size_t P = plo.size();
        nlo.assign(P, 0);
        nhi.assign(P, 0);
        std::vector<int64_t> stack{0};
        std::vector<char> seen(P, 0);
        // iterative DFS: a node's leaf range opens on entry, closes on exit
        while (!stack.empty()) {
            const int64_t e = stack.back();
            if (!seen[e]) {
                seen[e] = 1;
                nlo[e] = (int64_t)leafOff.size() - 1;
                if (pre[e] >= 0) {
                    expand((int32_t)e, res[pre[e]], plo[e]);
                    nhi[e] = (int64_t)leafOff.size() - 1;
                    stack.pop_back();
                } else {
                    stack.push_back(nr[e]);
                    stack.push_back(nl[e]);
                }
            } else {
                nhi[e] = (int64_t)leafOff.size() - 1;
                stack.pop_back();
            }
        }
    }

    // Appends the refined segment's sub-tree below node e (local node 0).
    void expand(int32_t e, const LrResult &r, int64_t base)
    {
        const int nn = (int)r.node.size();
        std::vector<int32_t> gid(nn, -1);
        gid[0] = e;
        for (int i = 1; i < nn; i++) {
            gid[i] = (int32_t)plo.size();
            plo.push_back(base + r.node[i].x);
            phi.push_back(base + r.node[i].y);
            nl.push_back(-1);
            nr.push_back(-1);
            for (int j = 0; j < PM_MP; j++) nw.push_back(0.f);
            nt.push_back(0.f);
            pre.push_back(-1);
            nlo.push_back(0);
            nhi.push_back(0);
        }
        for (int i = 0; i < nn; i++)
            if (r.node[i].z >= 0) {
                nl[gid[i]] = gid[r.node[i].z];
                nr[gid[i]] = gid[r.node[i].w];
            }
        // leaves in position order; a local node's leaves are those inside
        // its position range
        const int64_t firstLeaf = (int64_t)leafOff.size() - 1;
        for (size_t li = 0; li < r.leaf.size(); li++) {
            const int4 lf = r.leaf[li];
            const int cEnd = li + 1 < r.leaf.size() ? r.leaf[li + 1].w : (int)r.chunkEnd.size();
            for (int c = lf.w; c < cEnd; c++) chunkOff.push_back(base + r.chunkEnd[c]);
            leafChunk.push_back((int32_t)chunkOff.size() - 1);
            leafOff.push_back(base + lf.y);
        }
        for (int i = 1; i < nn; i++) {
            int64_t a = -1, b = -1;
            for (size_t li = 0; li < r.leaf.size(); li++)
                if (r.leaf[li].x >= r.node[i].x && r.leaf[li].y <= r.node[i].y) {
                    if (a < 0) a = firstLeaf + (int64_t)li;
                    b = firstLeaf + (int64_t)li + 1;
                }
            nlo[gid[i]] = a;
            nhi[gid[i]] = b;
        }
    }
};

// Orthonormalises the columns of V [d][K] (FP64, column c at V[j * K + c])
// by modified Gram-Schmidt, twice; a column that vanishes becomes zero.
void orthonormalize(std::vector<double> &V, int d, int K)
{
    for (int pass = 0; pass < 2; pass++)
        for (int c = 0; c < K; c++) {
            for (int b = 0; b < c; b++) {
                double dot = 0.0;
                for (int j = 0; j < d; j++) dot += V[(size_t)j * K + b] * V[(size_t)j * K + c];
                for (int j = 0; j < d; j++) V[(size_t)j * K + c] -= dot * V[(size_t)j * K + b];
            }
            double nn = 0.0;
            for (int j = 0; j < d; j++) nn += V[(size_t)j * K + c] * V[(size_t)j * K + c];
            const double inv = nn > 1e-24 ? 1.0 / std::sqrt(nn) : 0.0;
            for (int j = 0; j < d; j++) V[(size_t)j * K + c] *= inv;
        }
}

// PM_PCA leading principal directions of the leaf centres (rows of P,
// [PM_PCA][ld], zero padding columns), by subspace iteration from a seeded
// start.  Any rows that are orthonormal make ||P v|| <= ||v||, so the
// iteration count affects only how tight that bound is; rows beyond the
// rank of the centres (or beyond d) are zero.
void leaf_pca(const std::vector<float> &mu, int64_t L, int ld, int d, uint64_t seed, std::vector<double> &P)
{
    const int K = PM_PCA;
    std::vector<double> mean(d, 0.0);
    for (int64_t l = 0; l < L; l++)
        for (int j = 0; j < d; j++) mean[j] += mu[(size_t)l * ld + j];
    for (int j = 0; j < d; j++) mean[j] /= (double)L;
    std::vector<double> V((size_t)d * K), W((size_t)d * K), T((size_t)K);
    for (size_t i = 0; i < V.size(); i++)
        V[i] = (double)(pm_splitmix64(seed, i) >> 11) * 0x1.0p-52 - 1.0;
    orthonormalize(V, d, K);
    for (int it = 0; it < 5; it++) {
        std::fill(W.begin(), W.end(), 0.0);
        for (int64_t l = 0; l < L; l++) {
            const float *m = mu.data() + (size_t)l * ld;
            // T = (mu_l - mean) . V, then W += (mu_l - mean) T
            std::fill(T.begin(), T.end(), 0.0);
            for (int j = 0; j < d; j++) {
                const double x = m[j] - mean[j];
                const double *v = V.data() + (size_t)j * K;
                for (int c = 0; c < K; c++) T[c] += x * v[c];
            }
            for (int j = 0; j < d; j++) {
                const double x = m[j] - mean[j];
                double *w = W.data() + (size_t)j * K;
                for (int c = 0; c < K; c++) w[c] += x * T[c];
            }
        }
        V.swap(W);
        orthonormalize(V, d, K);
    }
    P.assign((size_t)K * ld, 0.0);
    for (int c = 0; c < K && c < d; c++)
        for (int j = 0; j < d; j++) P[(size_t)c * ld + j] = V[(size_t)j * K + c];
}

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
    cudaFree(ix->leafMu);
    cudaFree(ix->leafRx);
    cudaFree(ix->pcaP);
    cudaFree(ix->pcaP32);
    cudaFree(ix->leafPmu);
    cudaFree(ix->chunkOff);
    cudaFree(ix->leafChunk);
    cudaFree(ix->chunkMu);
    cudaFree(ix->chunkRx);
    cudaFree(ix->bOff);
    cudaFree(ix->Bsplit);
    cudaFree(ix->bNorm);
    cudaFree(ix->Xr);
    cudaFree(ix->rowErr);
    pm_release_work(ix->work);
}

void pm_release_work(KnnWork &w)
{
    DevBuf *bufs[] = {&w.Qd, &w.qp32, &w.qp64, &w.qnorm, &w.qpiv, &w.order, &w.keys,
                      &w.keys2, &w.vals2, &w.sortTmp, &w.qstate, &w.thr, &w.blkCnt,
                      &w.blkLeaves, &w.cntSure, &w.cntBand, &w.bandQ, &w.bandPos,
                      &w.bandIn, &w.bandCnt, &w.partD, &w.partI, &w.partSeen, &w.bandInQ,
                      &w.outD64, &w.outIds, &w.outErr, &w.dk, &w.flags, &w.selBuf,
                      &w.selOff, &w.selCnt, &w.selTau, &w.active, &w.misc, &w.blkMask,
                      &w.recheck, &w.leafBits, &w.fullBits, &w.cntPart, &w.cntTight, &w.subIdx, &w.subThr, &w.subBits, &w.qpca};
    for (DevBuf *b : bufs) b->release();
    w.stage.release();
}

pmlsh_status HostBuf::reserve(size_t b)
{
    if (b <= bytes) return PMLSH_OK;
    release();
    const size_t nb = std::max<size_t>(b, 4096);
    if (cudaMallocHost(&p, nb) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        pm_set_error("pinned host allocation of %zu bytes failed", nb);
        return PMLSH_ENOMEM;
    }
    bytes = nb;
    return PMLSH_OK;
}

void HostBuf::release()
{
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
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
    bs.key.resize(n);
    std::iota(bs.perm.begin(), bs.perm.end(), 0);
    bs.split(0, n);
    // original-space refinement of the segments on the device, over the
    // device copy of X (original order)
    {
        int32_t *permD = nullptr;
        PM_TRY(dalloc(&permD, n));
        struct G4 { int32_t *p; ~G4() { cudaFree(p); } } g4{permD};
        PM_CUDA(cudaMemcpyAsync(permD, bs.perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        std::vector<LrResult> res;
        PM_TRY(pm_refine_leaves(Xo, ld, d, permD, bs.preLo, bs.preHi, res, st));
        PM_CUDA(cudaMemcpyAsync(bs.perm.data(), permD, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        bs.assemble(res);
    }
    ix->permH = std::move(bs.perm);
    ix->chunkOffH = std::move(bs.chunkOff);
    ix->leafChunkH = std::move(bs.leafChunk);
    ix->leafOffH = std::move(bs.leafOff);
    ix->nodeLo = std::move(bs.nlo);
    ix->nodeHi = std::move(bs.nhi);
    ix->nodeLeft = std::move(bs.nl);
    ix->nodeRight = std::move(bs.nr);
    {
        size_t N = ix->nodeLo.size();
        std::vector<int32_t> ti(N * 4);
        std::vector<float> tv(N * (PM_MP + 1));
        for (size_t e = 0; e < N; e++) {
            ti[e * 4 + 0] = ix->nodeLeft[e];
            ti[e * 4 + 1] = ix->nodeRight[e];
            ti[e * 4 + 2] = 0;
            ti[e * 4 + 3] = (int32_t)ix->nodeLo[e];
            for (int j = 0; j < PM_MP; j++) tv[e * (PM_MP + 1) + j] = bs.nw[e * PM_MP + j];
            tv[e * (PM_MP + 1) + PM_MP] = bs.nt[e];
        }
        PM_TRY(dalloc(&ix->treeI, ti.size()));
        PM_TRY(dalloc(&ix->treeV, tv.size()));
        PM_CUDA(cudaMemcpyAsync(ix->treeI, ti.data(), ti.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaMemcpyAsync(ix->treeV, tv.data(), tv.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaStreamSynchronize(st));
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
    PM_LAUNCH("k_leaf_radii", st, k_leaf_radii<<<(unsigned)L, 256, 0, st>>>(ix->O64, ix->leafOff, m, ix->maxNorm, ro64,
                                                                          ix->leafMeta));
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
    // 8. original-space leaf centres and radii (lower bounds for verification)
    PM_TRY(dalloc(&ix->leafMu, (size_t)L * ld));
    PM_TRY(dalloc(&ix->leafRx, (size_t)L));
    PM_LAUNCH("k_leaf_orig", st, k_leaf_orig<<<(unsigned)L, 256, 0, st>>>(ix->X, ix->leafOff, ld, ix->leafMu, ix->leafRx));
    PM_CUDA(cudaGetLastError());
    // principal directions of the leaf centres: a cheap exact lower bound
    // ||P (q - mu)|| <= ||q - mu|| for the verification's leaf order
    {
        std::vector<float> muH((size_t)L * ld);
        PM_CUDA(cudaMemcpyAsync(muH.data(), ix->leafMu, muH.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        std::vector<double> P;
        leaf_pca(muH, L, ld, d, ix->seed + 5, P);
        std::vector<float> pmu((size_t)L * PM_PCA);
        double muMax = 0.0;
        for (int64_t l = 0; l < L; l++) {
            const float *m = muH.data() + (size_t)l * ld;
            double nn = 0.0;
            for (int j = 0; j < d; j++) nn += (double)m[j] * m[j];
            muMax = std::max(muMax, std::sqrt(nn));
            for (int r = 0; r < PM_PCA; r++) {
                double s = 0.0;
                for (int j = 0; j < d; j++) s += P[(size_t)r * ld + j] * (double)m[j];
                pmu[(size_t)l * PM_PCA + r] = (float)s;
            }
        }
        ix->muMax = muMax;
        std::vector<float> P32(P.begin(), P.end());
        PM_TRY(dalloc(&ix->pcaP32, P32.size()));
        PM_CUDA(cudaMemcpyAsync(ix->pcaP32, P32.data(), P32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        PM_TRY(dalloc(&ix->pcaP, P.size()));
        PM_TRY(dalloc(&ix->leafPmu, pmu.size()));
        PM_CUDA(cudaMemcpyAsync(ix->pcaP, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaMemcpyAsync(ix->leafPmu, pmu.data(), pmu.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaStreamSynchronize(st));
    }
    // tensor-core operand of the projected points (leaf-padded rows)
    if (o->bf16_shadow) {
        std::vector<int64_t> bo(L + 1, 0);
        for (int64_t l = 0; l < L; l++) {
            int64_t s = ix->leafOffH[l + 1] - ix->leafOffH[l];
            bo[l + 1] = bo[l] + (s + 15) / 16 * 16;
        }
        ix->bOffH = bo;
        const int64_t rows = bo[L];
        PM_TRY(dalloc(&ix->bOff, L + 1));
        PM_TRY(dalloc(&ix->Bsplit, (size_t)rows * 48));
        PM_TRY(dalloc(&ix->bNorm, (size_t)rows));
        PM_CUDA(cudaMemcpyAsync(ix->bOff, bo.data(), (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        PM_CUDA(cudaMemsetAsync(ix->Bsplit, 0, (size_t)rows * 48 * sizeof(uint16_t), st));
        // padding rows: NaN norms, so that every comparison on them is false
        PM_CUDA(cudaMemsetAsync(ix->bNorm, 0xFF, (size_t)rows * sizeof(float), st));
        PM_LAUNCH("k_build_bsplit", st, k_build_bsplit<<<(unsigned)L, 128, 0, st>>>(ix->O32, ix->leafOff, ix->bOff, L, ix->Bsplit, ix->bNorm));
        PM_CUDA(cudaGetLastError());
        // BF16 residual rows for the verification's first pass
        PM_TRY(dalloc(&ix->Xr, (size_t)n * ld));
        PM_TRY(dalloc(&ix->rowErr, (size_t)n));
        PM_LAUNCH("k_build_resid", st, k_build_resid<<<(unsigned)L, 256, 0, st>>>(ix->X, ix->leafOff, ld, ix->leafMu,
                                                                                  ix->Xr, ix->rowErr));
        PM_CUDA(cudaGetLastError());
    }
    // chunks of <= 32 points inside the leaves, with their own balls
    const int64_t C = (int64_t)ix->chunkOffH.size() - 1;
    ix->nChunks = C;
    PM_TRY(dalloc(&ix->chunkOff, C + 1));
    PM_TRY(dalloc(&ix->leafChunk, L + 1));
    PM_CUDA(cudaMemcpyAsync(ix->chunkOff, ix->chunkOffH.data(), (C + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(ix->leafChunk, ix->leafChunkH.data(), (L + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PM_TRY(dalloc(&ix->chunkMu, (size_t)C * ld));
    PM_TRY(dalloc(&ix->chunkRx, (size_t)C));
    PM_LAUNCH("k_leaf_orig", st, k_leaf_orig<<<(unsigned)C, 128, 0, st>>>(ix->X, ix->chunkOff, ld, ix->chunkMu, ix->chunkRx));
    PM_CUDA(cudaGetLastError());
    PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}
