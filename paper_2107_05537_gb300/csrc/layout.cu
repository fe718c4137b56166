// Original-space refinement of the leaf layout on the GPU (Sec. 4.1: the
// PM-tree's leaves are balls around routing objects; here a leaf that the
// projected-space bisection produced is split further where it straddles
// separate groups of points in the original space, so that the verification's
// original-space balls around leaves and chunks stay tight).
//
// One CTA per segment of the bisection (at most 1024 points).  The segment is
// refined depth first with an explicit stack:
//   1. outliers: the points farther from the mean than twice the median
//      distance are split off (each part refined again);
//   2. separate groups: a 2-means split (two starts: the mean and its
//      farthest point, and that point and its farthest point; at most six
//      Lloyd steps each; the lower sum of squared deviations wins) is kept if
//      it lowers the sum of squared deviations below 0.85 of the whole's
//      (each part refined again);
//   3. otherwise the segment is a leaf, cut into chunks of at most 32 points
//      by recursive 2-means (a degenerate split halves by position); the
//      points of a chunk are kept in id order.
// Every split is a stable partition of the segment's positions, so parts stay
// contiguous, and leaves and chunks come out in position order.  Sums run in
// a fixed order: the layout depends only on the data.
#include <algorithm>
#include <vector>

#include "pmlsh_impl.h"

namespace {

constexpr int LR_THREADS = 256;
constexpr int LR_MAXS = 1024;   // points per segment at most (the leaf capacity's range)

struct LrSeg {
    int64_t lo, hi;      // positions of the segment
    int64_t nodeBase;    // output slots: nodes [2 s], leaves [s], chunk ends [s]
    int64_t leafBase, chunkBase;
};

// Outputs, per segment: nodes {begin, end, left, right} (offsets from the
// segment's first position; local node ids, -1 for a leaf; node 0 is the
// segment), leaves {begin, end, node, first chunk}, chunk ends (offsets), and
// the three counts.
struct LrOut {
    int4 *node;
    int4 *leaf;
    int32_t *chunkEnd;
    int32_t *count;      // [segments][3]
    int *err;
};

__device__ __forceinline__ double lr_warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA-wide exclusive prefix sum of v (256 threads); *tot receives the sum.
__device__ __forceinline__ int lr_scan(int v, int *tmp, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) tmp[w] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int i = 0; i < LR_THREADS / 32; i++) {
        before += i < w ? tmp[i] : 0;
        all += tmp[i];
    }
    __syncthreads();
    *tot = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(LR_THREADS)
k_refine_leaves(const float *__restrict__ X, int ld, int d, int32_t *__restrict__ perm, int32_t *__restrict__ tmp,
                const LrSeg *__restrict__ segs, double *__restrict__ scratch, LrOut out)
{
    __shared__ float sDist[LR_MAXS];
    __shared__ unsigned char sSide[LR_MAXS], sSide2[LR_MAXS];
    __shared__ float sSort[LR_MAXS];
    __shared__ int sStackLo[LR_MAXS + 64], sStackHi[LR_MAXS + 64], sStackNode[LR_MAXS + 64];
    __shared__ int sScan[LR_THREADS / 32];
    __shared__ double sRed[LR_THREADS / 32];
    __shared__ int sInt[8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = LR_THREADS / 32;
    const LrSeg S = segs[blockIdx.x];
    const int s = (int)(S.hi - S.lo);
    int32_t *P = perm + S.lo;   // this segment's ids
    int32_t *T = tmp + S.lo;
    // centres: mu, a, b, a2, b2 (FP64 [ld] each, this CTA's scratch)
    double *mu = scratch + (size_t)blockIdx.x * 5 * ld;
    double *ca = mu + ld, *cb = ca + ld, *ca2 = cb + ld, *cb2 = ca2 + ld;
    int4 *onode = out.node + S.nodeBase;
    int4 *oleaf = out.leaf + S.leafBase;
    int32_t *ochunk = out.chunkEnd + S.chunkBase;
    if (s < 1 || s > LR_MAXS) {
        if (tid == 0) atomicOr(out.err, 1);
        return;
    }

    // ||x_P[i] - c||^2 for i in [a, b) into sDist (a warp per point, FP64 sums)
    auto dist_to = [&](const double *c, int a, int b) {
        for (int i = a + w; i < b; i += nw) {
            const float *x = X + (int64_t)P[i] * ld;
            double acc = 0.0;
            for (int j = lane; j < d; j += 32) {
                const double t = (double)x[j] - c[j];
                acc += t * t;
            }
            acc = lr_warp_sum(acc);
            if (lane == 0) sDist[i] = (float)acc;
        }
        __syncthreads();
    };
    // number of positions i in [a, b) with pred(i), by the whole CTA
    auto count_if = [&](int a, int b, auto pred) -> int {
        int cnt = 0;
        for (int i0 = a; i0 < b; i0 += LR_THREADS) {
            const int i = i0 + tid;
            cnt += __syncthreads_count(i < b && pred(i));
        }
        return cnt;
    };
    // FP64 mean of the points i in [a, b) with sSide[i] == side (side < 0: all)
    auto mean_of = [&](double *c, int a, int b, int side) {
        const int cnt = count_if(a, b, [&](int i) { return side < 0 || sSide[i] == side; });
        const double inv = cnt > 0 ? 1.0 / (double)cnt : 0.0;
        for (int j = tid; j < d; j += LR_THREADS) {
            double acc = 0.0;
            for (int i = a; i < b; i++)
                if (side < 0 || sSide[i] == side) acc += (double)X[(int64_t)P[i] * ld + j];
            c[j] = acc * inv;
        }
        __syncthreads();
        return cnt;
    };
    auto copy_point = [&](double *c, int i) {
        for (int j = tid; j < d; j += LR_THREADS) c[j] = (double)X[(int64_t)P[i] * ld + j];
        __syncthreads();
    };
    // index of the largest sDist[i] in [a, b) (first on ties)
    auto argmax = [&](int a, int b) -> int {
        float best = -1.f;
        int bi = a;
        for (int i = a + tid; i < b; i += LR_THREADS)
            if (sDist[i] > best) { best = sDist[i]; bi = i; }
        for (int o = 16; o; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
            sRed[w] = best;
            sScan[w] = bi;
        }
        __syncthreads();
        float bb = -1.f;
        int ri = a;
        for (int v = 0; v < nw; v++)
            if ((float)sRed[v] > bb || ((float)sRed[v] == bb && sScan[v] < ri)) { bb = (float)sRed[v]; ri = sScan[v]; }
        __syncthreads();
        return ri;
    };
    // FP64 sum over [a, b) of sDist where sSide == side (side < 0: all)
    auto sum_dist = [&](int a, int b, int side) -> double {
        double acc = 0.0;
        for (int i = a + tid; i < b; i += LR_THREADS)
            if (side < 0 || sSide[i] == side) acc += (double)sDist[i];
        acc = lr_warp_sum(acc);
        if (lane == 0) sRed[w] = acc;
        __syncthreads();
        double all = 0.0;
        for (int v = 0; v < nw; v++) all += sRed[v];
        __syncthreads();
        return all;
    };
    // Lloyd steps from centres (c0, c1) over [a, b): sides in sSide (1 =
    // nearer c1); returns the side-0 count, the two sums of squared
    // deviations in *s0, *s1
    auto lloyd = [&](double *c0, double *c1, int a, int b, double *s0, double *s1) -> int {
        const int size = b - a;
        int n0 = 0;
        for (int it = 0; it < 6; it++) {
            dist_to(c0, a, b);
            for (int i = a + tid; i < b; i += LR_THREADS) sSort[i] = sDist[i];
            __syncthreads();
            dist_to(c1, a, b);
            for (int i = a + tid; i < b; i += LR_THREADS) sSide[i] = sDist[i] < sSort[i] ? 1 : 0;
            __syncthreads();
            n0 = count_if(a, b, [&](int i) { return sSide[i] == 0; });
            if (n0 == 0 || n0 == size) break;
            // new centres (kept if they moved)
            if (tid == 0) sInt[1] = 0;
            __syncthreads();
            for (int j = tid; j < d; j += LR_THREADS) {
                double acc0 = 0.0, acc1 = 0.0;
                for (int i = a; i < b; i++) {
                    const double x = (double)X[(int64_t)P[i] * ld + j];
                    if (sSide[i]) acc1 += x; else acc0 += x;
                }
                const double v0 = acc0 / (double)n0, v1 = acc1 / (double)(size - n0);
                if (v0 != c0[j] || v1 != c1[j]) sInt[1] = 1;
                c0[j] = v0;
                c1[j] = v1;
            }
            __syncthreads();
            if (!sInt[1]) break;
        }
        // sums of squared deviations with the final centres
        dist_to(c0, a, b);
        for (int i = a + tid; i < b; i += LR_THREADS) sSort[i] = sDist[i];
        __syncthreads();
        dist_to(c1, a, b);
        for (int i = a + tid; i < b; i += LR_THREADS)
            if (!sSide[i]) sDist[i] = sSort[i];
        __syncthreads();
        *s0 = sum_dist(a, b, 0);
        *s1 = sum_dist(a, b, 1);
        return n0;
    };
    // the two-start 2-means of [a, b): sides in sSide, returns the side-0 count
    auto two_means = [&](int a, int b, double *s0, double *s1) -> int {
        const int size = b - a;
        mean_of(mu, a, b, -1);
        dist_to(mu, a, b);
        const int ib = argmax(a, b);
        for (int j = tid; j < d; j += LR_THREADS) ca[j] = mu[j];
        __syncthreads();
        copy_point(cb, ib);
        copy_point(ca2, ib);
        dist_to(ca2, a, b);
        const int ic = argmax(a, b);
        copy_point(cb2, ic);
        double t0, t1;
        int n0 = lloyd(ca, cb, a, b, s0, s1);
        for (int i = a + tid; i < b; i += LR_THREADS) sSide2[i] = sSide[i];
        __syncthreads();
        const int m0 = lloyd(ca2, cb2, a, b, &t0, &t1);
        if (m0 > 0 && m0 < size && (t0 + t1 < *s0 + *s1 || n0 == 0 || n0 == size)) {
            n0 = m0;
            *s0 = t0;
            *s1 = t1;
        } else {
            for (int i = a + tid; i < b; i += LR_THREADS) sSide[i] = sSide2[i];
            __syncthreads();
        }
        return n0;
    };
    // stable move of the side-0 positions of [a, b) to the front
    auto apply_sides = [&](int a, int b) {
        const int size = b - a;
        constexpr int PER = LR_MAXS / LR_THREADS;
        int z[PER], cz = 0;
        for (int u = 0; u < PER; u++) {
            const int i = tid * PER + u;
            z[u] = i < size && sSide[a + i] == 0;
            cz += z[u];
        }
        int totZ = 0;
        int pz = lr_scan(cz, sScan, &totZ);
        int po = tid * PER - pz;   // side-1 entries before this thread's
        for (int u = 0; u < PER; u++) {
            const int i = tid * PER + u;
            if (i < size) {
                if (z[u]) T[a + pz++] = P[a + i];
                else T[a + totZ + po++] = P[a + i];
            }
        }
        __syncthreads();
        for (int i = a + tid; i < b; i += LR_THREADS) P[i] = T[i];
        __syncthreads();
    };

    int nNode = 1, nLeaf = 0, nChunk = 0, sp = 0;
    if (tid == 0) onode[0] = make_int4(0, s, -1, -1);
    if (tid == 0) {
        sStackLo[0] = 0;
        sStackHi[0] = s;
        sStackNode[0] = 0;
    }
    sp = 1;
    __syncthreads();
    while (sp > 0) {
        sp--;
        const int a = sStackLo[sp], b = sStackHi[sp], nd = sStackNode[sp];
        __syncthreads();
        const int size = b - a;
        int left = -1;   // >= 0: split here
        if (size >= 2) {
            // 1. outliers beyond twice the median distance to the mean
            mean_of(mu, a, b, -1);
            dist_to(mu, a, b);
            for (int i = tid; i < LR_MAXS; i += LR_THREADS) sSort[i] = i < size ? sDist[a + i] : INFINITY;
            __syncthreads();
            for (int k2 = 2; k2 <= LR_MAXS; k2 <<= 1)
                for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                    for (int i = tid; i < LR_MAXS; i += LR_THREADS) {
                        const int l2 = i ^ j2;
                        if (l2 > i) {
                            const float x = sSort[i], y = sSort[l2];
                            if ((x > y) == ((i & k2) == 0)) { sSort[i] = y; sSort[l2] = x; }
                        }
                    }
                    __syncthreads();
                }
            // (squared distances: twice the median distance is four times
            // the median squared distance)
            const float cut = 4.f * sSort[size / 2];
            const int nout = count_if(a, b, [&](int i) { return sDist[i] > cut; });
            if (nout > 0 && nout < size) {
                for (int i = a + tid; i < b; i += LR_THREADS) sSide[i] = sDist[i] > cut;
                __syncthreads();
                apply_sides(a, b);
                left = size - nout;
            } else {
                // 2. separate groups
                double s0, s1;
                const int l2 = two_means(a, b, &s0, &s1);
                // the whole's sum of squared deviations
                mean_of(mu, a, b, -1);
                dist_to(mu, a, b);
                const double sse = sum_dist(a, b, -1);
                if (l2 >= 1 && l2 <= size - 1 && s0 + s1 < 0.85 * sse) {
                    // the sides of the chosen 2-means were overwritten by the
                    // distance pass above only in sDist, not sSide
                    apply_sides(a, b);
                    left = l2;
                }
            }
        }
        if (left >= 0) {
            // inner node with two children, each refined again
            if (nNode + 2 > 2 * s) {
                if (tid == 0) atomicOr(out.err, 2);
                break;
            }
            const int Lc = nNode, Rc = nNode + 1;
            nNode += 2;
            if (tid == 0) {
                onode[nd].z = Lc;
                onode[nd].w = Rc;
                onode[Lc] = make_int4(a, a + left, -1, -1);
                onode[Rc] = make_int4(a + left, b, -1, -1);
                sStackLo[sp] = a + left;
                sStackHi[sp] = b;
                sStackNode[sp] = Rc;
                sStackLo[sp + 1] = a;
                sStackHi[sp + 1] = a + left;
                sStackNode[sp + 1] = Lc;
            }
            sp += 2;
            __syncthreads();
            continue;
        }
        // 3. a leaf: chunks of <= 32 points, depth first
        if (tid == 0) oleaf[nLeaf] = make_int4(a, b, nd, nChunk);
        nLeaf++;
        // the chunk stack lives above the refinement stack
        int cs = sp;
        if (tid == 0) {
            sStackLo[cs] = a;
            sStackHi[cs] = b;
        }
        cs++;
        __syncthreads();
        while (cs > sp) {
            cs--;
            const int c0 = sStackLo[cs], c1 = sStackHi[cs];
            __syncthreads();
            const int cz = c1 - c0;
            if (cz <= 32) {
                // ids in ascending order inside the chunk
                if (tid < 32) {
                    const int32_t v = tid < cz ? P[c0 + tid] : 0x7fffffff;
                    int rank = 0;
                    for (int u = 0; u < cz; u++) {
                        const int32_t o = P[c0 + u];
                        rank += (o < v) ? 1 : 0;
                    }
                    __syncwarp();
                    if (tid < cz) T[c0 + rank] = v;
                    __syncwarp();
                    if (tid < cz) P[c0 + tid] = T[c0 + tid];
                }
                if (tid == 0) ochunk[nChunk] = c1;
                nChunk++;
                __syncthreads();
                continue;
            }
            double s0, s1;
            int l2 = two_means(c0, c1, &s0, &s1);
            const int minside = max(1, cz / 16);
            if (l2 < minside || l2 > cz - minside) l2 = cz / 2;   // degenerate: by position
            else apply_sides(c0, c1);
            if (tid == 0) {
                sStackLo[cs] = c0 + l2;
                sStackHi[cs] = c1;
                sStackLo[cs + 1] = c0;
                sStackHi[cs + 1] = c0 + l2;
            }
            cs += 2;
            __syncthreads();
        }
    }
    if (tid == 0) {
        out.count[blockIdx.x * 3 + 0] = nNode;
        out.count[blockIdx.x * 3 + 1] = nLeaf;
        out.count[blockIdx.x * 3 + 2] = nChunk;
    }
}

template <class T> pmlsh_status lr_alloc(T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        pm_set_error("cudaMalloc failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PMLSH_ENOMEM : PMLSH_ECUDA;
    }
    return PMLSH_OK;
}

}  // namespace

pmlsh_status pm_refine_leaves(const float *Xo, int ld, int d, int32_t *permD, const std::vector<int64_t> &segLo,
                              const std::vector<int64_t> &segHi, std::vector<LrResult> &res, cudaStream_t st)
{
    const int64_t ns = (int64_t)segLo.size();
    res.assign(ns, LrResult());
    if (ns == 0) return PMLSH_OK;
    std::vector<LrSeg> segs(ns);
    int64_t nb = 0, lb = 0, cb = 0;
    for (int64_t i = 0; i < ns; i++) {
        const int64_t sz = segHi[i] - segLo[i];
        if (sz < 1 || sz > LR_MAXS) {
            pm_set_error("leaf refinement: segment of %lld points (1..%d)", (long long)sz, LR_MAXS);
            return PMLSH_EINTERNAL;
        }
        segs[i] = LrSeg{segLo[i], segHi[i], nb, lb, cb};
        nb += 2 * sz;
        lb += sz;
        cb += sz;
    }
    const int64_t n = segHi[ns - 1];
    struct Mem {
        std::vector<void *> p;
        ~Mem() { for (void *q : p) cudaFree(q); }
    } mem;
    LrSeg *dSeg;
    int32_t *dTmp, *dChunk, *dCount;
    int4 *dNode, *dLeaf;
    double *dScratch;
    int *dErr;
    const int64_t grid = ns;
    PM_TRY(lr_alloc(&dSeg, ns)); mem.p.push_back(dSeg);
    PM_TRY(lr_alloc(&dTmp, n)); mem.p.push_back(dTmp);
    PM_TRY(lr_alloc(&dNode, nb)); mem.p.push_back(dNode);
    PM_TRY(lr_alloc(&dLeaf, lb)); mem.p.push_back(dLeaf);
    PM_TRY(lr_alloc(&dChunk, cb)); mem.p.push_back(dChunk);
    PM_TRY(lr_alloc(&dCount, ns * 3)); mem.p.push_back(dCount);
    PM_TRY(lr_alloc(&dScratch, (size_t)grid * 5 * ld)); mem.p.push_back(dScratch);
    PM_TRY(lr_alloc(&dErr, 1)); mem.p.push_back(dErr);
    PM_CUDA(cudaMemcpyAsync(dSeg, segs.data(), ns * sizeof(LrSeg), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
    LrOut o{dNode, dLeaf, dChunk, dCount, dErr};
    PM_LAUNCH("k_refine_leaves", st, k_refine_leaves<<<(unsigned)grid, LR_THREADS, 0, st>>>(Xo, ld, d, permD, dTmp, dSeg,
                                                                                          dScratch, o));
    PM_CUDA(cudaGetLastError());
    std::vector<int4> hNode(nb), hLeaf(lb);
    std::vector<int32_t> hChunk(cb), hCount(ns * 3);
    int hErr = 0;
    PM_CUDA(cudaMemcpyAsync(hNode.data(), dNode, nb * sizeof(int4), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaMemcpyAsync(hLeaf.data(), dLeaf, lb * sizeof(int4), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaMemcpyAsync(hChunk.data(), dChunk, cb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaMemcpyAsync(hCount.data(), dCount, ns * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaMemcpyAsync(&hErr, dErr, sizeof(int), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    if (hErr) {
        pm_set_error("leaf refinement: internal capacity exceeded (flags %d)", hErr);
        return PMLSH_EINTERNAL;
    }
    for (int64_t i = 0; i < ns; i++) {
        LrResult &r = res[i];
        const int nn = hCount[i * 3], nl = hCount[i * 3 + 1], nc = hCount[i * 3 + 2];
        r.node.assign(hNode.begin() + segs[i].nodeBase, hNode.begin() + segs[i].nodeBase + nn);
        r.leaf.assign(hLeaf.begin() + segs[i].leafBase, hLeaf.begin() + segs[i].leafBase + nl);
        r.chunkEnd.assign(hChunk.begin() + segs[i].chunkBase, hChunk.begin() + segs[i].chunkBase + nc);
    }
    return PMLSH_OK;
}
