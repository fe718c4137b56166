// (c,k)-ACP query path: Algorithm 4 (radius filtering) with FindLCA
// (Algorithm 5) over the index's leaf hierarchy.
//
//   k_cp_selfjoin   every pair inside each leaf: FP32 squared distance
//   k_node_ball     node balls (Sec. 4.1) in FP64, bounding-box midpoint and
//                   largest distance, the same arithmetic as the oracle
//   [host]          FindLCA: maximal inner nodes with radius < R = gamma t ub,
//                   sorted by (radius, node id)
//   k_cp_node_pairs cross-leaf pairs of a node's subtree with projected
//                   distance < t ub (FP32 with a proven band, FP64 inside it)
//   k_pair_*        exact top-k merges: radix select of an FP32 threshold,
//                   guard set, FP64 distances, sort by (dist, i, j)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pmlsh_impl.h"

namespace {

constexpr int PAIR_SORT_CAP = 4096;   // guard entries merged in one block

struct PairCand {
    float key;      // FP32 squared distance (original or projected space)
    int32_t a, b;   // leaf-order positions, a < b in position order
};

// All pairs inside leaf l, FP32 squared distance by direct difference
// (sequential over the row).  One block per leaf.
__global__ void k_cp_selfjoin(const float *__restrict__ X, int ld, const int64_t *__restrict__ off,
                              const int64_t *__restrict__ pairOff, PairCand *__restrict__ out)
{
    const int64_t l = blockIdx.x;
    const int64_t p0 = off[l], s = off[l + 1] - p0;
    const int64_t np = s * (s - 1) / 2;
    for (int64_t e = threadIdx.x; e < np; e += blockDim.x) {
        // e -> (i, j), i < j, row-major over the upper triangle: row i starts
        // at C(i) = i (2 s - i - 1) / 2; i from the root of C(i) = e in FP64,
        // then integer corrections (at most a step or two)
        const double b2 = 2.0 * (double)s - 1.0;
        int64_t i = (int64_t)((b2 - sqrt(fmax(0.0, b2 * b2 - 8.0 * (double)e))) * 0.5);
        i = i < 0 ? 0 : (i > s - 2 ? s - 2 : i);
        while (i > 0 && i * (2 * s - i - 1) / 2 > e) i--;
        while (i < s - 2 && (i + 1) * (2 * s - i - 2) / 2 <= e) i++;
        const int64_t j = i + 1 + (e - i * (2 * s - i - 1) / 2);
        const float *x = X + (p0 + i) * ld, *y = X + (p0 + j) * ld;
        float acc = 0.f;
        for (int c = 0; c < ld; c++) {
            float t = __fsub_rn(x[c], y[c]);
            acc = __fmaf_rn(t, t, acc);
        }
        PairCand pc;
        pc.key = acc;
        pc.a = (int32_t)(p0 + i);
        pc.b = (int32_t)(p0 + j);
        out[pairOff[l] + e] = pc;
    }
}

__device__ __forceinline__ double dmin_warp(double v)
{
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double dmax_warp(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Node ball in FP64: centre = midpoint of the bounding box of the node's
// projected points, radius = largest FP64 distance to it.  One block (256
// threads) per node.
__global__ void k_node_ball(const double *__restrict__ O64, const int64_t *__restrict__ posLo,
                            const int64_t *__restrict__ posHi, int m, double *__restrict__ rad)
{
    __shared__ double smn[8][PM_MP], smx[8][PM_MP], sro[PM_MP], srad[8];
    const int e = blockIdx.x;
    const int64_t a = posLo[e], b = posHi[e];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < PM_MP; j++) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) {
            double v = O64[p * PM_MP + j];
            mn = fmin(mn, v);
            mx = fmax(mx, v);
        }
        mn = dmin_warp(mn);
        mx = dmax_warp(mx);
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
    double r = 0.0;
    for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) r = fmax(r, pm_pdist64(O64 + p * PM_MP, sro, m));
    r = dmax_warp(r);
    if (lane == 0) srad[warp] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rr = srad[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) rr = fmax(rr, srad[w]);
        rad[e] = rr;
    }
}

// Cross-leaf pairs of positions [lo, hi) whose FP64 projected distance is
// < Rt (strict, Algorithm 4).  FP32: |sqrt(d'^2_32) - d'_64| <= eps, so
// d'^2_32 < loT is surely in, > hiT surely out, and the rest is decided in
// FP64.  Thread per first position a; loops over b > a.
// Sec. 6.3, setting of gamma: for every pair (a, b), a < b, of the n
// positions of a layout, R / ||o_a', o_b'|| with R the radius of their lowest
// common node (descending from the root while both leaves lie in one child;
// the leaf itself for two points of one leaf), FP64 projected distance with
// the oracle's arithmetic and a correctly rounded quotient; 0 / 0 -> 0,
// R / 0 -> +inf.  Block a writes pairs (a, b) at a n - a (a + 1) / 2 + b - a - 1.
__global__ void k_gamma_ratio(const double *__restrict__ O64, int64_t n, int m, const int32_t *__restrict__ leafOf,
                              const int64_t *__restrict__ node /*[N][4]: left, right, leaf lo, leaf hi*/,
                              const double *__restrict__ rad, double *__restrict__ out, int *__restrict__ err)
{
    const int64_t a = blockIdx.x;
    const int64_t base = a * n - a * (a + 1) / 2 - a - 1;
    const int64_t la = leafOf[a];
    for (int64_t b = a + 1 + threadIdx.x; b < n; b += blockDim.x) {
        const int64_t lb = leafOf[b];
        int64_t e = 0;
        int depth = 0;
        for (; depth < 4096; depth++) {
            const int64_t x = node[e * 4], y = node[e * 4 + 1];
            if (x < 0) break;
            if (la >= node[x * 4 + 2] && la < node[x * 4 + 3] && lb >= node[x * 4 + 2] && lb < node[x * 4 + 3])
                e = x;
            else if (la >= node[y * 4 + 2] && la < node[y * 4 + 3] && lb >= node[y * 4 + 2] && lb < node[y * 4 + 3])
                e = y;
            else
                break;
        }
        if (depth == 4096) atomicOr(err, 1);
        const double R = rad[e];
        const double dv = pm_pdist64(O64 + a * PM_MP, O64 + b * PM_MP, m);
        out[base + b] = dv > 0.0 ? __ddiv_rn(R, dv) : (R > 0.0 ? (double)INFINITY : 0.0);
    }
}

// 256-bin histogram of 8 bits at `shift` of the keys whose bits above them
// equal `prefix` (non-negative doubles and +inf order like their bits).
__global__ void k_gamma_hist(const unsigned long long *__restrict__ v, int64_t N, int shift,
                             unsigned long long hiMask, unsigned long long prefix, unsigned int *__restrict__ hist)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = v[e];
        if ((k & hiMask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Rows X[pos[i]] (leaf-order copy, row length ld) -> S[i] (row length d).
__global__ void k_gather_rows(const float *__restrict__ X, int ld, int d, const int64_t *__restrict__ pos,
                              int64_t ns, float *__restrict__ S)
{
    const int64_t i = blockIdx.x;
    if (i >= ns) return;
    const float *x = X + pos[i] * ld;
    for (int j = threadIdx.x; j < d; j += blockDim.x) S[i * d + j] = x[j];
}

__global__ void k_cp_node_pairs(const float *__restrict__ O32, const double *__restrict__ O64, int m,
                                const int32_t *__restrict__ leafOfPos, int64_t lo, int64_t hi, float loT,
                                float hiT, double Rt, PairCand *__restrict__ out, unsigned long long *cnt,
                                unsigned long long cap, unsigned long long *fp64n)
{
    const int64_t a = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= hi) return;
    float oa[PM_MP];
#pragma unroll
    for (int j = 0; j < PM_MP; j++) oa[j] = O32[a * PM_MP + j];
    const int la = leafOfPos[a];
    for (int64_t b = a + 1; b < hi; b++) {
        if (leafOfPos[b] == la) continue;
        const float v = pm_pd2_32(oa, O32 + b * PM_MP);
        bool in = v < loT;
        if (!in && v <= hiT) {
            atomicAdd(fp64n, 1ull);
            in = pm_pdist64(O64 + a * PM_MP, O64 + b * PM_MP, m) < Rt;
        }
        if (in) {
            unsigned long long slot = atomicAdd(cnt, 1ull);
            if (slot < cap) {
                PairCand pc;
                pc.key = v;
                pc.a = (int32_t)a;
                pc.b = (int32_t)b;
                out[slot] = pc;
            }
        }
    }
}

// Original-space FP32 squared distances of candidate pairs (overwrites key).
__global__ void k_pair_dist32(const float *__restrict__ X, int ld, PairCand *__restrict__ p, int64_t n)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float *x = X + (int64_t)p[e].a * ld, *y = X + (int64_t)p[e].b * ld;
    float acc = 0.f;
    for (int c = 0; c < ld; c++) {
        float t = __fsub_rn(x[c], y[c]);
        acc = __fmaf_rn(t, t, acc);
    }
    p[e].key = acc;
}

// Histogram of key bits [sh, sh+w) among keys whose bits above sh+w equal
// `prefix` (radix select pass over a global buffer).
__global__ void k_pair_hist(const PairCand *__restrict__ p, int64_t n, int sh, int w, unsigned int hiMask,
                            unsigned int prefix, unsigned int *__restrict__ hist)
{
    __shared__ unsigned int h[2048];
    for (int i = threadIdx.x; i < (1 << w); i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        unsigned int k = __float_as_uint(p[e].key);
        if ((k & hiMask) == (prefix & hiMask)) atomicAdd(&h[(k >> sh) & ((1u << w) - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << w); i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Entries with key <= thr, appended to `out` with FP64 distance (original or
// projected space) and original ids (i < j).
struct PairExact {
    double dist;
    int64_t i, j;
    int32_t a, b;   // positions
};

__global__ void k_pair_collect(const PairCand *__restrict__ p, int64_t n, float thr, const float *__restrict__ X,
                               int ld, int d, const double *__restrict__ O64, int m, int useProj,
                               const int32_t *__restrict__ perm, PairExact *__restrict__ out,
                               unsigned long long *cnt, unsigned long long cap)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const PairCand c = p[e];
    if (!(c.key <= thr)) return;
    unsigned long long slot = atomicAdd(cnt, 1ull);
    if (slot >= cap) return;
    PairExact x;
    x.dist = useProj ? pm_pdist64(O64 + (int64_t)c.a * PM_MP, O64 + (int64_t)c.b * PM_MP, m)
                     : pm_dist64(X + (int64_t)c.a * ld, X + (int64_t)c.b * ld, d);
    int64_t ia = perm[c.a], ib = perm[c.b];
    x.i = ia < ib ? ia : ib;
    x.j = ia < ib ? ib : ia;
    x.a = c.a;
    x.b = c.b;
    out[slot] = x;
}

__device__ __forceinline__ bool pe_less(const PairExact &x, const PairExact &y)
{
    if (x.dist != y.dist) return x.dist < y.dist;
    if (x.i != y.i) return x.i < y.i;
    return x.j < y.j;
}

// One block: sorts n (<= PAIR_SORT_CAP) entries by (dist, i, j) in place.
__global__ void k_pair_sort(PairExact *__restrict__ v, int n)
{
    extern __shared__ __align__(16) unsigned char psm[];
    PairExact *s = (PairExact *)psm;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < n) s[i] = v[i];
        else { s[i].dist = INFINITY; s[i].i = 0x7fffffffffffffffLL; s[i].j = 0x7fffffffffffffffLL; s[i].a = s[i].b = -1; }
    }
    __syncthreads();
    for (int k2 = 2; k2 <= P; k2 <<= 1)
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = (i & k2) == 0;
                    if (pe_less(s[ixj], s[i]) == up) {
                        PairExact t = s[i]; s[i] = s[ixj]; s[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = s[i];
}


// ------------------------------------------- Algorithm 3 (branch and bound)

// All pairs inside leaf l keyed by their FP32 projected squared distance.
// One block per leaf.
__global__ void k_bnb_selfjoin(const float *__restrict__ O32, const int64_t *__restrict__ off,
                               const int64_t *__restrict__ pairOff, PairCand *__restrict__ out)
{
    const int64_t l = blockIdx.x;
    const int64_t p0 = off[l], s = off[l + 1] - p0;
    const int64_t np = s * (s - 1) / 2;
    for (int64_t e = threadIdx.x; e < np; e += blockDim.x) {
        int64_t i = 0, rem = e;
        while (rem >= s - 1 - i) { rem -= s - 1 - i; i++; }
        const int64_t j = i + 1 + rem;
        PairCand pc;
        pc.key = pm_pd2_32(O32 + (p0 + i) * PM_MP, O32 + (p0 + j) * PM_MP);
        pc.a = (int32_t)(p0 + i);
        pc.b = (int32_t)(p0 + j);
        out[pairOff[l] + e] = pc;
    }
}

struct LeafPair {
    float md;      // lower bound of the projected distance of any pair in l1 x l2
    int32_t l1, l2;
};

// Mindist of Sec. 6.1 for leaf pairs (l1, l2), l1 < l2: the larger of
// ||RO1, RO2|| - r1 - r2 and the gaps between the pivot rings, from the leaf
// entries (FP32, rounded so that it stays a lower bound).  Pairs with
// Mindist <= dT are listed.  Block per l1, threads over l2.
__global__ void k_bnb_mindist(const float *__restrict__ meta, int s, int64_t L, float dLo, float dT,
                              LeafPair *__restrict__ out, unsigned long long *cnt, unsigned long long cap)
{
    const int64_t l1 = blockIdx.x;
    const float *M1 = meta + l1 * PM_LEAF_STRIDE;
    for (int64_t l2 = l1 + 1 + threadIdx.x; l2 < L; l2 += blockDim.x) {
        const float *M2 = meta + l2 * PM_LEAF_STRIDE;
        const float dc = __fsqrt_rn(pm_pd2_32(M1, M2));
        float md = __fsub_rn(__fsub_rn(__fmul_rn(dc, 1.f - 1e-5f), M1[16]), M2[16]);
        for (int i = 0; i < PM_MAX_PIVOTS; i++) {
            if (i < s) {
                // rings [min, max] of the two leaves (already widened outwards)
                md = fmaxf(md, __fsub_rn(M2[24 + i], M1[32 + i]));
                md = fmaxf(md, __fsub_rn(M1[24 + i], M2[32 + i]));
            }
        }
        if (md > dLo && md <= dT) {
            const unsigned long long slot = atomicAdd(cnt, 1ull);
            if (slot < cap) {
                LeafPair lp;
                lp.md = md;
                lp.l1 = (int32_t)l1;
                lp.l2 = (int32_t)l2;
                out[slot] = lp;
            }
        }
    }
}

// Listed leaf pairs in ascending (Mindist, l1, l2) on the device: a 64-bit
// key per pair, the order-preserving bits of Mindist (+0 and -0 taken as
// one) above the pair's rank in (l1, l2) order, l1 (2L - l1 - 1) / 2 +
// l2 - l1 - 1 (below 2^32 when L(L - 1)/2 is), sorted by a stable LSD radix
// sort of 8-bit digits and decoded back.
constexpr int RS_THREADS = 256, RS_ITEMS = 32;   // keys per block and pass: 8,192
constexpr int64_t LP_GPU_MAX_L = 92682;         // L (L - 1) / 2 < 2^32

__device__ __forceinline__ int64_t lp_rank_base(int64_t l1, int64_t L) { return l1 * (2 * L - l1 - 1) / 2; }

__global__ void k_lp_key(const LeafPair *__restrict__ lp, int64_t n, int64_t L, unsigned long long *__restrict__ key)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const LeafPair x = lp[e];
    const unsigned int u = __float_as_uint(__fadd_rn(x.md, 0.f));
    const unsigned int ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    const int64_t rk = lp_rank_base(x.l1, L) + (x.l2 - x.l1 - 1);
    key[e] = ((unsigned long long)ord << 32) | (unsigned long long)(uint32_t)rk;
}

// digit counts of each block's keys, digit-major: hist[d * nb + block]
__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const unsigned long long *__restrict__ key, int64_t n, int shift, unsigned int *__restrict__ hist, int nb)
{
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * RS_THREADS * RS_ITEMS;
    const int64_t b1 = b0 + (int64_t)RS_THREADS * RS_ITEMS < n ? b0 + (int64_t)RS_THREADS * RS_ITEMS : n;
    for (int64_t e = b0 + threadIdx.x; e < b1; e += RS_THREADS) atomicAdd(&h[(unsigned)(key[e] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// exclusive prefix sum of h[0, N) in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned int *__restrict__ h, int64_t N)
{
    __shared__ unsigned int ws[32];
    const int64_t seg = (N + 1023) / 1024;
    const int64_t t0 = threadIdx.x * seg, t1 = t0 + seg < N ? t0 + seg : N;
    unsigned int sum = 0u;
    for (int64_t i = t0; i < t1; i++) sum += h[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned int x = ws[lane], xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += v;
        }
        ws[lane] = xi - x;
    }
    __syncthreads();
    unsigned int run = ws[w] + incl - sum;
    for (int64_t i = t0; i < t1; i++) {
        const unsigned int v = h[i];
        h[i] = run;
        run += v;
    }
}

// stable scatter by one digit: each block walks its keys in order, 256 per
// round; a key's place is its digit's running base plus the keys of that
// digit before it in the round (earlier warps, then earlier lanes)
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const unsigned long long *__restrict__ in, unsigned long long *__restrict__ out, int64_t n, int shift,
             const unsigned int *__restrict__ off, int nb)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ unsigned int base[256];
    __shared__ unsigned int wc[NW][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    base[t] = off[(int64_t)t * nb + blockIdx.x];
    const int64_t b0 = (int64_t)blockIdx.x * RS_THREADS * RS_ITEMS;
    for (int r = 0; r < RS_ITEMS; r++) {
        for (int j = 0; j < NW; j++) wc[j][t] = 0u;
        __syncthreads();
        const int64_t e = b0 + (int64_t)r * RS_THREADS + t;
        const bool valid = e < n;
        const unsigned long long k = valid ? in[e] : 0ull;
        const unsigned int d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;
        const unsigned int peers = __match_any_sync(0xffffffffu, d);
        const int rankW = __popc(peers & ((1u << lane) - 1u));
        if (valid && rankW == 0) wc[w][d] = (unsigned)__popc(peers);
        __syncthreads();
        if (valid) {
            unsigned int pos = base[d] + (unsigned)rankW;
            for (int j = 0; j < w; j++) pos += wc[j][d];
            out[pos] = k;
        }
        __syncthreads();
        unsigned int add = 0u;
        for (int j = 0; j < NW; j++) add += wc[j][t];
        base[t] += add;
        __syncthreads();
    }
}

// keys back to leaf pairs; flags a key out of order (bit 1) or a rank that
// does not decode to l1 < l2 < L (bit 2)
__global__ void k_lp_decode(const unsigned long long *__restrict__ key, int64_t n, int64_t L,
                            LeafPair *__restrict__ out, int *__restrict__ bad)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const unsigned long long k = key[e];
    if (e > 0 && key[e - 1] > k) atomicOr(bad, 1);
    const unsigned int ord = (unsigned int)(k >> 32);
    const unsigned int u = (ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord;
    const int64_t rk = (int64_t)(k & 0xffffffffull);
    // l1: the largest l with lp_rank_base(l) <= rk (root of the quadratic,
    // then at most a few steps of correction)
    const double A = 2.0 * (double)L - 1.0;
    const double disc = A * A - 8.0 * (double)rk;
    int64_t l1 = (int64_t)floor((A - sqrt(disc > 0.0 ? disc : 0.0)) * 0.5);
    l1 = l1 < 0 ? 0 : (l1 > L - 2 ? L - 2 : l1);
    for (int it = 0; it < 4 && l1 + 1 <= L - 2 && lp_rank_base(l1 + 1, L) <= rk; it++) l1++;
    for (int it = 0; it < 4 && l1 > 0 && lp_rank_base(l1, L) > rk; it++) l1--;
    const int64_t l2 = rk - lp_rank_base(l1, L) + l1 + 1;
    LeafPair x;
    x.md = __uint_as_float(u);
    x.l1 = (int32_t)l1;
    x.l2 = (int32_t)l2;
    if (!(l1 >= 0 && l1 < l2 && l2 < L)) {
        atomicOr(bad, 2);
        x.l1 = 0;
        x.l2 = 1;
    }
    out[e] = x;
}

// Every cross pair of the listed leaf pairs, keyed by the FP32 projected
// squared distance, at the listed offsets.  Block per leaf pair.
__global__ void k_bnb_cross(const float *__restrict__ O32, const int64_t *__restrict__ off,
                            const int2 *__restrict__ lp, const int64_t *__restrict__ lpOff,
                            PairCand *__restrict__ out)
{
    const int2 pr = lp[blockIdx.x];
    const int64_t a0 = off[pr.x], na = off[pr.x + 1] - a0;
    const int64_t b0 = off[pr.y], nb = off[pr.y + 1] - b0;
    const int64_t base = lpOff[blockIdx.x];
    for (int64_t e = threadIdx.x; e < na * nb; e += blockDim.x) {
        const int64_t ia = e / nb, ib = e % nb;
        PairCand pc;
        pc.key = pm_pd2_32(O32 + (a0 + ia) * PM_MP, O32 + (b0 + ib) * PM_MP);
        pc.a = (int32_t)(a0 + ia);
        pc.b = (int32_t)(b0 + ib);
        out[base + e] = pc;
    }
}

// Entries with key < lo moved to out (order kept only per block).
__global__ void k_pair_below(const PairCand *__restrict__ p, int64_t n, float lo, PairCand *__restrict__ out,
                             unsigned long long *cnt)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const PairCand c = p[e];
    if (c.key < lo) out[atomicAdd(cnt, 1ull)] = c;
}


// Entries with lo <= key <= hi, appended with their FP64 projected distance.
__global__ void k_pair_band(const PairCand *__restrict__ p, int64_t n, float lo, float hi,
                            const double *__restrict__ O64, int m, const int32_t *__restrict__ perm,
                            PairExact *__restrict__ out, unsigned long long *cnt, unsigned long long cap)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const PairCand c = p[e];
    if (!(c.key >= lo && c.key <= hi)) return;
    const unsigned long long slot = atomicAdd(cnt, 1ull);
    if (slot >= cap) return;
    PairExact x;
    x.dist = pm_pdist64(O64 + (int64_t)c.a * PM_MP, O64 + (int64_t)c.b * PM_MP, m);
    const int64_t ia = perm[c.a], ib = perm[c.b];
    x.i = ia < ib ? ia : ib;
    x.j = ia < ib ? ib : ia;
    x.a = c.a;
    x.b = c.b;
    out[slot] = x;
}

template <class T> pmlsh_status dalloc(T **p, size_t count)
{
    PM_CUDA(cudaMalloc((void **)p, std::max<size_t>(1, count) * sizeof(T)));
    return PMLSH_OK;
}

struct DevPtrs {
    std::vector<void *> ps;
    ~DevPtrs() { for (void *p : ps) cudaFree(p); }
    template <class T> pmlsh_status get(T **p, size_t n)
    {
        PM_TRY(dalloc(p, n));
        ps.push_back(*p);
        return PMLSH_OK;
    }
};

// Radix select over a device pair buffer: the rank-th smallest FP32 key
// (1-based).  Three passes of 11/11/10 bits.
pmlsh_status pair_kth(const PairCand *p, int64_t n, int64_t rank, unsigned int *hist, float *out, cudaStream_t st)
{
    unsigned int prefix = 0;
    int64_t need = rank;
    const int shifts[3] = {21, 10, 0}, widths[3] = {11, 11, 10};
    std::vector<unsigned int> hh(2048);
    for (int pass = 0; pass < 3; pass++) {
        const int sh = shifts[pass], w = widths[pass];
        const unsigned int hiMask = pass == 0 ? 0u : (0xffffffffu << (sh + w));
        PM_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 2048, st));
        int grid = (int)std::min<int64_t>(1024, (n + 255) / 256);
        PM_LAUNCH("k_pair_hist", st, k_pair_hist<<<std::max(1, grid), 256, 0, st>>>(p, n, sh, w, hiMask, prefix, hist));
        PM_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned int) * (1u << w), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        int64_t acc = 0;
        int bin = 0;
        for (; bin < (1 << w); bin++) {
            if (acc + (int64_t)hh[bin] >= need) break;
            acc += hh[bin];
        }
        need -= acc;
        prefix |= (unsigned int)bin << sh;
    }
    float f;
    std::memcpy(&f, &prefix, sizeof(f));
    *out = f;
    return PMLSH_OK;
}

// Exact top-k merge: the current list `top` (sorted by (dist, i, j), FP64
// distances, size kc <= k) and the candidate buffer p[0, n) with FP32
// original-space squared distances.  A candidate can enter only if its FP32
// value is <= min(K32 (1 + 3 eps_v), D_k^2 (1 + 3 eps_v)) (K32: k-th smallest
// FP32 candidate value, D_k: current k-th distance); those are recomputed in
// FP64 and sorted with the current list.
struct TopK {
    std::vector<PairExact> v;   // host copy, sorted
};

pmlsh_status pair_merge(TopK &top, int k, const PairCand *p, int64_t n, const pmlsh_index *ix, unsigned int *hist,
                        PairExact *scratch, unsigned long long *cnt, cudaStream_t st)
{
    if (n <= 0) return PMLSH_OK;
    const double epsv = (double)(ix->ld + 8) * 0x1.0p-24;
    double thr = INFINITY;
    if (n >= k) {
        float K32;
        PM_TRY(pair_kth(p, n, k, hist, &K32, st));
        thr = (double)K32 * (1.0 + 3.0 * epsv) + 1e-36;
    }
    if ((int)top.v.size() >= k) {
        double Dk = top.v[k - 1].dist;
        thr = std::min(thr, Dk * Dk * (1.0 + 3.0 * epsv) + 1e-36);
    }
    float thr32 = std::isinf(thr) ? INFINITY : (float)thr;
    if (!std::isinf(thr) && (double)thr32 < thr) thr32 = nextafterf(thr32, INFINITY);
    PM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    const unsigned long long cap = PAIR_SORT_CAP - (unsigned long long)top.v.size();
    PM_LAUNCH("k_pair_collect", st, k_pair_collect<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        p, n, thr32, ix->X, ix->ld, ix->d, ix->O64, ix->m, 0, ix->perm, scratch + top.v.size(), cnt, cap));
    PM_CUDA(cudaGetLastError());
    unsigned long long got = 0;
    PM_CUDA(cudaMemcpyAsync(&got, cnt, sizeof(got), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    if (got > cap) {
        pm_set_error("closest pairs: %llu candidates tied inside the FP32 guard band (capacity %llu)", got, cap);
        return PMLSH_EINTERNAL;
    }
    const int tot = (int)(top.v.size() + got);
    if (!top.v.empty())
        PM_CUDA(cudaMemcpyAsync(scratch, top.v.data(), top.v.size() * sizeof(PairExact), cudaMemcpyHostToDevice, st));
    int P = 1;
    while (P < tot) P <<= 1;
    PM_LAUNCH("k_pair_sort", st, k_pair_sort<<<1, 1024, (size_t)P * sizeof(PairExact), st>>>(scratch, tot));
    PM_CUDA(cudaGetLastError());
    const int keep = std::min(tot, k);
    top.v.resize(keep);
    PM_CUDA(cudaMemcpyAsync(top.v.data(), scratch, keep * sizeof(PairExact), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}

// Keeps the `need` candidates with the smallest (FP64 projected distance,
// i, j) of p[0, n) (the count > T cut of Algorithm 4).
pmlsh_status pair_truncate(PairCand *p, int64_t n, int64_t need, const pmlsh_index *ix, unsigned int *hist,
                           PairExact *scratch, unsigned long long *cnt, int64_t *nOut, cudaStream_t st)
{
    if (need >= n) { *nOut = n; return PMLSH_OK; }
    if (need <= 0) { *nOut = 0; return PMLSH_OK; }
    // FP32 projected keys: |sqrt(key) - d'_64| <= eps(d'); select the need-th
    // and resolve the band around it in FP64
    float K;
    PM_TRY(pair_kth(p, n, need, hist, &K, st));
    const double tau = std::sqrt((double)K);
    const double eps = 0x1.0p-22 * ix->maxNorm + 0x1.0p-19 * tau + 1e-300;
    const float hiK = (float)((tau + 2 * eps) * (tau + 2 * eps));
    PM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    PM_LAUNCH("k_pair_collect", st, k_pair_collect<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        p, n, nextafterf(hiK, INFINITY), ix->X, ix->ld, ix->d, ix->O64, ix->m, 1, ix->perm, scratch, cnt,
        PAIR_SORT_CAP));
    unsigned long long got = 0;
    PM_CUDA(cudaMemcpyAsync(&got, cnt, sizeof(got), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    if (got > PAIR_SORT_CAP) {
        pm_set_error("closest pairs: %llu candidates tied at the count > T cut (capacity %d)", got, PAIR_SORT_CAP);
        return PMLSH_EINTERNAL;
    }
    int P = 1;
    while (P < (int)got) P <<= 1;
    PM_LAUNCH("k_pair_sort", st, k_pair_sort<<<1, 1024, (size_t)P * sizeof(PairExact), st>>>(scratch, (int)got));
    std::vector<PairExact> v(got);
    PM_CUDA(cudaMemcpyAsync(v.data(), scratch, got * sizeof(PairExact), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    const int64_t keep = std::min<int64_t>(need, (int64_t)got);
    std::vector<PairCand> kept(keep);
    for (int64_t e = 0; e < keep; e++) {
        kept[e].key = 0.f;
        kept[e].a = v[e].a;
        kept[e].b = v[e].b;
    }
    PM_CUDA(cudaMemcpyAsync(p, kept.data(), keep * sizeof(PairCand), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaStreamSynchronize(st));
    *nOut = keep;
    return PMLSH_OK;
}


// The T candidates of p[0, n) with the smallest (FP64 projected distance,
// i, j) go to out[0, T) (any order): the T-th FP32 key by radix select;
// keys below its FP32 band are in, keys inside the band are ordered by
// (FP64 projected distance, i, j) and the first ones fill up to T.  tauHi:
// an upper bound of the T-th FP64 projected distance.
pmlsh_status pair_select(const PairCand *p, int64_t n, int64_t T, PairCand *out, const pmlsh_index *ix,
                         unsigned int *hist, PairExact *scratch, unsigned long long *cnt, int64_t *fp64,
                         double *tauHi, cudaStream_t st)
{
    float K;
    PM_TRY(pair_kth(p, n, T, hist, &K, st));
    const double tau = std::sqrt((double)K);
    const double eps = 0x1.0p-22 * ix->maxNorm + 0x1.0p-19 * tau + 1e-300;
    const double loD = tau - 2 * eps;
    float lo = loD > 0 ? (float)(loD * loD) : 0.f;
    if (loD > 0 && (double)lo > loD * loD) lo = nextafterf(lo, -INFINITY);
    if (!(loD > 0)) lo = 0.f;
    float hi = (float)((tau + 2 * eps) * (tau + 2 * eps));
    if ((double)hi < (tau + 2 * eps) * (tau + 2 * eps)) hi = nextafterf(hi, INFINITY);
    PM_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    if (loD > 0)
        PM_LAUNCH("k_pair_below", st, k_pair_below<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, lo, out, cnt));
    PM_LAUNCH("k_pair_band", st, k_pair_band<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        p, n, loD > 0 ? lo : -INFINITY, hi, ix->O64, ix->m, ix->perm, scratch, cnt + 1, PAIR_SORT_CAP));
    PM_CUDA(cudaGetLastError());
    unsigned long long hc[2];
    PM_CUDA(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    const int64_t nBelow = (int64_t)hc[0], nBand = (int64_t)hc[1];
    if (nBand > PAIR_SORT_CAP || nBelow > T || nBelow + nBand < T) {
        pm_set_error("closest pairs: %lld candidates inside the FP32 band at the T-th projected distance "
                     "(capacity %d)", (long long)nBand, PAIR_SORT_CAP);
        return PMLSH_EINTERNAL;
    }
    *fp64 += nBand;
    int P = 1;
    while (P < (int)nBand) P <<= 1;
    if (nBand > 0)
        PM_LAUNCH("k_pair_sort", st, k_pair_sort<<<1, 1024, (size_t)P * sizeof(PairExact), st>>>(scratch, (int)nBand));
    std::vector<PairExact> v(nBand);
    PM_CUDA(cudaMemcpyAsync(v.data(), scratch, nBand * sizeof(PairExact), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    const int64_t need = T - nBelow;
    std::vector<PairCand> kept(need);
    for (int64_t e = 0; e < need; e++) {
        kept[e].key = 0.f;
        kept[e].a = v[e].a;
        kept[e].b = v[e].b;
    }
    if (need > 0)
        PM_CUDA(cudaMemcpyAsync(out + nBelow, kept.data(), need * sizeof(PairCand), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaStreamSynchronize(st));
    *tauHi = tau + eps;
    return PMLSH_OK;
}

}  // namespace

// gamma of Sec. 6.3 over all pairs of the index `lx` (its own layout).
static pmlsh_status gamma_of_layout(const pmlsh_index *lx, double pr, double *gamma, cudaStream_t st)
{
    const int64_t n = lx->n, L = lx->L, N = (int64_t)lx->nodeLo.size();
    const int64_t npairs = n * (n - 1) / 2;
    DevPtrs mem;
    // node balls (FP64, the oracle's arithmetic)
    std::vector<int64_t> pLo(N), pHi(N), nodeH((size_t)N * 4);
    for (int64_t e = 0; e < N; e++) {
        pLo[e] = lx->leafOffH[lx->nodeLo[e]];
        pHi[e] = lx->leafOffH[lx->nodeHi[e]];
        nodeH[e * 4] = lx->nodeLeft[e];
        nodeH[e * 4 + 1] = lx->nodeRight[e];
        nodeH[e * 4 + 2] = lx->nodeLo[e];
        nodeH[e * 4 + 3] = lx->nodeHi[e];
    }
    std::vector<int32_t> lof(n);
    for (int64_t l = 0; l < L; l++)
        for (int64_t p = lx->leafOffH[l]; p < lx->leafOffH[l + 1]; p++) lof[p] = (int32_t)l;
    int64_t *dLo, *dHi, *dNode;
    double *dRad, *ratio;
    int32_t *dLeafOf;
    unsigned int *hist;
    int *err;
    PM_TRY(mem.get(&dLo, N));
    PM_TRY(mem.get(&dHi, N));
    PM_TRY(mem.get(&dNode, (size_t)N * 4));
    PM_TRY(mem.get(&dRad, N));
    PM_TRY(mem.get(&dLeafOf, n));
    PM_TRY(mem.get(&ratio, (size_t)npairs));
    PM_TRY(mem.get(&hist, 256));
    PM_TRY(mem.get(&err, 1));
    PM_CUDA(cudaMemcpyAsync(dLo, pLo.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(dHi, pHi.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(dNode, nodeH.data(), N * 4 * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(dLeafOf, lof.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    PM_LAUNCH("k_node_ball", st, k_node_ball<<<(unsigned)N, 256, 0, st>>>(lx->O64, dLo, dHi, lx->m, dRad));
    PM_LAUNCH("k_gamma_ratio", st, k_gamma_ratio<<<(unsigned)(n - 1), 256, 0, st>>>(lx->O64, n, lx->m, dLeafOf, dNode,
                                                                                     dRad, ratio, err));
    PM_CUDA(cudaGetLastError());
    // exact rank-th smallest ratio: radix select, 8 passes of 8 bits
    int64_t rank = (int64_t)std::ceil(pr * (double)npairs - 1e-9);
    rank = std::max<int64_t>(1, std::min<int64_t>(npairs, rank));
    unsigned long long prefix = 0, hiMask = 0;
    unsigned int hh[256];
    const int grid = (int)std::min<int64_t>(4096, (npairs + 255) / 256);
    for (int shift = 56; shift >= 0; shift -= 8) {
        PM_CUDA(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st));
        PM_LAUNCH("k_gamma_hist", st, k_gamma_hist<<<grid, 256, 0, st>>>((const unsigned long long *)ratio, npairs,
                                                                           shift, hiMask, prefix, hist));
        PM_CUDA(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        int dg = 0;
        int64_t below = 0;
        while (dg < 255 && below + (int64_t)hh[dg] < rank) below += hh[dg++];
        rank -= below;
        prefix |= (unsigned long long)dg << shift;
        hiMask |= 0xFFull << shift;
    }
    int herr = 0;
    PM_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        pm_set_error("gamma calibration: the hierarchy is deeper than 4096 levels");
        return PMLSH_EINTERNAL;
    }
    double g;
    std::memcpy(&g, &prefix, sizeof(g));
    *gamma = g;
    return PMLSH_OK;
}

pmlsh_status pm_gamma_calibrate(pmlsh_index *ix, double pr, int64_t nsample, uint64_t seed, double *gamma,
                                cudaStream_t st)
{
    const int64_t n = ix->n;
    if (nsample >= n) return gamma_of_layout(ix, pr, gamma, st);
    // the sample: partial Fisher-Yates shuffle of 0..n-1 driven by the
    // counter-based stream `seed`, the first nsample ids sorted
    std::vector<int64_t> ids(n);
    for (int64_t i = 0; i < n; i++) ids[i] = i;
    for (int64_t i = 0; i < nsample; i++) {
        const int64_t j = i + (int64_t)(pm_splitmix64(seed, (uint64_t)i) % (uint64_t)(n - i));
        std::swap(ids[i], ids[j]);
    }
    ids.resize(nsample);
    std::sort(ids.begin(), ids.end());
    // their rows (original order) from the leaf-order copy of X
    std::vector<int64_t> inv(n), pos(nsample);
    for (int64_t p = 0; p < n; p++) inv[ix->permH[p]] = p;
    for (int64_t i = 0; i < nsample; i++) pos[i] = inv[ids[i]];
    DevPtrs mem;
    int64_t *dPos;
    float *S;
    PM_TRY(mem.get(&dPos, nsample));
    PM_TRY(mem.get(&S, (size_t)nsample * ix->d));
    PM_CUDA(cudaMemcpyAsync(dPos, pos.data(), nsample * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_LAUNCH("k_gather_rows", st, k_gather_rows<<<(unsigned)nsample, 128, 0, st>>>(ix->X, ix->ld, ix->d, dPos, nsample, S));
    PM_CUDA(cudaGetLastError());
    // the layout of the sample: the same build with the same projection,
    // pivot count and leaf capacity
    pmlsh_build_opts bo;
    pmlsh_build_opts_default(&bo);
    bo.m = ix->m;
    bo.s = ix->s;
    bo.leaf_size = ix->M;
    bo.seed = ix->seed;
    bo.proj = ix->A_host.data();
    bo.bf16_shadow = 0;
    pmlsh_index *sub = nullptr;
    pmlsh_status s = pmlsh_build(S, nsample, ix->d, &bo, st, &sub);
    if (s == PMLSH_OK) s = gamma_of_layout(sub, pr, gamma, st);
    pmlsh_free(sub);
    return s;
}

pmlsh_status pm_closest_pair(pmlsh_index *ix, const pmlsh_cp_opts *o, int64_t *out_pairs, float *out_dists,
                             pmlsh_cp_stats *stats, cudaStream_t st)
{
    const int64_t n = ix->n, L = ix->L;
    const int k = o->k;
    const double t = o->t > 0.0 ? o->t : std::sqrt(pm_chi2_upper_quantile(o->alpha1, ix->m));
    double gamma = o->gamma;
    if (!(gamma > 0.0)) PM_TRY(pm_gamma_calibrate(ix, 0.85, 10000, ix->seed + 7, &gamma, st));
    const int64_t T = o->T > 0 ? o->T : (int64_t)std::ceil(o->alpha2 * (double)n * (double)(n - 1) - 1e-9) + k;
    DevPtrs mem;
    // 1. self-join of every leaf
    std::vector<int64_t> pairOff(L + 1, 0);
    for (int64_t l = 0; l < L; l++) {
        int64_t s = ix->leafOffH[l + 1] - ix->leafOffH[l];
        pairOff[l + 1] = pairOff[l] + s * (s - 1) / 2;
    }
    const int64_t nSelf = pairOff[L];
    int64_t *dPairOff;
    PairCand *pairs;
    unsigned int *hist;
    PairExact *scratch;
    unsigned long long *cnt;
    PM_TRY(mem.get(&dPairOff, L + 1));
    PM_TRY(mem.get(&pairs, (size_t)std::max<int64_t>(nSelf, 1)));
    PM_TRY(mem.get(&hist, 2048));
    PM_TRY(mem.get(&scratch, PAIR_SORT_CAP));
    PM_TRY(mem.get(&cnt, 4));
    PM_CUDA(cudaMemcpyAsync(dPairOff, pairOff.data(), (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_TRY(pm_allow_max_dyn_smem((const void *)k_pair_sort));
    if (nSelf > 0) {
        PM_LAUNCH("k_cp_selfjoin", st, k_cp_selfjoin<<<(unsigned)L, 128, 0, st>>>(ix->X, ix->ld, ix->leafOff, dPairOff, pairs));
        PM_CUDA(cudaGetLastError());
    }
    TopK top;
    PM_TRY(pair_merge(top, k, pairs, nSelf, ix, hist, scratch, cnt, st));
    int64_t count = nSelf;
    double ub = (int)top.v.size() >= k ? top.v[k - 1].dist : INFINITY;
    const double ubSelf = ub;
    const double R = gamma * t * ub;
    // 2. node balls (FP64) and FindLCA (Algorithm 5) over the hierarchy
    const int64_t N = (int64_t)ix->nodeLo.size();
    std::vector<int64_t> pLo(N), pHi(N);
    for (int64_t e = 0; e < N; e++) {
        pLo[e] = ix->leafOffH[ix->nodeLo[e]];
        pHi[e] = ix->leafOffH[ix->nodeHi[e]];
    }
    int64_t *dLo, *dHi;
    double *dRad;
    PM_TRY(mem.get(&dLo, N));
    PM_TRY(mem.get(&dHi, N));
    PM_TRY(mem.get(&dRad, N));
    PM_CUDA(cudaMemcpyAsync(dLo, pLo.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_CUDA(cudaMemcpyAsync(dHi, pHi.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PM_LAUNCH("k_node_ball", st, k_node_ball<<<(unsigned)N, 256, 0, st>>>(ix->O64, dLo, dHi, ix->m, dRad));
    PM_CUDA(cudaGetLastError());
    std::vector<double> rad(N);
    PM_CUDA(cudaMemcpyAsync(rad.data(), dRad, N * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> A;
    {
        std::vector<int64_t> stack{0};
        while (!stack.empty()) {
            int64_t e = stack.back();
            stack.pop_back();
            if (ix->nodeLeft[e] < 0) continue;             // leaf nodes are never inserted
            if (rad[e] < R) { A.push_back(e); continue; }
            stack.push_back(ix->nodeRight[e]);             // visit left first (order is irrelevant:
            stack.push_back(ix->nodeLeft[e]);              // A is sorted below)
        }
        std::sort(A.begin(), A.end(), [&rad](int64_t x, int64_t y) { return rad[x] < rad[y] || (rad[x] == rad[y] && x < y); });
    }
    // leaf of each position
    int32_t *dLeafOf;
    PM_TRY(mem.get(&dLeafOf, n));
    {
        std::vector<int32_t> lof(n);
        for (int64_t l = 0; l < L; l++)
            for (int64_t p = ix->leafOffH[l]; p < ix->leafOffH[l + 1]; p++) lof[p] = (int32_t)l;
        PM_CUDA(cudaMemcpyAsync(dLeafOf, lof.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    // 3. nodes in ascending radius while count <= T
    int64_t nodesDone = 0, fp64 = 0;
    PairCand *cand = nullptr;
    size_t candCap = 0;
    for (size_t ai = 0; ai < A.size() && count <= T; ai++) {
        const int64_t e = A[ai];
        const int64_t lo = pLo[e], hi = pHi[e];
        const double Rt = t * ub;
        int64_t ncand = 0;
        for (int attempt = 0; attempt < 2; attempt++) {
            if (!cand) {
                candCap = std::max<size_t>(candCap, (size_t)1 << 20);
                PM_TRY(mem.get(&cand, candCap));
            }
            PM_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
            float loT = -1.f, hiT = INFINITY;
            if (!std::isinf(Rt)) {
                const double eps = 0x1.0p-22 * ix->maxNorm + 0x1.0p-19 * Rt + 1e-300;
                loT = Rt - eps > 0 ? (float)((Rt - eps) * (Rt - eps)) : -1.f;
                if ((double)loT > (Rt - eps) * (Rt - eps)) loT = nextafterf(loT, -INFINITY);
                hiT = (float)((Rt + eps) * (Rt + eps));
                if ((double)hiT < (Rt + eps) * (Rt + eps)) hiT = nextafterf(hiT, INFINITY);
            } else {
                loT = INFINITY;   // every pair is a candidate
                hiT = INFINITY;
            }
            PM_LAUNCH("k_cp_node_pairs", st, k_cp_node_pairs<<<(unsigned)((hi - lo + 127) / 128), 128, 0, st>>>(
                ix->O32, ix->O64, ix->m, dLeafOf, lo, hi, loT, hiT, Rt, cand, cnt, candCap, cnt + 1));
            PM_CUDA(cudaGetLastError());
            unsigned long long hc[2];
            PM_CUDA(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
            PM_CUDA(cudaStreamSynchronize(st));
            fp64 += (int64_t)hc[1];
            if (hc[0] <= candCap) { ncand = (int64_t)hc[0]; break; }
            // grow and redo this node
            candCap = (size_t)hc[0];
            cand = nullptr;
            if (attempt == 1) {
                pm_set_error("closest pairs: candidate buffer growth failed");
                return PMLSH_EINTERNAL;
            }
        }
        int64_t keep = ncand;
        if (count + ncand > T) PM_TRY(pair_truncate(cand, ncand, T + 1 - count, ix, hist, scratch, cnt, &keep, st));
        if (keep > 0) {
            PM_LAUNCH("k_pair_dist32", st, k_pair_dist32<<<(unsigned)((keep + 255) / 256), 256, 0, st>>>(ix->X, ix->ld, cand, keep));
            PM_TRY(pair_merge(top, k, cand, keep, ix, hist, scratch, cnt, st));
        }
        count += keep;
        ub = (int)top.v.size() >= k ? top.v[k - 1].dist : INFINITY;
        nodesDone++;
    }
    // results
    std::vector<int64_t> op((size_t)2 * k, -1);
    std::vector<float> od(k, INFINITY);
    for (int e = 0; e < k && e < (int)top.v.size(); e++) {
        op[2 * e] = top.v[e].i;
        op[2 * e + 1] = top.v[e].j;
        od[e] = (float)top.v[e].dist;
    }
    PM_CUDA(cudaMemcpy(out_pairs, op.data(), op.size() * sizeof(int64_t),
                       pm_is_device_ptr(out_pairs) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    PM_CUDA(cudaMemcpy(out_dists, od.data(), od.size() * sizeof(float),
                       pm_is_device_ptr(out_dists) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    if (stats) {
        stats->count = count;
        stats->ub_self = ubSelf;
        stats->lca_nodes = (int64_t)A.size();
        stats->nodes_done = nodesDone;
        stats->self_pairs = nSelf;
        stats->fp64_checks = fp64;
        stats->t = t;
        stats->T = T;
        stats->gamma = gamma;
    }
    return PMLSH_OK;
}

// Algorithm 3 (Sec. 6.1): the T pairs nearest in the projected space, found
// by branch and bound over leaf pairs, verified, cut to the k nearest.
//   1. every leaf's self-join, keyed by projected distance; if it yields T
//      pairs, the T-th of them bounds d_T from above;
//   2. Mindist of every leaf pair (a flat stand-in for the priority queue
//      over node pairs: with a lower bound per leaf pair the same pairs are
//      examined), the pairs with Mindist <= that bound taken in ascending
//      (Mindist, l1, l2);
//   3. their cross pairs in batches; after each batch the candidates are cut
//      to the exact T nearest (FP64-resolved band at the cut) and the search
//      stops at the first leaf pair whose Mindist exceeds the T-th distance;
//   4. the T pairs verified in the original space, exact top-k.
// The result equals the oracle's: the T pairs with the smallest (FP64
// projected distance, i, j), then the k smallest (FP64 distance, i, j).
pmlsh_status pm_closest_pair_bnb(pmlsh_index *ix, const pmlsh_cp_opts *o, int64_t *out_pairs, float *out_dists,
                                 pmlsh_cp_stats *stats, cudaStream_t st)
{
    const int64_t n = ix->n, L = ix->L;
    const int k = o->k;
    const int64_t P = n * (n - 1) / 2;
    int64_t T = o->T > 0 ? o->T : (int64_t)std::ceil(o->alpha2 * (double)n * (double)(n - 1) - 1e-9) + k;
    T = std::min(std::max<int64_t>(T, k), P);
    DevPtrs mem;
    unsigned int *hist;
    PairExact *scratch;
    unsigned long long *cnt;
    PM_TRY(mem.get(&hist, 2048));
    PM_TRY(mem.get(&scratch, PAIR_SORT_CAP));
    PM_TRY(mem.get(&cnt, 4));
    PM_TRY(pm_allow_max_dyn_smem((const void *)k_pair_sort));
    // 1. self-joins
    std::vector<int64_t> pairOff(L + 1, 0);
    for (int64_t l = 0; l < L; l++) {
        const int64_t s = ix->leafOffH[l + 1] - ix->leafOffH[l];
        pairOff[l + 1] = pairOff[l] + s * (s - 1) / 2;
    }
    const int64_t nSelf = pairOff[L];
    // candidate buffer: up to T kept pairs followed by a batch
    const int64_t batchCap = std::max<int64_t>((int64_t)1 << 24, nSelf);
    PairCand *buf, *sel;
    int64_t *dPairOff;
    PM_TRY(mem.get(&buf, (size_t)(T + batchCap)));
    PM_TRY(mem.get(&sel, (size_t)T));
    PM_TRY(mem.get(&dPairOff, L + 1));
    PM_CUDA(cudaMemcpyAsync(dPairOff, pairOff.data(), (L + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (nSelf > 0)
        PM_LAUNCH("k_bnb_selfjoin", st, k_bnb_selfjoin<<<(unsigned)L, 128, 0, st>>>(ix->O32, ix->leafOff, dPairOff, buf));
    PM_CUDA(cudaGetLastError());
    int64_t nBuf = nSelf, fp64 = 0;
    double dT = INFINITY;   // upper bound of the T-th projected distance
    auto cut = [&]() -> pmlsh_status {
        if (nBuf <= T) return PMLSH_OK;
        double tauHi = INFINITY;
        PM_TRY(pair_select(buf, nBuf, T, sel, ix, hist, scratch, cnt, &fp64, &tauHi, st));
        PM_CUDA(cudaMemcpyAsync(buf, sel, T * sizeof(PairCand), cudaMemcpyDeviceToDevice, st));
        nBuf = T;
        dT = std::min(dT, tauHi);
        return PMLSH_OK;
    };
    PM_TRY(cut());
    // 2./3. leaf pairs in bands of Mindist, (lo, hi]: each band's pairs in
    // ascending (Mindist, l1, l2), cut to the T nearest after each batch;
    // the search ends at the first leaf pair whose Mindist exceeds the T-th
    // projected distance (dT), and once a band's upper end reaches dT no
    // later band holds such a pair.  The first band ends at a generous
    // quantile of a sample of projected pair distances (near the T-th
    // distance), so that the leaf pairs listed stay few; each further band
    // quadruples the quantile.
    std::vector<double> F;
    PM_TRY(pm_distance_sample(ix, (int64_t)1 << 16, ix->seed + 8, F, st));
    const double pT = (double)T / (double)P;
    double pBand = std::min(1.0, 4.0 * pT + 64.0 / (double)F.size());
    auto quantile = [&](double p) -> double {
        if (p >= 1.0 || F.empty()) return INFINITY;
        const int64_t r = std::min<int64_t>((int64_t)F.size() - 1, (int64_t)std::ceil(p * (double)F.size()));
        return F[r];
    };
    double bandHi = quantile(pBand);
    float lo32 = -INFINITY;   // FP32 end of the previous band: bands are disjoint in FP32
    LeafPair *dlp;
    const unsigned long long lpCap = (unsigned long long)std::max<int64_t>(1, L * (L - 1) / 2);
    PM_TRY(mem.get(&dlp, (size_t)lpCap));
    int2 *dPairs;
    int64_t *dOff;
    const size_t lpBatch = (size_t)1 << 16;
    PM_TRY(mem.get(&dPairs, lpBatch));
    PM_TRY(mem.get(&dOff, lpBatch));
    unsigned long long *keyA = nullptr, *keyB = nullptr;   // device sort of the listed leaf pairs
    unsigned int *rsHist = nullptr;
    unsigned long long keyCap = 0;
    int64_t examined = 0, crossPairs = 0, listed = 0;
    for (;;) {
        const double hiCut = std::min(bandHi, dT);
        PM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
        // the band is (lo32, hi32] in FP32 Mindist, hi32 >= hiCut
        const float hi32 = std::isinf(hiCut) ? INFINITY : nextafterf((float)hiCut, INFINITY);
        if (L > 1)
            PM_LAUNCH("k_bnb_mindist", st, k_bnb_mindist<<<(unsigned)L, 256, 0, st>>>(ix->leafMeta, ix->s, L, lo32,
                                                                                       hi32, dlp, cnt, lpCap));
        PM_CUDA(cudaGetLastError());
        unsigned long long nlp = 0;
        PM_CUDA(cudaMemcpyAsync(&nlp, cnt, sizeof(nlp), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        const bool gpuSort = L <= LP_GPU_MAX_L && nlp > 1;
        if (gpuSort) {
            // ascending (Mindist, l1, l2) by the device radix sort
            if (nlp > keyCap) {
                PM_TRY(mem.get(&keyA, (size_t)nlp));
                PM_TRY(mem.get(&keyB, (size_t)nlp));
                PM_TRY(mem.get(&rsHist, (size_t)256 * ((nlp + RS_THREADS * RS_ITEMS - 1) / (RS_THREADS * RS_ITEMS))));
                keyCap = nlp;
            }
            const int64_t nl = (int64_t)nlp;
            const int nb = (int)((nl + RS_THREADS * RS_ITEMS - 1) / (RS_THREADS * RS_ITEMS));
            const unsigned g = (unsigned)((nl + 255) / 256);
            PM_LAUNCH("k_lp_key", st, k_lp_key<<<g, 256, 0, st>>>(dlp, nl, L, keyA));
            unsigned long long *src = keyA, *dst = keyB;
            for (int shift = 0; shift < 64; shift += 8) {
                PM_LAUNCH("k_rs_hist", st, k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, st>>>(src, nl, shift, rsHist, nb));
                PM_LAUNCH("k_rs_scan", st, k_rs_scan<<<1, 1024, 0, st>>>(rsHist, (int64_t)256 * nb));
                PM_LAUNCH("k_rs_scatter", st, k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, st>>>(src, dst, nl, shift,
                                                                                              rsHist, nb));
                std::swap(src, dst);
            }
            PM_CUDA(cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned long long), st));
            PM_LAUNCH("k_lp_decode", st, k_lp_decode<<<g, 256, 0, st>>>(src, nl, L, dlp, (int *)(cnt + 1)));
            PM_CUDA(cudaGetLastError());
        }
        std::vector<LeafPair> lps(nlp);
        PM_CUDA(cudaMemcpyAsync(lps.data(), dlp, nlp * sizeof(LeafPair), cudaMemcpyDeviceToHost, st));
        if (gpuSort) {
            unsigned long long badH = 0;
            PM_CUDA(cudaMemcpyAsync(&badH, cnt + 1, sizeof(badH), cudaMemcpyDeviceToHost, st));
            PM_CUDA(cudaStreamSynchronize(st));
            if (badH != 0) {
                pm_set_error("closest pairs: the device sort of %llu leaf pairs failed its check (%llu)", nlp, badH);
                return PMLSH_EINTERNAL;
            }
        } else {
            PM_CUDA(cudaStreamSynchronize(st));
            std::sort(lps.begin(), lps.end(), [](const LeafPair &x, const LeafPair &y) {
                if (x.md != y.md) return x.md < y.md;
                if (x.l1 != y.l1) return x.l1 < y.l1;
                return x.l2 < y.l2;
            });
        }
        listed += (int64_t)nlp;
        size_t next = 0;
        bool stop = false;
        while (next < lps.size()) {
            if ((double)lps[next].md > dT) { stop = true; break; }   // no pair under it can beat the T-th
            std::vector<int2> bp;
            std::vector<int64_t> bo;
            int64_t tot = 0;
            while (next < lps.size() && bp.size() < lpBatch && (double)lps[next].md <= dT) {
                const int64_t na = ix->leafOffH[lps[next].l1 + 1] - ix->leafOffH[lps[next].l1];
                const int64_t nb = ix->leafOffH[lps[next].l2 + 1] - ix->leafOffH[lps[next].l2];
                if (tot > 0 && tot + na * nb > batchCap) break;
                bp.push_back(make_int2(lps[next].l1, lps[next].l2));
                bo.push_back(nBuf + tot);
                tot += na * nb;
                next++;
            }
            if (tot > batchCap) {
                pm_set_error("closest pairs: one leaf pair holds more pairs than the batch capacity");
                return PMLSH_EINTERNAL;
            }
            PM_CUDA(cudaMemcpyAsync(dPairs, bp.data(), bp.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
            PM_CUDA(cudaMemcpyAsync(dOff, bo.data(), bo.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            PM_LAUNCH("k_bnb_cross", st, k_bnb_cross<<<(unsigned)bp.size(), 256, 0, st>>>(ix->O32, ix->leafOff, dPairs,
                                                                                            dOff, buf));
            PM_CUDA(cudaGetLastError());
            nBuf += tot;
            examined += (int64_t)bp.size();
            crossPairs += tot;
            PM_TRY(cut());
        }
        // done when this band reached dT (every later pair has Mindist > dT)
        // or covered everything
        if (stop || std::isinf(bandHi) || dT <= bandHi) break;
        lo32 = hi32;
        pBand = std::min(1.0, pBand * 4.0);
        bandHi = std::max(quantile(pBand), (double)hi32);
    }
    // 4. verification and the exact top-k
    if (nBuf > 0)
        PM_LAUNCH("k_pair_dist32", st, k_pair_dist32<<<(unsigned)((nBuf + 255) / 256), 256, 0, st>>>(ix->X, ix->ld, buf, nBuf));
    TopK top;
    PM_TRY(pair_merge(top, k, buf, nBuf, ix, hist, scratch, cnt, st));
    std::vector<int64_t> op((size_t)2 * k, -1);
    std::vector<float> od(k, INFINITY);
    for (int e = 0; e < k && e < (int)top.v.size(); e++) {
        op[2 * e] = top.v[e].i;
        op[2 * e + 1] = top.v[e].j;
        od[e] = (float)top.v[e].dist;
    }
    PM_CUDA(cudaMemcpy(out_pairs, op.data(), op.size() * sizeof(int64_t),
                       pm_is_device_ptr(out_pairs) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    PM_CUDA(cudaMemcpy(out_dists, od.data(), od.size() * sizeof(float),
                       pm_is_device_ptr(out_dists) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    if (stats) {
        stats->count = nBuf;
        stats->ub_self = INFINITY;
        stats->lca_nodes = listed;
        stats->nodes_done = examined;
        stats->self_pairs = nSelf;
        stats->fp64_checks = fp64;
        stats->t = 0.0;
        stats->T = T;
        stats->gamma = o->gamma;
    }
    (void)crossPairs;
    return PMLSH_OK;
}
