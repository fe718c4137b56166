// (c,k)-ANN query path: Algorithm 2 over a batch of queries.
//
// One round of Algorithm 2 for every still-active query is a fixed sequence
// of kernels:
//   k_thresholds   radius R = t r and the FP32 classification thresholds
//   k_class        Eq. 5 leaf test for (query block x leaf); counts whole-leaf
//                  members and lists, per query block, the leaves that some
//                  query covers partially, with the bit mask of those queries
//   k_count        per-point test in partially covered leaves; points whose
//   (k_count_tc)   FP32 distance is inside the error band go to a band list
//                  (k_count_tc: the same decisions from tensor-core dot
//                  products, PMLSH_BF16_TENSOR)
//   k_band64       FP64 decision for band points (equal to the FP64 oracle)
//   [host]         |S_i| per query -> which queries reach the budget B
//   k_collect,     for budget queries: the B nearest in projected space
//   k_select       (radix select, FP64 resolution of the band at the cut)
//   k_verify       one warp per query: exact FP32 distances of the candidates
//                  that can reach the top-k (leaves visited best first by an
//                  original-space lower bound, chunks of <= 32 points skipped
//                  by their own), guard set, FP64 distances, exact top-k and
//                  the k-th distance for stop rule 1
//   [host]         stop rules, r <- c r for the rest
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>

#include "knn_shared.cuh"

namespace {

using namespace pmk;


// ------------------------------------------------------------ prep kernels

// Routes each query down the bisection hierarchy to a leaf (locality key).
__global__ void k_leaf_key(const float *__restrict__ qp32, int64_t nq, const int32_t *__restrict__ T,
                           const float *__restrict__ V, unsigned int *__restrict__ key)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    int e = 0;
    for (int guard = 0; guard < 4096; guard++) {
        int l = T[e * 4 + 0];
        if (l < 0) break;
        const float *w = V + (int64_t)e * (PM_MP + 1);
        float s = 0.f;
        for (int j = 0; j < PM_MP; j++) s = fmaf(w[j], qp32[q * PM_MP + j], s);
        e = s < w[PM_MP] ? l : T[e * 4 + 1];
    }
    key[q] = (unsigned int)T[e * 4 + 3];
}

// q norms (FP64 coordinates) and FP32 distances to the pivots.
__global__ void k_query_aux(const double *__restrict__ qp64, const float *__restrict__ qp32,
                            int64_t nq, const float *__restrict__ piv, int s,
                            double *__restrict__ qnorm, float *__restrict__ qpiv)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double nn = 0.0;
    for (int j = 0; j < PM_MP; j++) nn = fma(qp64[q * PM_MP + j], qp64[q * PM_MP + j], nn);
    qnorm[q] = sqrt(nn);
    for (int i = 0; i < PM_MAX_PIVOTS; i++)
        qpiv[q * PM_MAX_PIVOTS + i] = i < s ? sqrtf(pm_pd2_32(qp32 + q * PM_MP, piv + i * PM_MP)) : 0.f;
}

// Query coordinates along the leaf centres' principal directions in FP32
// (P rounded to FP32, sequential fma over the row; each coordinate within
// (ld + 2) 2^-24 ||q|| of the exact one, which the verification's slack
// covers) and ||q|| (FP64, rounded up to FP32).  One thread per query.
__global__ void k_query_pca(const float *__restrict__ Qd, int64_t nq, int ld, const float *__restrict__ P,
                            float *__restrict__ qpca, float *__restrict__ qnx)
{
    // one warp per query: lanes over the coordinates (16-byte loads), one
    // partial sum per direction and lane, then a butterfly (any summation
    // order is within the slack of the bound that uses P q)
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;   // warp-uniform
    const float4 *x4 = (const float4 *)(Qd + q * ld);
    const int nf4 = ld >> 2;
    float acc[PM_PCA];
#pragma unroll
    for (int r = 0; r < PM_PCA; r++) acc[r] = 0.f;
    double nn = 0.0;
    for (int j4 = lane; j4 < nf4; j4 += 32) {
        const float4 xv = x4[j4];
        nn = fma((double)xv.x, (double)xv.x, nn);
        nn = fma((double)xv.y, (double)xv.y, nn);
        nn = fma((double)xv.z, (double)xv.z, nn);
        nn = fma((double)xv.w, (double)xv.w, nn);
#pragma unroll
        for (int r = 0; r < PM_PCA; r++) {
            const float4 pv = ((const float4 *)(P + (int64_t)r * ld))[j4];
            acc[r] = __fmaf_rn(pv.x, xv.x, acc[r]);
            acc[r] = __fmaf_rn(pv.y, xv.y, acc[r]);
            acc[r] = __fmaf_rn(pv.z, xv.z, acc[r]);
            acc[r] = __fmaf_rn(pv.w, xv.w, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < PM_PCA; r++)
        for (int o = 16; o; o >>= 1) acc[r] = __fadd_rn(acc[r], __shfl_xor_sync(0xffffffffu, acc[r], o));
    for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane < PM_PCA) {
        float v = acc[0];
#pragma unroll
        for (int r = 1; r < PM_PCA; r++) v = lane == r ? acc[r] : v;
        qpca[q * PM_PCA + lane] = v;
    }
    // ||q|| for the slack: the FP64 sum (any order, within 2^-45 relative of
    // exact) rounded up to FP32 with a relative margin
    if (lane == 0) qnx[q] = __double2float_ru(sqrt(nn) * (1.0 + 0x1.0p-40));
}

__global__ void k_thresholds(const int32_t *__restrict__ act, int na, const double *__restrict__ r,
                             double t, double maxNorm, const double *__restrict__ qnorm,
                             Thr *__restrict__ thr)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    int q = act[a];
    double R = t * r[q];
    double eps = band_eps(R, maxNorm, qnorm[q]);
    Thr T;
    T.R = R;
    T.lo = R - eps > 0.0 ? __double2float_rd((R - eps) * (R - eps)) : -1.f;
    T.hi = __double2float_ru((R + eps) * (R + eps));
    T.lov = T.lo;
    T.pad = 0.f;
    thr[a] = T;
}

// ------------------------------------------------------------ range round

// Leaf classification of a round (Eq. 5): for a block of QBT active queries,
// the leaves that some query of the block covers only partially are listed
// for the block as {leaf, first position, size, first tensor-operand row},
// each with the QBT-bit mask of those queries (bit qq of word qq / 32).  Also,
// per query, the bit set of the leaves that Eq. 5 does not exclude
// (leafBits [active query][ceil(L / 32)]), which the verification kernel
// walks instead of testing every leaf again, and the whole-leaf sizes
// (cntSure) and partial-leaf sizes (cntPart), which bound |S_i| from below
// and above.  The test is leaf_class's with the same slack and cheaper
// arithmetic: the centre test on the squared distance against thresholds
// rounded outward (no square root), the pivot-ring tests against per-query
// thresholds precomputed with directed rounding.  Every decision is implied
// by the exact form of leaf_class's inequalities (so a leaf called out holds
// no point within Rout and a full one only points within Rin); the two tests
// may differ only at those slack boundaries.
constexpr float CL_INV_LO = 1.0f / (1.f - SLACK) * (1.f + 1e-7f);   // >= 1 / (1 - SLACK)
constexpr float CL_INV_HI = 1.0f / (1.f + SLACK) * (1.f - 1e-7f);   // <= 1 / (1 + SLACK)

// Query-stationary form (and, on request, the bit set of the leaves the test
// calls full, fullBits): thread qq of the CTA
// holds query qq of the block (coordinates as packed pairs and its pivot
// thresholds in registers) and the CTA walks its share of the leaves in tiles
// of CQ_LT, reading each leaf record with loads that every lane of a warp
// shares.  A thread keeps its whole-leaf and partial sizes and its leaf
// bit-set words in registers.  The centre test is the only work for a
// (query, leaf) pair that it excludes; the pivot rings, the full-leaf test,
// the counts and the ballot of the partial-leaf mask run only for a leaf
// that some query of the warp keeps.  The warps' masks of a tile meet in
// shared memory (double-buffered, one barrier per tile), where the tile's
// partially covered leaves are listed.  Queries beyond the batch sit at
// +1e18 on every coordinate, so the centre test excludes them.
constexpr int CQ_LT = 256;   // leaves per tile: eight bit-set words (one 32-byte sector) per query
// words per query in a leaf bit set: L bits padded to whole tiles
static inline int64_t pm_leaf_words(int64_t L) { return (L + CQ_LT - 1) / CQ_LT * (CQ_LT / 32); }

template <int QBT>
__global__ void __launch_bounds__(QBT, QBT == 256 ? 4 : 16)
k_class(const int32_t *__restrict__ act, int na, const Thr *__restrict__ thr,
        const float *__restrict__ qp32, const float *__restrict__ qpiv, int s,
        const float *__restrict__ meta, const int64_t *__restrict__ off, const int64_t *__restrict__ bOff,
        int64_t L, int *__restrict__ cntSure, int *__restrict__ blkCnt, int4 *__restrict__ blkEnt,
        uint32_t *__restrict__ blkMask, uint32_t *__restrict__ leafBits, int W32, int *__restrict__ cntPart,
        uint32_t *__restrict__ fullBits)
{
    constexpr int W = QBT / 32;   // warps = mask words per list entry
    constexpr int NWD = CQ_LT / 32;   // bit-set words per query and tile
    __shared__ uint32_t sM[2][CQ_LT][W];
    __shared__ uint32_t sW[NWD][QBT];   // the thread's words of the tile, written out as whole sectors
    __shared__ uint32_t sF[NWD][QBT];   // the same for the whole-leaf bits
    const int b = blockIdx.y;
    const int a0 = b * QBT;
    const int nb = min(QBT, na - a0);
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    for (int e = t; e < 2 * CQ_LT * W; e += QBT) (&sM[0][0][0])[e] = 0u;

    unsigned long long qv[PM_MP / 2];
    // per pivot: out if HR.max < lowT or HR.min > highT
    float lowT[PM_MAX_PIVOTS], highT[PM_MAX_PIVOTS];
    float roL = 0.f, rinLo = -1.f;   // Rout (1 + SLACK) CL_INV_LO rounded up; Rin (1 - SLACK) rounded down
    const bool qv_ok = t < nb;
    if (qv_ok) {
        const int q = act[a0 + t];
        const float4 *src = (const float4 *)(qp32 + (int64_t)q * PM_MP);
#pragma unroll
        for (int j4 = 0; j4 < PM_MP / 4; j4++) {
            const float4 v = src[j4];
            qv[2 * j4] = f32x2_pack(v.x, v.y);
            qv[2 * j4 + 1] = f32x2_pack(v.z, v.w);
        }
        const Thr T = thr[a0 + t];
        const float Rin = T.lo > 0.f ? __fsqrt_rn(T.lo) : -1.f;
        const float ro = __fmul_ru(__fsqrt_rn(T.hi), 1.f + SLACK);
        roL = __fmul_ru(ro, CL_INV_LO);
        rinLo = Rin > 0.f ? __fmul_rd(Rin, 1.f - SLACK) : -1.f;
#pragma unroll
        for (int i = 0; i < PM_MAX_PIVOTS; i++) {
            const float dq = qpiv[(int64_t)q * PM_MAX_PIVOTS + i];
            // pivots beyond s never exclude
            lowT[i] = i < s ? __fsub_rd(__fmul_rd(dq, 1.f - SLACK), ro) : -INFINITY;
            highT[i] = i < s ? __fadd_ru(__fmul_ru(dq, 1.f + SLACK), ro) : INFINITY;
        }
    } else {
#pragma unroll
        for (int j = 0; j < PM_MP / 2; j++) qv[j] = f32x2_pack(1e18f, 1e18f);
#pragma unroll
        for (int i = 0; i < PM_MAX_PIVOTS; i++) {
            lowT[i] = -INFINITY;
            highT[i] = INFINITY;
        }
    }
    __syncthreads();
    int sure = 0, part = 0;
    const int64_t nTiles = (L + CQ_LT - 1) / CQ_LT;
    int buf = 0;
    for (int64_t tile = blockIdx.x; tile < nTiles; tile += gridDim.x, buf ^= 1) {
        const int64_t l0 = tile * CQ_LT;
        const int nl = L - l0 < CQ_LT ? (int)(L - l0) : CQ_LT;
#pragma unroll 1
        for (int w4 = 0; w4 < NWD; w4++) {
            uint32_t bits = 0u, fbits = 0u;
            const int jn = min(32, nl - w4 * 32);
#pragma unroll 2
            for (int jj = 0; jj < jn; jj++) {
                const int j = w4 * 32 + jj;
                const float *M = meta + (l0 + j) * PM_LEAF_STRIDE;
                const float4 *c4 = (const float4 *)M;
                unsigned long long acc0 = 0ull, acc1 = 0ull;
#pragma unroll
                for (int j4 = 0; j4 < PM_MP / 4; j4 += 2) {
                    const float4 v = __ldg(c4 + j4), u = __ldg(c4 + j4 + 1);
                    f32x2_sqdiff_acc(acc0, qv[2 * j4], f32x2_pack(v.x, v.y));
                    f32x2_sqdiff_acc(acc1, qv[2 * j4 + 1], f32x2_pack(v.z, v.w));
                    f32x2_sqdiff_acc(acc0, qv[2 * j4 + 2], f32x2_pack(u.x, u.y));
                    f32x2_sqdiff_acc(acc1, qv[2 * j4 + 3], f32x2_pack(u.z, u.w));
                }
                unsigned long long acc;
                asm("add.rn.f32x2 %0, %1, %2;" : "=l"(acc) : "l"(acc0), "l"(acc1));
                // out: sqrt(d^2) (1 - SLACK) - r > ro, i.e. d^2 > ((ro + r) / (1 - SLACK))^2
                const float rr = __ldg(M + 16);
                const float lo = __fadd_rd(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
                const float tb = __fadd_ru(roL, __fmul_ru(rr, CL_INV_LO));
                const bool in = !(lo > __fmul_ru(tb, tb));
                if (__any_sync(VW_FULL, in)) {
                    // pivot rings of Sec. 4.1, then the full-leaf test
                    unsigned char c = CL_OUT;
                    if (in) {
                        const float4 *h4 = (const float4 *)(M + 24);   // HR.min [8], HR.max [8]
                        const float4 n0 = __ldg(h4), n1 = __ldg(h4 + 1), x0 = __ldg(h4 + 2), x1 = __ldg(h4 + 3);
                        const bool out = x0.x < lowT[0] || x0.y < lowT[1] || x0.z < lowT[2] || x0.w < lowT[3] ||
                                         x1.x < lowT[4] || x1.y < lowT[5] || x1.z < lowT[6] || x1.w < lowT[7] ||
                                         n0.x > highT[0] || n0.y > highT[1] || n0.z > highT[2] || n0.w > highT[3] ||
                                         n1.x > highT[4] || n1.y > highT[5] || n1.z > highT[6] || n1.w > highT[7];
                        if (!out) {
                            c = CL_PART;
                            // full: sqrt(d^2) (1 + SLACK) + r <= Rin (1 - SLACK)
                            const float hi = __fadd_ru(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
                            const float f = __fmul_rd(__fsub_rd(rinLo, rr), CL_INV_HI);
                            if (rinLo > 0.f && f > 0.f && hi <= __fmul_rd(f, f)) c = CL_FULL;
                            const int n = (int)(__ldg(off + l0 + j + 1) - __ldg(off + l0 + j));
                            if (c == CL_FULL) {
                                sure += n;
                                fbits |= 1u << jj;
                            } else {
                                part += n;
                            }
                            bits |= 1u << jj;
                        }
                    }
                    const uint32_t m = __ballot_sync(VW_FULL, c == CL_PART);
                    if (lane == 0) sM[buf][j][wp] = m;
                }
            }
            sW[w4][t] = bits;
            sF[w4][t] = fbits;
        }
        // the tile's words of this query's leaf bit set: one 32-byte sector
        // (rows are W32 words, a multiple of 8, so the sector is aligned)
        if (qv_ok) {
            uint4 *dst = (uint4 *)(leafBits + (int64_t)(a0 + t) * W32 + l0 / 32);
            dst[0] = make_uint4(sW[0][t], sW[1][t], sW[2][t], sW[3][t]);
            dst[1] = make_uint4(sW[4][t], sW[5][t], sW[6][t], sW[7][t]);
            if (fullBits) {
                uint4 *fd = (uint4 *)(fullBits + (int64_t)(a0 + t) * W32 + l0 / 32);
                fd[0] = make_uint4(sF[0][t], sF[1][t], sF[2][t], sF[3][t]);
                fd[1] = make_uint4(sF[4][t], sF[5][t], sF[6][t], sF[7][t]);
            }
        }
        __syncthreads();
        // the tile's leaves that some query of the block covers partially;
        // the masks are cleared for the tile after next
        for (int j = t; j < nl; j += QBT) {
            uint32_t mw[W], any = 0u;
#pragma unroll
            for (int w = 0; w < W; w++) {
                mw[w] = sM[buf][j][w];
                any |= mw[w];
                sM[buf][j][w] = 0u;
            }
            if (any) {
                const int64_t l = l0 + j;
                const int slot = atomicAdd(&blkCnt[b], 1);
                const int64_t e = (int64_t)b * L + slot;
                blkEnt[e] = make_int4((int)l, (int)off[l], (int)(off[l + 1] - off[l]), bOff ? (int)bOff[l] : 0);
#pragma unroll
                for (int w = 0; w < W; w++) blkMask[e * W + w] = mw[w];
            }
        }
    }
    if (qv_ok) {
        if (sure) atomicAdd(&cntSure[a0 + t], sure);
        if (part) atomicAdd(&cntPart[a0 + t], part);
    }
}

// Tightened bounds of |S_i| for the active queries whose whole-leaf bounds
// (cntSure from below, cntSure + cntPart from above) straddle T = min(B, n);
// the others exit at once.  A CTA per query walks its partially covered
// leaves (leafBits without fullBits) and applies each leaf's radial profile
// (meta [17, 24): for g = 2 .. 8 an upper bound v_g of the ceil(g s / 8)-th
// largest member radius): with d the centre distance, members of radius
// < d (1 - SLACK) - Rout (1 + SLACK) lie beyond Rout and those of radius
// <= Rin (1 - SLACK) - d (1 + SLACK) within Rin (the leaf tests'
// inequalities for the sub-ball of the members from that rank on).
// cntTight[a] = (members of partial leaves surely inside, possibly inside).
__global__ void __launch_bounds__(256)
k_tight(const int32_t *__restrict__ act, int na, const Thr *__restrict__ thr, const float *__restrict__ qp32,
        const float *__restrict__ meta, const int64_t *__restrict__ off, const uint32_t *__restrict__ leafBits,
        const uint32_t *__restrict__ fullBits, int W32, int64_t L, const int *__restrict__ cntSure,
        const int *__restrict__ cntPart, int64_t T, int2 *__restrict__ cntTight)
{
    // one CTA per active query; a warp compacts the partial leaves of 32
    // bit-set words into shared memory, then its lanes take one leaf each
    __shared__ int sLeaf[8][1024];
    __shared__ int sRed[2][8];
    const int a = blockIdx.x;
    const int sure = cntSure[a], part = cntPart[a];
    if (sure >= T || (int64_t)sure + part < T) return;   // block-uniform
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int q = act[a];
    float qv[PM_MP];
#pragma unroll
    for (int j = 0; j < PM_MP; j++) qv[j] = qp32[(int64_t)q * PM_MP + j];
    const Thr th = thr[a];
    const float Rin = th.lo > 0.f ? __fsqrt_rn(th.lo) : -1.f;
    const float ro = __fmul_ru(__fsqrt_rn(th.hi), 1.f + SLACK);
    const float rinLo = Rin > 0.f ? __fmul_rd(Rin, 1.f - SLACK) : -1.f;
    int lb = 0, ub = 0;
    int *buf = sLeaf[wp];
    for (int w0 = wp * 32; w0 < W32; w0 += 8 * 32) {
        const int wi = w0 + lane;
        uint32_t word = 0u;
        if (wi < W32) word = leafBits[(int64_t)a * W32 + wi] & ~fullBits[(int64_t)a * W32 + wi];
        const int c = __popc(word);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int at = incl - c;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            buf[at++] = wi * 32 + b;
        }
        __syncwarp();
        for (int e = lane; e < total; e += 32) {
            const int64_t l = buf[e];
            if (l >= L) continue;
            const float *M = meta + l * PM_LEAF_STRIDE;
            // FP32 squared centre distance (its rounding is within SLACK)
            const float4 *c4 = (const float4 *)M;
            float d2 = 0.f;
#pragma unroll
            for (int j4 = 0; j4 < PM_MP / 4; j4++) {
                const float4 cc = __ldg(c4 + j4);
                float u = __fsub_rn(qv[4 * j4], cc.x);
                d2 = __fmaf_rn(u, u, d2);
                u = __fsub_rn(qv[4 * j4 + 1], cc.y);
                d2 = __fmaf_rn(u, u, d2);
                u = __fsub_rn(qv[4 * j4 + 2], cc.z);
                d2 = __fmaf_rn(u, u, d2);
                u = __fsub_rn(qv[4 * j4 + 3], cc.w);
                d2 = __fmaf_rn(u, u, d2);
            }
            const int n = (int)(off[l + 1] - off[l]);
            const float tOut = __fsub_rd(__fmul_rd(__fsqrt_rd(d2), 1.f - SLACK), ro);
            const float tIn = rinLo > 0.f ? __fsub_rd(rinLo, __fmul_ru(__fsqrt_ru(d2), 1.f + SLACK)) : -INFINITY;
            // v_g falls with g: the smallest g passing a test gives its bound
            int u1 = n, l1 = 0;
            const float4 r0 = __ldg((const float4 *)(M + 16)), r1 = __ldg((const float4 *)(M + 20));
            const float vg[7] = {r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
            for (int g = 2; g <= 8; g++) {
                const int kg = (g * n + 7) / 8;
                if (vg[g - 2] < tOut && u1 == n) u1 = kg - 1;
                if (vg[g - 2] <= tIn && l1 == 0) l1 = n - kg + 1;
            }
            lb += l1;
            ub += u1;
        }
        __syncwarp();
    }
    lb = __reduce_add_sync(0xffffffffu, lb);
    ub = __reduce_add_sync(0xffffffffu, ub);
    if (lane == 0) {
        sRed[0][wp] = lb;
        sRed[1][wp] = ub;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tl = 0, tu = 0;
        for (int w = 0; w < 8; w++) {
            tl += sRed[0][w];
            tu += sRed[1][w];
        }
        cntTight[a] = make_int2(tl, tu);
    }
}

// Block leaf lists of a gathered sub-batch from the classification its
// queries already have (the full batch's leafBits without fullBits: the
// partially covered leaves): for a block of QBT sub-batch queries, every
// leaf that some of them cover partially, with their QBT-bit mask, as
// k_class lists it; and the sub-batch's whole-leaf counts copied from the
// batch's.  Grid (block, chunk slice); a chunk is 8 bit-set words (256
// leaves); each warp turns its queries' words into per-leaf masks by ballots.
template <int QBT>
__global__ void __launch_bounds__(QBT)
k_sublists(const int32_t *__restrict__ amb, int na2, const uint32_t *__restrict__ leafBits,
           const uint32_t *__restrict__ fullBits, int W32, int64_t L, const int64_t *__restrict__ off,
           const int64_t *__restrict__ bOff, const int *__restrict__ cntSureAll, int *__restrict__ cntSure,
           int *__restrict__ blkCnt, int4 *__restrict__ blkEnt, uint32_t *__restrict__ blkMask)
{
    constexpr int W = QBT / 32;
    __shared__ uint32_t sM[256][W];
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int i = b * QBT + t;
    const bool ok = i < na2;
    const int a = ok ? amb[i] : 0;
    if (ok && blockIdx.y == 0) cntSure[i] = cntSureAll[a];
    for (int c = blockIdx.y; c * 8 < W32; c += gridDim.y) {
        uint32_t pw[8];
        if (ok) {
            // eight words of this query's rows: one aligned 32-byte sector each
            const uint4 *lb = (const uint4 *)(leafBits + (int64_t)a * W32 + c * 8);
            const uint4 *fb = (const uint4 *)(fullBits + (int64_t)a * W32 + c * 8);
            const uint4 l0 = lb[0], l1 = lb[1], f0 = fb[0], f1 = fb[1];
            pw[0] = l0.x & ~f0.x; pw[1] = l0.y & ~f0.y; pw[2] = l0.z & ~f0.z; pw[3] = l0.w & ~f0.w;
            pw[4] = l1.x & ~f1.x; pw[5] = l1.y & ~f1.y; pw[6] = l1.z & ~f1.z; pw[7] = l1.w & ~f1.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) pw[k] = 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const unsigned any = __ballot_sync(0xffffffffu, pw[k] != 0u);
#pragma unroll 4
            for (int j = 0; j < 32; j++) {
                const unsigned m = any ? __ballot_sync(0xffffffffu, (pw[k] >> j) & 1u) : 0u;
                if (lane == 0) sM[k * 32 + j][wp] = m;
            }
        }
        __syncthreads();
        for (int j = t; j < 256; j += QBT) {
            const int64_t l = (int64_t)c * 256 + j;
            uint32_t mw[W], any = 0u;
#pragma unroll
            for (int w = 0; w < W; w++) {
                mw[w] = sM[j][w];
                any |= mw[w];
            }
            if (l < L && any) {
                const int slot = atomicAdd(&blkCnt[b], 1);
                const int64_t e = (int64_t)b * L + slot;
                blkEnt[e] = make_int4((int)l, (int)off[l], (int)(off[l + 1] - off[l]), bOff ? (int)bOff[l] : 0);
#pragma unroll
                for (int w = 0; w < W; w++) blkMask[e * W + w] = mw[w];
            }
        }
        __syncthreads();
    }
}

// Per-point test in partially covered leaves (the queries of the block's
// list mask).  Grid (block, split).
__global__ void __launch_bounds__(256)
k_count(const int32_t *__restrict__ act, int na, const Thr *__restrict__ thr,
        const float *__restrict__ qp32, const float *__restrict__ O32,
        const int *__restrict__ blkCnt, const int4 *__restrict__ blkEnt,
        const uint32_t *__restrict__ blkMask, int64_t L,
        int *__restrict__ cntSure, int *__restrict__ cntBand,
        int *__restrict__ bandN, int bandCap, int *__restrict__ bandA, int *__restrict__ bandPos)
{
    __shared__ float sq[QB][PM_MP];
    __shared__ float sLo[QB], sHi[QB];
    __shared__ int sSure[QB], sBand[QB];
    const int b = blockIdx.x;
    const int a0 = b * QB;
    const int nb = min(QB, na - a0);
    for (int e = threadIdx.x; e < QB * PM_MP; e += blockDim.x) {
        int qq = e / PM_MP, j = e % PM_MP;
        sq[qq][j] = qq < nb ? qp32[(int64_t)act[a0 + qq] * PM_MP + j] : 0.f;
    }
    for (int qq = threadIdx.x; qq < QB; qq += blockDim.x) {
        if (qq < nb) {
            Thr T = thr[a0 + qq];
            sLo[qq] = T.lo;
            sHi[qq] = T.hi;
        }
        sSure[qq] = 0;
        sBand[qq] = 0;
    }
    __syncthreads();
    const int nl = blkCnt[b];
    for (int li = blockIdx.y; li < nl; li += gridDim.y) {
        const int64_t e = (int64_t)b * L + li;
        const int4 ent = blkEnt[e];
        const unsigned long long part =
            ((unsigned long long)blkMask[e * 2 + 1] << 32) | (unsigned long long)blkMask[e * 2];
        const int64_t p0 = ent.y, p1 = (int64_t)ent.y + ent.z;
        for (int64_t base = p0; base < p1; base += blockDim.x) {
            const int64_t pos = base + threadIdx.x;
            const bool valid = pos < p1;
            float o[PM_MP];
#pragma unroll
            for (int j = 0; j < PM_MP; j++) o[j] = valid ? O32[pos * PM_MP + j] : 0.f;
            unsigned long long bits = part;
            while (bits) {
                const int qq = __ffsll(bits) - 1;
                bits &= bits - 1;
                float v = pm_pd2_32(o, sq[qq]);
                bool sure = valid && v <= sLo[qq];
                bool band = valid && !sure && v <= sHi[qq];
                unsigned bs = __ballot_sync(0xffffffffu, sure);
                unsigned bb = __ballot_sync(0xffffffffu, band);
                if ((threadIdx.x & 31) == 0) {
                    if (bs) atomicAdd(&sSure[qq], __popc(bs));
                    if (bb) atomicAdd(&sBand[qq], __popc(bb));
                }
                if (band) {
                    int e2 = atomicAdd(bandN, 1);
                    if (e2 < bandCap) {
                        bandA[e2] = a0 + qq;
                        bandPos[e2] = (int)pos;
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int qq = threadIdx.x; qq < nb; qq += blockDim.x) {
        if (sSure[qq]) atomicAdd(&cntSure[a0 + qq], sSure[qq]);
        if (sBand[qq]) atomicAdd(&cntBand[a0 + qq], sBand[qq]);
    }
}

// FP64 decision for band points: ||o', q'|| <= t r exactly as the oracle.
__global__ void k_band64(const int *__restrict__ bandN, int bandCap, const int *__restrict__ bandA,
                         const int *__restrict__ bandPos, const int32_t *__restrict__ act,
                         const Thr *__restrict__ thr, const double *__restrict__ O64,
                         const double *__restrict__ qp64, int m, int *__restrict__ inTrue,
                         int *__restrict__ inN, int *__restrict__ inPos, int *__restrict__ fp64cnt,
                         int *__restrict__ errFlag)
{
    const int nbd = min(*bandN, bandCap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nbd; e += gridDim.x * blockDim.x) {
        const int a = bandA[e];
        const int64_t pos = bandPos[e];
        const int q = act[a];
        const double pd = pm_pdist64(O64 + pos * PM_MP, qp64 + (int64_t)q * PM_MP, m);
        atomicAdd(&fp64cnt[a], 1);
        if (pd <= thr[a].R) {
            atomicAdd(&inTrue[a], 1);
            const int slot = atomicAdd(&inN[a], 1);
            if (slot < BCAP) inPos[(int64_t)a * BCAP + slot] = (int)pos;
            else atomicOr(errFlag, 2);
        }
    }
}

// Zeroes up to ZL_MAX int arrays in one launch (grid-stride over each).
constexpr int ZL_MAX = 12;
struct ZeroList {
    int *p[ZL_MAX];
    int64_t n[ZL_MAX];
    int cnt = 0;
    void add(int *ptr, int64_t count)
    {
        if (ptr && count > 0 && cnt < ZL_MAX) {
            p[cnt] = ptr;
            n[cnt] = count;
            cnt++;
        }
    }
};

__global__ void k_zero(ZeroList z)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int i = 0; i < z.cnt; i++)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < z.n[i]; e += stride) z.p[i][e] = 0;
}

// --------------------------------------------------------- budget (rule 2)

// Collects (FP32 d'^2, position) of every point with d'^2 <= hi for one
// budget query.  Grid (budget query, leaf slice): a warp classifies 32
// leaves at once (leaf_class, a lane per leaf), then takes the kept ones in
// turn, its lanes testing 32 points at once (rows read together), and
// appends the selected points with one atomic on the query's counter.
__global__ void __launch_bounds__(256)
k_collect(const int32_t *__restrict__ sel, const int32_t *__restrict__ act,
          const Thr *__restrict__ thr, const float *__restrict__ qp32,
          const float *__restrict__ qpiv, int s, const float *__restrict__ meta,
          const int64_t *__restrict__ off, int64_t L, const float *__restrict__ O32,
          const int64_t *__restrict__ selOff, const int64_t *__restrict__ selCap,
          int *__restrict__ selCnt, float *__restrict__ selKey,
          int *__restrict__ selPos, int *__restrict__ errFlag)
{
    const int si = blockIdx.x;
    const int a = sel[si];
    const int q = act[a];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    float qv[PM_MP], qpv[PM_MAX_PIVOTS];
    for (int j = 0; j < PM_MP; j++) qv[j] = qp32[(int64_t)q * PM_MP + j];
    for (int i = 0; i < PM_MAX_PIVOTS; i++) qpv[i] = qpiv[(int64_t)q * PM_MAX_PIVOTS + i];
    const Thr T = thr[a];
    const float Rin = T.lo > 0.f ? __fsqrt_rn(T.lo) : -1.f, Rout = __fsqrt_rn(T.hi);
    const int64_t base = selOff[si], cap = selCap[si];
    const int64_t step = (int64_t)gridDim.y * wpb * 32;
    for (int64_t l0 = ((int64_t)blockIdx.y * wpb + (threadIdx.x >> 5)) * 32; l0 < L; l0 += step) {
        // the lanes classify 32 leaves, then the warp takes the kept ones
        const int64_t lme = l0 + lane;
        const unsigned char cme = lme < L ? leaf_class(qv, qpv, s, Rin, Rout, meta + lme * PM_LEAF_STRIDE) : CL_OUT;
        unsigned kept = __ballot_sync(0xffffffffu, cme != CL_OUT);
        while (kept) {
            const int src = __ffs(kept) - 1;
            kept &= kept - 1;
            const int64_t l = l0 + src;
            const unsigned char c = (unsigned char)__shfl_sync(0xffffffffu, (int)cme, src);
            const int64_t p0 = off[l], p1 = off[l + 1];
            for (int64_t b0 = p0; b0 < p1; b0 += 32) {
                const int64_t pos = b0 + lane;
                const bool valid = pos < p1;
                const float v = valid ? pm_pd2_32(O32 + pos * PM_MP, qv) : INFINITY;
                const bool take = valid && (c == CL_FULL || v <= T.hi);
                const unsigned m = __ballot_sync(0xffffffffu, take);
                if (m == 0u) continue;
                int e0 = 0;
                if (lane == 0) e0 = atomicAdd(&selCnt[si], __popc(m));
                e0 = __shfl_sync(0xffffffffu, e0, 0);
                if (take) {
                    const int64_t e = (int64_t)e0 + __popc(m & ((1u << lane) - 1u));
                    if (e < cap) {
                        selKey[base + e] = v;
                        selPos[base + e] = (int)pos;
                    } else {
                        atomicOr(errFlag, 64);
                    }
                }
            }
        }
    }
}

// Radix select of the B-th smallest FP32 key, then the FP64-resolved cut:
// keys < LO are surely among the B nearest, keys in [LO, HI] are ordered by
// (FP64 d', id) and the first B - |{key < LO}| of them join.  One block of
// 1024 threads per budget query.
__global__ void __launch_bounds__(1024)
k_select(const int32_t *__restrict__ sel, const int32_t *__restrict__ act, Thr *__restrict__ thr,
         const int64_t *__restrict__ selOff, const int *__restrict__ selCnt,
         const float *__restrict__ selKey, const int *__restrict__ selPos, int64_t B,
         double maxNorm, const double *__restrict__ qnorm, const double *__restrict__ O64,
         const double *__restrict__ qp64, int m, const int32_t *__restrict__ perm,
         int *__restrict__ inN, int *__restrict__ inPos, int *__restrict__ fp64cnt,
         int *__restrict__ errFlag)
{
    __shared__ unsigned int hist[2048];
    __shared__ unsigned int sPrefix, sNeed;
    __shared__ double bd[SELBAND];
    __shared__ int bpos[SELBAND];
    __shared__ int bid[SELBAND];
    __shared__ int sSure, sBand;
    __shared__ unsigned int sWarp[32];
    const int si = blockIdx.x;
    const int a = sel[si];
    const int q = act[a];
    const int64_t base = selOff[si];
    const int cnt = min(selCnt[si], (int)(selOff[si + 1] - selOff[si]));
    const unsigned int *keys = (const unsigned int *)(selKey + base);
    if (threadIdx.x == 0) { sPrefix = 0; sNeed = (unsigned int)B; }
    const int shifts[3] = {21, 10, 0};
    const int widths[3] = {11, 11, 10};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int pass = 0; pass < 3; pass++) {
        for (int i = threadIdx.x; i < 2048; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const int sh = shifts[pass];
        const unsigned int hiMask = pass == 0 ? 0u : (0xffffffffu << (sh + widths[pass]));
        const unsigned int pre = sPrefix;
        const unsigned int need = sNeed;
        // histogram: lanes with the same bin add once (keys of one query
        // share their leading bits, so bins are few and hot)
        for (int e0 = wid * 32; e0 < cnt; e0 += nwarp * 32) {
            const int e = e0 + lane;
            unsigned int bin = 0xFFFFFFFFu;
            if (e < cnt) {
                const unsigned int k = keys[e];
                if ((k & hiMask) == (pre & hiMask)) bin = (k >> sh) & ((1u << widths[pass]) - 1);
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, bin);
            if (bin != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned int)__popc(peers));
        }
        __syncthreads();
        // the bin holding the need-th key: block-wide prefix over the bins
        // (two per thread), the thread whose range holds it records it
        const int nbins = 1 << widths[pass];
        const int b0 = 2 * threadIdx.x;
        const unsigned int h0 = b0 < nbins ? hist[b0] : 0u, h1 = b0 + 1 < nbins ? hist[b0 + 1] : 0u;
        unsigned int incl = h0 + h1;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) sWarp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned int w = lane < nwarp ? sWarp[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < nwarp) sWarp[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const unsigned int ex = incl - (h0 + h1) + (wid > 0 ? sWarp[wid - 1] : 0u);
        if (b0 < nbins && ex < need && need <= ex + h0 + h1) {
            const bool first = need <= ex + h0;
            sNeed = need - ex - (first ? 0u : h0);
            sPrefix = pre | ((unsigned int)(first ? b0 : b0 + 1) << sh);
        }
        __syncthreads();
    }
    const float tau32 = __uint_as_float(sPrefix);
    const double tau = sqrt((double)tau32);
    const double eps = band_eps(tau, maxNorm, qnorm[q]);
    const float LO = tau - 2.0 * eps > 0.0 ? __double2float_rd((tau - 2.0 * eps) * (tau - 2.0 * eps)) : 0.f;
    const float HI = __double2float_ru((tau + 2.0 * eps) * (tau + 2.0 * eps));
    if (threadIdx.x == 0) { sSure = 0; sBand = 0; }
    __syncthreads();
    int mySure = 0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        float v = selKey[base + e];
        if (v < LO) mySure++;
        else if (v <= HI) {
            int slot = atomicAdd(&sBand, 1);
            if (slot < SELBAND) {
                int64_t pos = selPos[base + e];
                bd[slot] = pm_pdist64(O64 + pos * PM_MP, qp64 + (int64_t)q * PM_MP, m);
                bpos[slot] = (int)pos;
                bid[slot] = perm[pos];
            }
        }
    }
    mySure = __reduce_add_sync(0xffffffffu, mySure);
    if (lane == 0 && mySure) atomicAdd(&sSure, mySure);
    __syncthreads();
    const int nband = sBand;
    const int need = (int)B - sSure;
    if (nband > SELBAND || need < 0 || need > nband) {
        if (threadIdx.x == 0) atomicOr(errFlag, 4);
        return;
    }
    // bitonic sort of the band by (FP64 d', id)
    int P = 1;
    while (P < nband) P <<= 1;
    for (int i = nband + threadIdx.x; i < P; i += blockDim.x) { bd[i] = INFINITY; bid[i] = 0x7fffffff; bpos[i] = -1; }
    __syncthreads();
    for (int k2 = 2; k2 <= P; k2 <<= 1)
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = (i & k2) == 0;
                    bool gt = bd[i] > bd[ixj] || (bd[i] == bd[ixj] && bid[i] > bid[ixj]);
                    if (gt == up) {
                        double td = bd[i]; bd[i] = bd[ixj]; bd[ixj] = td;
                        int ti = bid[i]; bid[i] = bid[ixj]; bid[ixj] = ti;
                        int tp = bpos[i]; bpos[i] = bpos[ixj]; bpos[ixj] = tp;
                    }
                }
            }
            __syncthreads();
        }
    if (need > BCAP) {
        if (threadIdx.x == 0) atomicOr(errFlag, 8);
        return;
    }
    for (int i = threadIdx.x; i < need; i += blockDim.x) inPos[(int64_t)a * BCAP + i] = bpos[i];
    if (threadIdx.x == 0) {
        inN[a] = need;
        atomicAdd(&fp64cnt[a], nband);
        Thr T = thr[a];
        T.lov = LO > 0.f ? __uint_as_float(__float_as_uint(LO) - 1u) : -1.f;  // v <= lov  <=>  v < LO
        T.pad = 1.f;   // the band-in points of this query are listed (inPos)
        thr[a] = T;
    }
}

constexpr int VW_MAXWARPS = 8;                // queries in flight per block (one per warp)
constexpr int VW_MINBLOCKS = 4;               // blocks per SM the register budget allows
struct VwArgs {
    const int32_t *act;
    int na;
    const Thr *thr;
    const float *qp32, *qpiv;
    int s;
    const float *meta;
    int64_t L;
    const float *O32, *X, *Qd;
    int ld, d;
    const float *leafMu, *leafRx;
    const int64_t *chunkOff;
    const int32_t *leafChunk;
    const float *chunkMu, *chunkRx;
    int KP, k;
    const int *inN, *inPos;
    const int32_t *perm;
    int64_t *outIds;
    float *outD, *outErr;
    double *dk;
    int *fp64cnt, *nverOut, *nleafOut, *errFlag;
    int *workCtr;   // next entry of `order` to take (persistent warps)
    const int *order;   // [na] active queries, the costliest first
    int *dbg;       // [3]: site, value, query of the first failed index check
    int64_t n;      // points
    int2 *lists;    // [warps][L]: per-warp candidate leaves {leaf, lower bound bits}
    const uint32_t *leafBits;   // [na][W32]: leaves Eq. 5 does not exclude (k_class)
    const uint32_t *fullBits;   // [na][W32]: leaves k_class calls full (all members within the radius)
    int W32;
    const double *O64, *qp64;   // FP64 projected points and queries
    const float *leafPmu;       // [L][PM_PCA] leaf centres along the principal directions
    const float *qpca, *qnx;    // [nq][PM_PCA] queries along them, [nq] ||q|| (rounded up)
    float muMax;                // max ||mu_l|| (rounded up)
    int m;
    int inlineBand;             // 1: decide FP32 band points in FP64 here (no exact count ran)
    int nwork;                  // entries of `order` to take
    // BF16 first pass (bf16 != 0): residual rows and their rounding bounds;
    // a query whose first-pass bounds cannot settle its rerank set is
    // marked in redo[a] and verified again without the first pass
    int bf16;
    const uint16_t *Xr;
    const float *rowErr;
    int *redo;
};

constexpr int VW_WIN = 64;                    // leaves per window of the best-first walk
constexpr uint32_t VW_TAKEN = 0xFFFFFFFFu;    // list key of a leaf already windowed

// Shared memory of one warp: gd[KP] f64, gid[KP] i64, q[ld], vals[KP],
// idxs[KP], gpos[KP], q'[16], pivot distances[8], P q [PM_PCA], window keys
// and leaves [VW_WIN], select histogram [256] (BF16 first pass: u[ld],
// lows[KP]).
__host__ __device__ __forceinline__ size_t verify_smem_warp(int ld, int KP, int bf16 = 0)
{
    // BF16 first pass: also the query's residual from the current leaf centre
    // [ld] and the first-pass lower bounds of the top-KP [KP]
    return (size_t)KP * 28 + (size_t)ld * 4 + 96 + PM_PCA * 4 + VW_WIN * 8 + 256 * 4 +
           (bf16 ? (size_t)ld * 4 + (size_t)KP * 4 : 0);
}

// Total order of FP32 values as unsigned keys (finite and infinite values).
__device__ __forceinline__ uint32_t vw_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float vw_unkey(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// The want-th smallest (1-based) of the keys list[e].y != VW_TAKEN,
// e < cnt, by the warp: four 8-bit histogram passes (want must not exceed
// their number).
__device__ uint32_t warp_select(const int2 *list, int cnt, int want, uint32_t *hist, int lane)
{
    uint32_t prefix = 0, pmask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0u;
        __syncwarp();
        for (int e = lane; e < cnt; e += 32) {
            const uint32_t k = (uint32_t)list[e].y;
            if (k != VW_TAKEN && (k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncwarp();
        uint32_t h[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            h[j] = hist[lane * 8 + j];
            sum += h[j];
        }
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(VW_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned hit = __ballot_sync(VW_FULL, incl >= (uint32_t)want);
        const int fl = hit ? __ffs(hit) - 1 : 31;
        uint32_t rem = (uint32_t)want - (incl - sum);
        int j = 0;
        while (j < 7 && rem > h[j]) {
            rem -= h[j];
            j++;
        }
        const int digit = __shfl_sync(VW_FULL, lane * 8 + j, fl);
        want = (int)__shfl_sync(VW_FULL, rem, fl);
        prefix |= (uint32_t)digit << shift;
        pmask |= 0xFFu << shift;
        __syncwarp();
    }
    return prefix;
}

// Ascending bitonic sort of VW_WIN (key, value) pairs by (key, value).
__device__ __forceinline__ void warp_sort_win(uint32_t *key, int32_t *val, int lane)
{
    for (int size = 2; size <= VW_WIN; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int i = (lane / stride) * 2 * stride + lane % stride, j = i + stride;
            const uint32_t ka = key[i], kb = key[j];
            const int32_t va = val[i], vb = val[j];
            const bool gt = ka > kb || (ka == kb && va > vb);
            if (gt == ((i & size) == 0)) {
                key[i] = kb;
                key[j] = ka;
                val[i] = vb;
                val[j] = va;
            }
            __syncwarp();
        }
}

#define VW_CHECK(cond, site, val)                                              \
    (((cond)) ? true                                                           \
              : (atomicCAS(&A.dbg[0], 0, (site)) == 0 ? (A.dbg[1] = (int)(val), A.dbg[2] = a, \
                                                         atomicOr(A.errFlag, 1024), false)    \
                                                      : (atomicOr(A.errFlag, 1024), false)))

// Exact top-k of the candidate set, one warp per query (persistent warps
// take active queries from a counter).  The candidates are the points with
// FP32 d'^2 <= lov plus the FP64-resolved band-in points: listed by the
// exact count or the budget selection, or (inlineBand, when neither ran for
// the query) decided here for the points of the visited leaves with
// lov < d'^2 <= hi by the FP64 test of k_band64.  Only their k nearest
// matter (stop rule 1 tests the k-th distance).
//  1. The leaves that Eq. 5 does not exclude for radius sqrt(lov) are listed
//     with the lower bound lb = ||q - mu_l|| - Rx_l of their members'
//     distances (original-space leaf balls).
//  2. Best first: the listed leaf with the smallest lb is visited while lb
//     does not exclude it from the guard set {d^2_32 <= K (1 + 3 eps_v)},
//     K the current KP-th smallest FP32 d^2 (an upper bound of the k-th);
//     inside a leaf, chunks of <= 32 points are skipped by their own ball.
//     Each candidate's FP32 d^2 is offered to a per-warp top-KP.
//  3. Guard set: the entries of the top-KP within (1 + 3 eps_v) of its k-th
//     value provably contain the exact k nearest; they are recomputed in
//     FP64 and ranked by (FP64 distance, id).
// The result equals verifying every candidate.
template <bool WIDE, bool BF>
__global__ void __launch_bounds__(32 * VW_MAXWARPS, WIDE ? 2 : VW_MINBLOCKS)
k_verify(VwArgs A)
{
    extern __shared__ __align__(16) unsigned char vsm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int ld = A.ld, KP = A.KP, KPW = A.KP >> 5, k = A.k, s = A.s, nf4 = A.ld >> 2;
    const int64_t L = A.L;
    // BF = false compiles the first pass out (the register-rich form without
    // it has registers to spare); the 64-register form keeps one copy for
    // both modes, measured faster than its FP32-only copy (1.74 vs 1.98 ms)
    const bool bfAll = BF && A.bf16 != 0;
    unsigned char *wbase = vsm + (size_t)wib * verify_smem_warp(ld, KP, A.bf16);
    double *gd = (double *)wbase;
    long long *gid = (long long *)(gd + KP);
    float *qs = (float *)(gid + KP);
    float *vals = qs + ld;
    int *idxs = (int *)(vals + KP);
    int *gpos = idxs + KP;
    float *sq = (float *)(gpos + KP);
    float *sp = sq + PM_MP;
    float *sPq = sp + PM_MAX_PIVOTS;
    uint32_t *wkey = (uint32_t *)(sPq + PM_PCA);
    int32_t *wleaf = (int32_t *)(wkey + VW_WIN);
    uint32_t *whist = (uint32_t *)(wleaf + VW_WIN);
    float *us = (float *)(whist + 256);   // BF16 first pass: fl32(q - mu_l)
    float *lows = us + ld;                // BF16 first pass: lower bounds (squared) of the top-KP
    const float4 *q4 = (const float4 *)qs;
    int2 *list = A.lists + ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * L;
    const double epsv = (double)(ld + 8) * 0x1.0p-24;
    // the bound test in FP32 with directed rounding: lb^2 (1 - eps_v) rounded
    // down against K (1 + 3 eps_v) rounded up, so it prunes only what the
    // exact test prunes
    const float lbMulF = __double2float_rd(1.0 - epsv), cutMulF = __double2float_ru(1.0 + 3.0 * epsv);
    const float cutMulF5 = __double2float_ru(1.0 + 5.0 * epsv);
    const float lbSlack = 1.f - (float)((ld + 8) * 0x1.0p-24) - 1e-6f;
    // first pass: sqrt(S) in [sqrt(s) (1 - eps_v), sqrt(s) (1 + eps_v)] for
    // the FP32 value s of the exact sum S
    const float epsLoF = __double2float_rd(1.0 - epsv), epsHiF = __double2float_ru(1.0 + epsv);
    for (;;) {
        int a = 0;
        if (lane == 0) a = atomicAdd(A.workCtr, 1);
        a = __shfl_sync(VW_FULL, a, 0);
        if (a >= A.nwork) break;
        a = A.order[a];
        if (!VW_CHECK(a >= 0, 7, a)) break;
        const int q = A.act[a];
        const Thr T = A.thr[a];
        const float lov = T.lov;
        const float Rv = lov > 0.f ? __fsqrt_rn(lov) : -1.f;
        const bool inl = A.inlineBand != 0 && T.pad == 0.f;
        const float Rout = inl ? __fsqrt_rn(T.hi) : Rv;   // leaves beyond hold no candidate
        // with the BF16 first pass: pass 0 uses it; a query whose bounds
        // cannot settle its rerank set is verified again by pass 1 (FP32
        // rows only), by the same warp
        for (int pass = bfAll ? 0 : 1; pass < 2; pass++) {
        const bool bf = pass == 0;
        // the pruning factor: K (1 + 3 eps_v) for FP32 values; with the
        // first pass K is an upper bound of the KP-th distance^2, and
        // K (1 + 5 eps_v) keeps every point of the FP32 guard set unpruned
        const float cutF = bf ? cutMulF5 : cutMulF;
        int nfp = 0;                                       // FP64 decisions (this lane)
        for (int i = lane; i < ld; i += 32) qs[i] = A.Qd[(int64_t)q * ld + i];
        if (lane < PM_MP) sq[lane] = A.qp32[(int64_t)q * PM_MP + lane];
        if (lane < PM_MAX_PIVOTS) sp[lane] = A.qpiv[(int64_t)q * PM_MAX_PIVOTS + lane];
        if (lane < PM_PCA) sPq[lane] = A.qpca[(int64_t)q * PM_PCA + lane];
        for (int e = lane; e < KP; e += 32) {
            vals[e] = INFINITY;
            idxs[e] = 0x7fffffff;
        }
        __syncwarp();
        auto D2 = [&](const float *p) -> float {
            return WIDE ? warp_d2x4w(q4, p, nf4, lane) : warp_d2x4(q4, p, nf4, lane);
        };
        // top-KP state: lane owns slots lane, lane + 32, ...; cmax is the
        // largest entry (the KP-th smallest so far), cslot its slot
        float cmax = INFINITY, myMax = INFINITY;
        int cslot = 0, mySlot = lane;
        int seen = 0, leaves = 0;
        auto pruned = [&](float lb) -> bool {
            return lb > 0.f && __fmul_rd(__fmul_rd(lb, lb), lbMulF) > __fmul_ru(cmax, cutF);
        };
        int fill = 0;   // slots of the top-KP taken so far (its maximum is +inf until all are)
        // BF16 first pass: the smallest lower bound (squared) of a candidate
        // left out of the top-KP (this lane's share)
        float dropLo = INFINITY;
        // offers the lanes' values (cand) to the top-KP, in lane order; lo:
        // the first pass's lower bound (squared), kept beside the value
        auto offer = [&](bool cand, float v, float lo, int pos) {
            if (fill < KP) {
                // empty slots first: appended in lane order, no maximum to keep
                const unsigned all = __ballot_sync(VW_FULL, cand);
                const int rank = __popc(all & ((1u << lane) - 1u));
                const int take = min(__popc(all), KP - fill);
                if (cand && rank < take) {
                    vals[fill + rank] = v;
                    idxs[fill + rank] = pos;
                    if (bf) lows[fill + rank] = lo;
                }
                fill += take;
                cand = cand && rank >= take;
                if (fill == KP) {
                    __syncwarp();
                    float mm = -1.f;
                    int ms = lane;
                    for (int j = 0; j < KPW; j++) {
                        const float x = vals[lane + 32 * j];
                        if (x > mm) { mm = x; ms = lane + 32 * j; }
                    }
                    myMax = mm;
                    mySlot = ms;
                    const unsigned mb = __reduce_max_sync(VW_FULL, __float_as_uint(myMax));
                    const unsigned who = __ballot_sync(VW_FULL, __float_as_uint(myMax) == mb);
                    cmax = __uint_as_float(mb);
                    cslot = __shfl_sync(VW_FULL, mySlot, __ffs(who) - 1);
                }
            }
            if (bf && cand && !(v < cmax)) dropLo = fminf(dropLo, lo);
            unsigned bits = __ballot_sync(VW_FULL, cand && v < cmax);
            while (bits) {
                const int src = __ffs(bits) - 1;
                bits &= bits - 1;
                const float val = __shfl_sync(VW_FULL, v, src);
                const int ps = __shfl_sync(VW_FULL, pos, src);
                const float lv = bf ? __shfl_sync(VW_FULL, lo, src) : 0.f;
                if (!(val < cmax)) {
                    if (bf && lane == src) dropLo = fminf(dropLo, lo);
                    continue;
                }
                if (lane == (cslot & 31)) {
                    if (bf) {
                        dropLo = fminf(dropLo, lows[cslot]);
                        lows[cslot] = lv;
                    }
                    vals[cslot] = val;
                    idxs[cslot] = ps;
                    float mm = -1.f;
                    int ms = lane;
                    for (int j = 0; j < KPW; j++) {
                        const float x = vals[lane + 32 * j];
                        if (x > mm) { mm = x; ms = lane + 32 * j; }
                    }
                    myMax = mm;
                    mySlot = ms;
                }
                // values are >= +0 or +inf: their bit patterns order like them
                const unsigned mb = __reduce_max_sync(VW_FULL, __float_as_uint(myMax));
                const unsigned who = __ballot_sync(VW_FULL, __float_as_uint(myMax) == mb);
                cmax = __uint_as_float(mb);
                cslot = __shfl_sync(VW_FULL, mySlot, __ffs(who) - 1);
            }
        };
        // FP32 pass: candidate rows wait in a warp queue (the histogram
        // space, unused while leaves are visited) and their distances are
        // taken 32 at a time, so a chunk with few candidates does not cost a
        // whole 32-row distance pass; the K that prunes meanwhile is that of
        // the rows already offered, never below the exact one
        int *cq = (int *)whist;
        int qn = 0;
        auto flushq = [&](int nq) {
            const bool c = lane < nq;
            const int pos = c ? cq[lane] : 0;
            const int rest = qn - nq;
            const int mv = lane < rest ? cq[nq + lane] : 0;
            __syncwarp();
            if (lane < rest) cq[lane] = mv;
            qn = rest;
            __syncwarp();
            const float d2 = D2(c ? A.X + (int64_t)pos * ld : nullptr);
            offer(c, d2, d2, pos);
        };
        // verifies the candidates of leaf l
        // (lbl: the leaf's full lower bound, ||q - mu_l|| lbSlack - Rx_l)
        auto visit = [&](int l, float lbl) {
            leaves++;
            // k_class's decision for this round's radius (its full test is
            // sound for lov = its lower threshold); a query whose radius the
            // budget selection moved (T.pad) takes the test again
            const unsigned char cl = T.pad == 0.f
                ? (((A.fullBits[(int64_t)a * A.W32 + (l >> 5)] >> (l & 31)) & 1u) ? CL_FULL : CL_PART)
                : leaf_class(sq, sp, s, Rv, Rout, A.meta + (int64_t)l * PM_LEAF_STRIDE);
            const int cb = A.leafChunk[l], ce = A.leafChunk[l + 1];
            // chunk bounds only if one can prune: every member lies within
            // ub = ||q - mu_l|| + Rx_l of q (rounded up generously from lbl),
            // and a chunk's bound never exceeds its nearest member's distance,
            // so ub^2 <= K leaves every chunk alive
            const float rxl = A.leafRx[l];
            const float ubl = __fadd_ru(__fmul_ru(__fadd_ru(fmaxf(lbl, 0.f), rxl), 1.0001f), rxl);
            const bool chunkBounds = __fmul_ru(ubl, ubl) > cmax;
            // BF16 first pass: u = fl32(q - mu_l) and a bound wErr on
            // ||u - (q - mu_l)|| (each coordinate within 2^-24 of its value)
            float wErr = 0.f;
            if (bf) {
                const float *mu = A.leafMu + (int64_t)l * ld;
                float un = 0.f;
                for (int i = lane; i < ld; i += 32) {
                    const float uu = __fsub_rn(qs[i], mu[i]);
                    us[i] = uu;
                    un = __fmaf_ru(uu, uu, un);
                }
                for (int o = 16; o; o >>= 1) un = __fadd_ru(un, __shfl_xor_sync(VW_FULL, un, o));
                wErr = __fmul_ru(0x1.0p-23f, __fsqrt_ru(__fmul_ru(un, 1.0001f)));
                __syncwarp();
            }
            for (int c0 = cb; c0 < ce; c0 += 32) {
                const int c = c0 + lane;
                const bool vc = c < ce;
                float lbc = -INFINITY;
                if (chunkBounds) {
                    const float d2c = D2(vc ? A.chunkMu + (int64_t)c * ld : nullptr);
                    lbc = vc ? __fsub_rn(__fmul_rn(__fsqrt_rn(d2c), lbSlack), A.chunkRx[c]) : INFINITY;
                }
                // the chunks' row ranges, one chunk per lane
                const long long cOff = vc ? A.chunkOff[c] : 0, cEnd = vc ? A.chunkOff[c + 1] : 0;
                unsigned alive = __ballot_sync(VW_FULL, vc && !pruned(lbc));
                while (alive) {
                    const int src = __ffs(alive) - 1;
                    alive &= alive - 1;
                    if (pruned(__shfl_sync(VW_FULL, lbc, src))) continue;   // K fell since
                    const int64_t r0 = __shfl_sync(VW_FULL, cOff, src);
                    int rows = (int)(__shfl_sync(VW_FULL, cEnd, src) - r0);
                    if (!VW_CHECK(rows >= 1 && rows <= 32 && r0 >= 0 && r0 + rows <= A.n, 2, rows)) rows = 0;
                    bool cand = false;
                    if (lane < rows) {
                        if (cl == CL_FULL) {
                            cand = true;
                        } else {
                            const float pd = pd2_row(A.O32 + (r0 + lane) * PM_MP, sq);
                            cand = pd <= lov;
                            if (!cand && inl && pd <= T.hi) {
                                // inside the FP32 error band: k_band64's FP64 test
                                cand = pm_pdist64(A.O64 + (r0 + lane) * PM_MP, A.qp64 + (int64_t)q * PM_MP, A.m) <= T.R;
                                nfp++;
                            }
                        }
                    }
                    if (__ballot_sync(VW_FULL, cand) == 0u) continue;
                    seen += __popc(__ballot_sync(VW_FULL, cand));
                    if (!bf) {
                        const unsigned cm = __ballot_sync(VW_FULL, cand);
                        if (cand) cq[qn + __popc(cm & ((1u << lane) - 1u))] = (int)(r0 + lane);
                        qn += __popc(cm);
                        __syncwarp();
                        if (qn >= 32) flushq(32);
                    } else {
                        // first pass: ||q - x|| within sqrt(S) +- (wErr + e_row), S the
                        // exact ||u - r~||^2; offered by the upper bound (squared)
                        const float s2 = warp_d2_bf16x4(us, cand ? A.Xr + (r0 + lane) * ld : nullptr, ld, lane);
                        float hi2 = INFINITY, lo2 = INFINITY;
                        if (cand) {
                            const float ae = __fadd_ru(A.rowErr[r0 + lane], wErr);
                            const float lo = fmaxf(0.f, __fsub_rd(__fmul_rd(__fsqrt_rd(s2), epsLoF), ae));
                            const float hi = __fadd_ru(__fmul_ru(__fsqrt_ru(s2), epsHiF), ae);
                            lo2 = __fmul_rd(lo, lo);
                            hi2 = __fmul_ru(hi, hi);
                        }
                        offer(cand, hi2, lo2, (int)(r0 + lane));
                    }
                }
            }
        };

        // 1. candidate leaves (k_class's bit set for this round's radius,
        // a superset of the leaves Eq. 5 keeps for sqrt(lov) <= its radius)
        // and their lower bounds
        int cnt = 0;
        if (Rv > 0.f || inl) {
            const uint32_t *bits = A.leafBits + (int64_t)a * A.W32;
            for (int w0 = 0; w0 < A.W32; w0 += 32) {
                const int wi = w0 + lane;
                uint32_t word = wi < A.W32 ? bits[wi] : 0u;
                const int c = __popc(word);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(VW_FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                int at = cnt + incl - c;
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1u;
                    const int64_t l = (int64_t)wi * 32 + b;
                    if (l < L) list[at++] = make_int2((int)l, 0);
                }
                cnt += __shfl_sync(VW_FULL, incl, 31);
            }
        }
        __syncwarp();
        // cheap bounds first: ||P q - P mu|| <= ||q - mu|| for the
        // orthonormal rows P (the FP32 errors of P q, P mu and the sum covered
        // by the slack); an entry is {leaf, ordered key of its bound}
        // slack: FP32 P q ((ld + 2) 2^-24 ||q|| per coordinate, 4 x over 16),
        // FP32 P mu and the FP32 difference and sum, rounded generously up
        const float pSlack = __fmul_ru(1.01f, __fadd_ru(__fmul_ru((float)(4 * (ld + 2)) * 0x1.0p-24f, A.qnx[q]),
                                                        __fmul_ru(0x1.0p-20f, __fadd_ru(A.qnx[q], A.muMax))));
        // two batches of 32 entries per step: their leaf records are loaded
        // together (a dependent list -> record chain per step, not per batch)
        for (int e0 = 0; e0 < cnt; e0 += 64) {
            const int ea = e0 + lane, eb = e0 + 32 + lane;
            const int la = ea < cnt ? list[ea].x : 0, lb = eb < cnt ? list[eb].x : 0;
            const float4 *pa = (const float4 *)(A.leafPmu + (int64_t)la * PM_PCA);
            const float4 *pb = (const float4 *)(A.leafPmu + (int64_t)lb * PM_PCA);
            float4 va[PM_PCA / 4], vb[PM_PCA / 4];
#pragma unroll
            for (int r4 = 0; r4 < PM_PCA / 4; r4++) {
                va[r4] = __ldg(pa + r4);
                vb[r4] = __ldg(pb + r4);
            }
            const float rxa = A.leafRx[la], rxb = A.leafRx[lb];
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int r4 = 0; r4 < PM_PCA / 4; r4++) {
                float u = __fsub_rn(sPq[4 * r4], va[r4].x);
                sa = __fmaf_rn(u, u, sa);
                u = __fsub_rn(sPq[4 * r4 + 1], va[r4].y);
                sa = __fmaf_rn(u, u, sa);
                u = __fsub_rn(sPq[4 * r4 + 2], va[r4].z);
                sa = __fmaf_rn(u, u, sa);
                u = __fsub_rn(sPq[4 * r4 + 3], va[r4].w);
                sa = __fmaf_rn(u, u, sa);
                u = __fsub_rn(sPq[4 * r4], vb[r4].x);
                sb = __fmaf_rn(u, u, sb);
                u = __fsub_rn(sPq[4 * r4 + 1], vb[r4].y);
                sb = __fmaf_rn(u, u, sb);
                u = __fsub_rn(sPq[4 * r4 + 2], vb[r4].z);
                sb = __fmaf_rn(u, u, sb);
                u = __fsub_rn(sPq[4 * r4 + 3], vb[r4].w);
                sb = __fmaf_rn(u, u, sb);
            }
            if (ea < cnt) {
                const float lbp = __fsub_rn(__fsub_rn(__fmul_rn(__fsqrt_rn(sa), 1.f - 0x1.0p-18f), pSlack), rxa);
                list[ea] = make_int2(la, (int)vw_key(lbp));
            }
            if (eb < cnt) {
                const float lbp = __fsub_rn(__fsub_rn(__fmul_rn(__fsqrt_rn(sb), 1.f - 0x1.0p-18f), pSlack), rxb);
                list[eb] = make_int2(lb, (int)vw_key(lbp));
            }
        }
        __syncwarp();
        // 2. best first, in windows: the VW_WIN listed leaves with the
        // smallest cheap bounds (warp radix select) get their full bound
        // (original-space leaf ball) and are visited in ascending full bound
        // until one is pruned; the next window follows while the cheap bound
        // at the window's edge is not pruned (every leaf left has a cheap
        // bound, and so a full bound, at least that large)
        int remaining = cnt;
        while (remaining > 0) {
            const uint32_t tau = warp_select(list, cnt, min(VW_WIN, remaining), whist, lane);
            int nw = 0;
            for (int pass = 0; pass < 2; pass++)
                for (int e0 = 0; e0 < cnt; e0 += 32) {
                    const int e = e0 + lane;
                    const int2 v = e < cnt ? list[e] : make_int2(0, (int)VW_TAKEN);
                    const uint32_t k = (uint32_t)v.y;
                    const bool take = k != VW_TAKEN && (pass == 0 ? k < tau : k == tau);
                    const unsigned m = __ballot_sync(VW_FULL, take);
                    const int at = nw + __popc(m & ((1u << lane) - 1u));
                    if (take && at < VW_WIN) {
                        wkey[at] = k;
                        wleaf[at] = v.x;
                        list[e].y = (int)VW_TAKEN;
                    }
                    nw = min(VW_WIN, nw + __popc(m));
                }
            __syncwarp();
            if (nw == 0) break;
            remaining -= nw;
            // full bounds, 32 leaves per pass
            for (int i0 = 0; i0 < nw; i0 += 32) {
                const int i = i0 + lane;
                bool need = i < nw && !pruned(vw_unkey(wkey[i]));
                int lr = need ? wleaf[i] : -1;
                if (need && !(lr >= 0 && lr < L)) {
                    VW_CHECK(false, 10, lr);
                    need = false;
                    lr = -1;
                }
                const float d2 = D2(need ? A.leafMu + (int64_t)lr * ld : nullptr);
                if (i < nw)
                    wkey[i] = need ? vw_key(__fsub_rn(__fmul_rn(__fsqrt_rn(d2), lbSlack), A.leafRx[lr])) : VW_TAKEN;
            }
            for (int i = nw + lane; i < VW_WIN; i += 32) {
                wkey[i] = VW_TAKEN;
                wleaf[i] = -1;
            }
            __syncwarp();
            warp_sort_win(wkey, wleaf, lane);
            for (int i = 0; i < nw; i++) {
                const uint32_t kk = wkey[i];
                if (kk == VW_TAKEN || pruned(vw_unkey(kk))) break;
                const int x = wleaf[i];
                if (!VW_CHECK(x >= 0 && x < L, 1, x)) break;
                visit(x, vw_unkey(kk));
            }
            __syncwarp();
            if (qn > 0) flushq(qn);
            if (pruned(vw_unkey(tau))) break;
        }
        // band-in points (FP64-resolved members just inside the radius)
        const int nIn = min(A.inN[a], BCAP);
        for (int e0 = 0; e0 < nIn; e0 += 32) {
            const int e = e0 + lane;
            int pos = e < nIn ? A.inPos[(int64_t)a * BCAP + e] : -1;
            if (e < nIn && !VW_CHECK(pos >= 0 && pos < A.n, 4, pos)) pos = -1;
            const bool cand = pos >= 0;
            const float d2 = D2(cand ? A.X + (int64_t)pos * ld : nullptr);
            seen += __popc(__ballot_sync(VW_FULL, cand));
            if (!bf) offer(cand, d2, d2, pos);
            else offer(cand, __fmul_ru(d2, epsHiF), __fmul_rd(d2, epsLoF), pos);
        }
        __syncwarp();
        // the kk-th smallest value of the top-KP, +inf if fewer are finite
        // (radix select on the value bits: values are >= +0 or +inf)
        auto kth_value = [&](int kk) -> float {
            int nf = 0;
            for (int j = 0; j < KPW; j++) nf += vals[lane + 32 * j] < INFINITY ? 1 : 0;
            nf = __reduce_add_sync(VW_FULL, nf);
            if (nf < kk) return INFINITY;
            uint32_t prefix = 0, pmask = 0;
            int want = kk;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int i = lane; i < 256; i += 32) whist[i] = 0u;
                __syncwarp();
                for (int j = 0; j < KPW; j++) {
                    const uint32_t kb = __float_as_uint(vals[lane + 32 * j]);
                    if ((kb & pmask) == prefix) atomicAdd(&whist[(kb >> shift) & 255u], 1u);
                }
                __syncwarp();
                uint32_t h[8], sum = 0;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    h[j] = whist[lane * 8 + j];
                    sum += h[j];
                }
                uint32_t incl = sum;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(VW_FULL, incl, o);
                    if (lane >= o) incl += t;
                }
                const unsigned hit = __ballot_sync(VW_FULL, incl >= (uint32_t)want);
                const int fl = hit ? __ffs(hit) - 1 : 31;
                uint32_t rem = (uint32_t)want - (incl - sum);
                int j = 0;
                while (j < 7 && rem > h[j]) {
                    rem -= h[j];
                    j++;
                }
                const int digit = __shfl_sync(VW_FULL, lane * 8 + j, fl);
                want = (int)__shfl_sync(VW_FULL, rem, fl);
                prefix |= (uint32_t)digit << shift;
                pmask |= 0xFFu << shift;
                __syncwarp();
            }
            return __uint_as_float(prefix);
        };
        if (bf) {
            // BF16 first pass -> FP32 rerank.  H = the k-th smallest upper
            // bound; a candidate whose lower bound exceeds H (1 + 6 eps_v)
            // is farther than the k-th nearest by more than the FP32 guard
            // band (FP32 values within (1 + eps_v) of exact, guard factor
            // (1 + 3 eps_v)), so the rest is the rerank set; it must hold
            // every candidate that qualifies, including those the top-KP
            // left out (their smallest lower bound is dropLo)
            const float H = kth_value(k);
            const float rthr = H < INFINITY ? __fmul_ru(H, __double2float_ru(1.0 + 6.0 * epsv)) : INFINITY;
            // (lower bounds are >= +0 or +inf: their bits order like them)
            dropLo = __uint_as_float(__reduce_min_sync(VW_FULL, __float_as_uint(dropLo)));
            if (!(dropLo > rthr) && H < INFINITY) {
                if (lane == 0) A.redo[a] = 1;
                continue;   // pass 1: FP32 rows only
            }
            int nR = 0;
            for (int j = 0; j < KPW; j++) {
                const int e = lane + 32 * j;
                const bool in = vals[e] < INFINITY && lows[e] <= rthr;
                const unsigned m = __ballot_sync(VW_FULL, in);
                if (in) gpos[nR + __popc(m & ((1u << lane) - 1u))] = idxs[e];
                nR += __popc(m);
            }
            __syncwarp();
            // exact FP32 values of the rerank set replace the top-KP
            for (int e0 = 0; e0 < KP; e0 += 32) {
                const int e = e0 + lane;
                const int p = e < nR ? gpos[e] : -1;
                const bool ok = p >= 0 && p < A.n;
                const float d2 = D2(ok ? A.X + (int64_t)p * ld : nullptr);
                vals[e] = ok ? d2 : INFINITY;
                idxs[e] = ok ? p : 0x7fffffff;
            }
            __syncwarp();
        }
        // 3. guard set: the k-th smallest value of the top-KP
        const float K32 = kth_value(k);
        const float thrv = K32 < INFINITY ? (float)((double)K32 * (1.0 + 3.0 * epsv) + 1e-36) : INFINITY;
        // entries dropped from the top-KP are >= its final maximum
        if (!bf && lane == 0 && seen > KP && cmax <= thrv) atomicOr(A.errFlag, 16);
        int G = 0;
        for (int j = 0; j < KPW; j++) {
            const int e = lane + 32 * j;
            const float v = vals[e];
            const bool in = v <= thrv && v < INFINITY;
            const unsigned m = __ballot_sync(VW_FULL, in);
            if (in) gpos[G + __popc(m & ((1u << lane) - 1u))] = idxs[e];
            G += __popc(m);
        }
        __syncwarp();
        // two rows per lane at a time: two independent chains of the
        // sequential FP64 sum (each row's own order is unchanged)
        for (int e = lane; e < G; e += 64) {
            const int e2 = e + 32;
            int p = gpos[e], p2 = e2 < G ? gpos[e2] : -1;
            if (!VW_CHECK(p >= 0 && p < A.n, 5, p)) p = -1;
            if (e2 < G && !VW_CHECK(p2 >= 0 && p2 < A.n, 5, p2)) p2 = -1;
            double s1 = 0.0, s2 = 0.0;
            const float *x1 = A.X + (int64_t)max(p, 0) * ld, *x2 = A.X + (int64_t)max(p2, 0) * ld;
            // the same sequential sum over i = 0 .. d - 1, four coordinates per
            // 16-byte load in the register-rich form (rows and the query are
            // 16-byte aligned, zero-padded to ld; the tail past d is not summed)
            const bool two = p2 >= 0;
            int i = 0;
            // (the 64-register form keeps scalar loads: its register budget
            // is better spent elsewhere)
            for (; WIDE && i + 4 <= A.d; i += 4) {
                const float4 qv = *(const float4 *)(qs + i);
                const float4 a1 = __ldg((const float4 *)(x1 + i));
                const float4 a2 = two ? __ldg((const float4 *)(x2 + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const double q0 = f2d_exact(qv.x), q1 = f2d_exact(qv.y), q2 = f2d_exact(qv.z), q3 = f2d_exact(qv.w);
                double t = __dsub_rn(f2d_exact(a1.x), q0);
                s1 = __dadd_rn(s1, __dmul_rn(t, t));
                t = __dsub_rn(f2d_exact(a1.y), q1);
                s1 = __dadd_rn(s1, __dmul_rn(t, t));
                t = __dsub_rn(f2d_exact(a1.z), q2);
                s1 = __dadd_rn(s1, __dmul_rn(t, t));
                t = __dsub_rn(f2d_exact(a1.w), q3);
                s1 = __dadd_rn(s1, __dmul_rn(t, t));
                if (two) {
                    t = __dsub_rn(f2d_exact(a2.x), q0);
                    s2 = __dadd_rn(s2, __dmul_rn(t, t));
                    t = __dsub_rn(f2d_exact(a2.y), q1);
                    s2 = __dadd_rn(s2, __dmul_rn(t, t));
                    t = __dsub_rn(f2d_exact(a2.z), q2);
                    s2 = __dadd_rn(s2, __dmul_rn(t, t));
                    t = __dsub_rn(f2d_exact(a2.w), q3);
                    s2 = __dadd_rn(s2, __dmul_rn(t, t));
                }
            }
            for (; i < A.d; i++) {
                const double qd = f2d_exact(qs[i]);
                const double t1 = __dsub_rn(f2d_exact(x1[i]), qd);
                s1 = __dadd_rn(s1, __dmul_rn(t1, t1));
                if (two) {
                    const double t2 = __dsub_rn(f2d_exact(x2[i]), qd);
                    s2 = __dadd_rn(s2, __dmul_rn(t2, t2));
                }
            }
            gd[e] = p >= 0 ? __dsqrt_rn(s1) : (double)INFINITY;
            gid[e] = p >= 0 ? (long long)A.perm[p] : 0x7fffffffffffffffLL;
            if (e2 < G) {
                gd[e2] = p2 >= 0 ? __dsqrt_rn(s2) : (double)INFINITY;
                gid[e2] = p2 >= 0 ? (long long)A.perm[p2] : 0x7fffffffffffffffLL;
            }
        }
        __syncwarp();
        // rank by (FP64 distance, id); the k nearest are written in order
        for (int e = lane; e < G; e += 32) {
            const double dv = gd[e];
            const long long iv = gid[e];
            // non-negative doubles and +inf order like their bit patterns
            const long long db = __double_as_longlong(dv);
            int rank = 0;
            for (int f = 0; f < G; f++) {
                const long long fb = __double_as_longlong(gd[f]);
                rank += (fb < db || (fb == db && gid[f] < iv)) ? 1 : 0;
            }
            if (rank < k) {
                const int64_t o = (int64_t)q * k + rank;
                const float fv = __double2float_rn(dv);
                A.outIds[o] = iv;
                A.outD[o] = fv;
                A.outErr[o] = (float)fabs((double)fv - dv);
            }
            if (rank == k - 1) A.dk[a] = dv;
        }
        for (int e = G + lane; e < k; e += 32) {
            const int64_t o = (int64_t)q * k + e;
            A.outIds[o] = -1;
            A.outD[o] = INFINITY;
            A.outErr[o] = 0.f;
        }
        for (int o = 16; o; o >>= 1) nfp += __shfl_xor_sync(VW_FULL, nfp, o);
        if (lane == 0) {
            if (G < k) A.dk[a] = INFINITY;
            atomicAdd(&A.fp64cnt[a], G + nfp);
            A.nverOut[a] = seen;
            A.nleafOut[a] = leaves;
        }
        __syncwarp();
        break;
        }
    }
}

// ---------------------------------------- tensor-core range count (tcgen05)

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major: start address,
// leading byte offset (between core matrices adjacent in K), stride byte
// offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 16 consecutive FP32 accumulator columns of this warp's lane quarter.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

constexpr int TC_QN = 256;         // queries per block
constexpr int TC_MT = 128;         // compacted queries per MMA (M, TMEM lanes)
constexpr int TC_NT = 128;         // points per job at most (N)
constexpr int TC_K = 48;           // [hi | lo | hi] . [hi | hi | lo] of 16 coordinates
constexpr int TC_ROWB = TC_K * 2;  // bytes per operand row
constexpr int TC_SO = 4;           // operand stages (released when the MMA completes)
constexpr int TC_SJ = 8;           // job slots: norms, rank -> query map (released by the epilogue)
constexpr int TC_EPI = 16;         // epilogue warps: 2 TMEM buffers x 2 M-tiles x 4 lane quarters
constexpr int TC_THREADS = 32 * (2 + 4 + TC_EPI);   // loader, MMA, 4 builder warps, epilogue
constexpr int TC_MW = TC_QN / 32;  // mask words per list entry
constexpr int TC_MAYBE = 224;      // pairs inside the error band staged per epilogue warp
// dynamic shared memory
constexpr int TC_ASZ = 2 * TC_MT * TC_ROWB;                    // two M-tiles per stage, 24 KB
constexpr int TC_BSZ = TC_NT * TC_ROWB;                        // 12 KB
constexpr int TC_JSZ = TC_NT * 4 + TC_QN * 4;                  // norms + map, 1.5 KB
constexpr int TC_OFF_B = TC_SO * TC_ASZ;
constexpr int TC_OFF_J = TC_OFF_B + TC_SO * TC_BSZ;
constexpr int TC_OFF_QR = TC_OFF_J + TC_SJ * TC_JSZ;           // query rows [256][96 B]
constexpr int TC_OFF_PAR = TC_OFF_QR + TC_QN * TC_ROWB;
constexpr int TC_OFF_MAY = TC_OFF_PAR + TC_QN * 16;
constexpr int TC_OFF_CNT = TC_OFF_MAY + TC_EPI * TC_MAYBE * 8;
constexpr int TC_SMEM = TC_OFF_CNT + TC_QN * 4;
static_assert(TC_SMEM <= 222 * 1024, "tensor-count shared memory");

// The CUDA-core count's decision for one pair: 1 surely in (<= lo), 2 in
// the band (<= hi), 0 out.
__device__ __forceinline__ int exact_class(const float *o, const float *q, float lo, float hi)
{
    const float ex = pm_pd2_32(o, q);
    return ex <= lo ? 1 : (ex <= hi ? 2 : 0);
}

// Appends this warp's staged pairs to the global recheck list (one atomic
// per warp) and empties the stage.
__device__ __forceinline__ void may_flush(int2 *stage, int &n, int lane, int *recheckN, int recheckCap,
                                          int2 *recheck)
{
    int base = 0;
    if (lane == 0 && n) base = atomicAdd(recheckN, n);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int m = lane; m < n; m += 32)
        if (base + m < recheckCap) recheck[base + m] = stage[m];
    __syncwarp();
    n = 0;
}

// OR of `p` over the 128 threads of named barrier 1 (the operand builders).
__device__ __forceinline__ bool bar1_or_128(bool p)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

// Waits for phase `ph` of `bar`, giving up on the iteration limit or when
// another role has already failed (fail != 0).
__device__ __forceinline__ bool mbar_wait_or_fail(uint64_t *bar, uint32_t ph, volatile int *fail)
{
    for (int it = 0; it < (1 << 22); it++) {
        if (mbar_try_wait(bar, ph)) return true;
        if ((it & 255) == 255 && *fail) return false;
    }
    return false;
}

// Range count of one round on the tensor cores.  A job is a listed leaf (or
// its next 128 points) of a block of up to 256 queries: the queries that
// cover the leaf partially are compacted into one or two 128-row operands,
// and TMEM receives their dot products q'.o' with the leaf's points (BF16
// split of the FP32 coordinates, three products, FP32 accumulate).  A lane
// of the epilogue is a query: with E bounding |d'^2~ - pm_pd2_32| for d'^2~ =
// ||o'||^2 + ||q'||^2 - 2 q'.o' (split and accumulation error, FP32 rounding
// of the norms, the CUDA-core computation's own error), d'^2~ <= lo - E is
// surely in and > hi + E surely out; the pairs in between go to a recheck
// list that k_recheck decides exactly as k_count does.  Counts and band
// lists therefore equal k_count's.
//
// Roles: warp 0 streams point tiles (operand ring) and their norms (job
// ring) with TMA bulk copies, warps 2-5 build the compacted query operand
// and the job's rank -> query map, warp 1 issues tcgen05.mma into one of two
// TMEM buffers (even / odd jobs) and releases the operand stages on
// completion, 16 epilogue warps (buffer x M-tile x lane quarter) read TMEM
// and release the buffer and the job slot.  Every wait is bounded; on a
// timeout the CTA records error bit 128, waits (bounded) for the copies and
// MMAs it issued and frees its TMEM.
__global__ void __launch_bounds__(TC_THREADS, 1)
k_count_tc(const int32_t *__restrict__ act, int na, const Thr *__restrict__ thr,
           const float *__restrict__ qp32, const uint16_t *__restrict__ Bsplit, const float *__restrict__ bNorm,
           const int *__restrict__ blkCnt, const int4 *__restrict__ blkEnt, const uint32_t *__restrict__ blkMask,
           int64_t L, double maxNorm, int *__restrict__ cntSure, int *__restrict__ recheckN, int recheckCap,
           int2 *__restrict__ recheck, int *__restrict__ errFlag)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char *sA = tsm;
    unsigned char *sB = tsm + TC_OFF_B;
    unsigned char *sJ = tsm + TC_OFF_J;
    unsigned char *sQr = tsm + TC_OFF_QR;
    float4 *sPar = (float4 *)(tsm + TC_OFF_PAR);   // ||q'||^2, lo - E, hi + E
    int2 *sMay = (int2 *)(tsm + TC_OFF_MAY);
    int *sCntS = (int *)(tsm + TC_OFF_CNT);
    __shared__ __align__(8) uint64_t barBFull[TC_SO], barBEmpty[TC_SO], barAFull[TC_SO], barAEmpty[TC_SO];
    __shared__ __align__(8) uint64_t barJFull[TC_SJ], barJEmpty[TC_SJ], barTFull[2], barTEmpty[2];
    __shared__ uint32_t sTmem;
    __shared__ int sFail;
    __shared__ int sNpart[TC_SJ];
    __shared__ int sIssB[TC_SO], sSeenB[TC_SO], sIssJ[TC_SJ], sSeenJ[TC_SJ], sCommitted[2], sSeenT[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, S = gridDim.y, sidx = blockIdx.y;
    const int a0 = b * TC_QN;
    const int nb = min(TC_QN, na - a0);
    volatile int *vFail = &sFail;

    // query rows [hi | lo | hi], per-query thresholds and error bound
    if (tid < TC_QN) {
        const int j = tid;
        float qv[PM_MP];
        float4 par = make_float4(0.f, -INFINITY, -INFINITY, 0.f);
        if (j < nb) {
            const int q = act[a0 + j];
            double nn = 0.0;
            for (int c = 0; c < PM_MP; c++) {
                qv[c] = qp32[(int64_t)q * PM_MP + c];
                nn += (double)qv[c] * (double)qv[c];
            }
            const Thr T = thr[a0 + j];
            const double qn = sqrt(nn);
            // split: lo*lo and both rounding residues dropped, each <= 2^-16
            // |q_c| |o_c|, so <= 3 * 2^-16 ||q'|| ||o'|| (Cauchy-Schwarz); the
            // FP32 accumulation of 48 exact products <= 128 * 2^-23 of the
            // same, whatever the adder's alignment; norms, their sum and the
            // final fma rounded to FP32; pm_pd2_32 within 18 * 2^-24 relative.
            // Everything is taken 1.25 times.
            const double E = 1.25 * (2.0 * (3.0 * 0x1.0p-16 + 128.0 * 0x1.0p-23) * qn * maxNorm +
                                     0x1.0p-22 * (nn + maxNorm * maxNorm) + 0x1.0p-18 * (double)T.hi) + 1e-30;
            par = make_float4((float)nn, (float)((double)T.lo - E), (float)((double)T.hi + E), 0.f);
        } else {
            for (int c = 0; c < PM_MP; c++) qv[c] = 0.f;
        }
        sPar[j] = par;
        sCntS[j] = 0;
        uint16_t *row = (uint16_t *)(sQr + j * TC_ROWB);
        for (int c = 0; c < PM_MP; c++) {
            const __nv_bfloat16 h = __float2bfloat16_rn(qv[c]);
            const __nv_bfloat16 l = __float2bfloat16_rn(qv[c] - __bfloat162float(h));
            row[c] = __bfloat16_as_ushort(h);
            row[16 + c] = __bfloat16_as_ushort(l);
            row[32 + c] = __bfloat16_as_ushort(h);
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        sFail = 0;
        for (int st = 0; st < TC_SO; st++) {
            mbar_init(&barBFull[st], 1);
            mbar_init(&barBEmpty[st], 1);
            mbar_init(&barAFull[st], 1);
            mbar_init(&barAEmpty[st], 1);
            sIssB[st] = 0;
            sSeenB[st] = 0;
        }
        for (int s = 0; s < TC_SJ; s++) {
            mbar_init(&barJFull[s], 2);   // loader (norms, with tx) + builders (map)
            mbar_init(&barJEmpty[s], TC_EPI / 2);
            sIssJ[s] = 0;
            sSeenJ[s] = 0;
        }
        for (int t = 0; t < 2; t++) {
            mbar_init(&barTFull[t], 1);
            mbar_init(&barTEmpty[t], TC_EPI / 2);
            sCommitted[t] = 0;
            sSeenT[t] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;
    const int nl = blkCnt[b];
    const int64_t lbase = (int64_t)b * L;

    if (warp == 0) {
        // ---- TMA loader: points into the operand ring, norms into the job slot
        if (lane == 0) {
            int i = 0;
            int4 nxt = sidx < nl ? blkEnt[lbase + sidx] : make_int4(0, 0, 0, 0);
            for (int li = sidx; li < nl && !*vFail; li += S) {
                const int4 ent = nxt;
                if (li + S < nl) nxt = blkEnt[lbase + li + S];
                for (int t0 = 0; t0 < ent.z; t0 += TC_NT, i++) {
                    const int so = i % TC_SO, sj = i % TC_SJ;
                    if (!mbar_wait_or_fail(&barBEmpty[so], ((i / TC_SO) & 1) ^ 1, vFail) ||
                        !mbar_wait_or_fail(&barJEmpty[sj], ((i / TC_SJ) & 1) ^ 1, vFail)) {
                        atomicOr(&sFail, 1);
                        break;
                    }
                    const int nr = (min(TC_NT, ent.z - t0) + 15) & ~15;
                    const int64_t r = (int64_t)ent.w + t0;
                    mbar_expect_tx(&barBFull[so], (uint32_t)(nr * TC_ROWB));
                    bulk_g2s(sB + so * TC_BSZ, Bsplit + r * TC_K, (uint32_t)(nr * TC_ROWB), &barBFull[so]);
                    sIssB[so]++;
                    mbar_expect_tx(&barJFull[sj], (uint32_t)(nr * 4));
                    bulk_g2s(sJ + sj * TC_JSZ, bNorm + r, (uint32_t)(nr * 4), &barJFull[sj]);
                    sIssJ[sj]++;
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int i = 0;
            int4 nxt = sidx < nl ? blkEnt[lbase + sidx] : make_int4(0, 0, 0, 0);
            for (int li = sidx; li < nl && !*vFail; li += S) {
                const int4 ent = nxt;
                if (li + S < nl) nxt = blkEnt[lbase + li + S];
                for (int t0 = 0; t0 < ent.z; t0 += TC_NT, i++) {
                    const int so = i % TC_SO, tb = i & 1;
                    const uint32_t ph = (i / TC_SO) & 1;
                    if (!mbar_wait_or_fail(&barBFull[so], ph, vFail)) {
                        atomicOr(&sFail, 1);
                        break;
                    }
                    sSeenB[so]++;
                    if (!mbar_wait_or_fail(&barAFull[so], ph, vFail) ||
                        !mbar_wait_or_fail(&barTEmpty[tb], ((i >> 1) & 1) ^ 1, vFail)) {
                        atomicOr(&sFail, 1);
                        break;
                    }
                    tc_fence_after();
                    const int N = (min(TC_NT, ent.z - t0) + 15) & ~15;
                    const uint32_t idesc = umma_idesc_bf16(TC_MT, N);
                    const int nmt = sNpart[i % TC_SJ] > TC_MT ? 2 : 1;
                    const uint32_t bBase = smem_u32(sB + so * TC_BSZ);
                    for (int mt = 0; mt < nmt; mt++) {
                        const uint32_t aBase = smem_u32(sA + so * TC_ASZ + mt * (TC_MT * TC_ROWB));
#pragma unroll
                        for (int ks = 0; ks < TC_K / 16; ks++) {
                            const uint64_t ad = umma_sdesc(aBase + ks * 256, 128, 6 * 128);
                            const uint64_t bd = umma_sdesc(bBase + ks * 256, 128, 6 * 128);
                            umma_bf16(tmem + (uint32_t)(tb * 256 + mt * TC_NT), ad, bd, idesc, ks > 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(&barBEmpty[so]);
                    umma_commit(&barAEmpty[so]);
                    umma_commit(&barTFull[tb]);
                    sCommitted[tb]++;
                }
            }
        }
    } else if (warp < 6) {
        // ---- operand builders (128 threads): compact the partial queries;
        // every decision is uniform over the builders (named barrier 1)
        const int t = tid - 64, wb = warp - 2;
        int i = 0;
        int4 nxt = sidx < nl ? blkEnt[lbase + sidx] : make_int4(0, 0, 0, 0);
        uint32_t mnxt = (sidx < nl && lane < TC_MW) ? blkMask[(lbase + sidx) * TC_MW + lane] : 0u;
        for (int li = sidx; li < nl; li += S) {
            const int4 ent = nxt;
            const uint32_t mwl = mnxt;
            if (li + S < nl) {
                nxt = blkEnt[lbase + li + S];
                mnxt = lane < TC_MW ? blkMask[(lbase + li + S) * TC_MW + lane] : 0u;
            }
            // builder warp wb handles queries j = t (word wb) and t + 128
            // (word wb + 4); prefix popcounts of the mask words by shuffles
            const uint32_t pc = lane < TC_MW ? (uint32_t)__popc(mwl) : 0u;
            uint32_t inc = pc;
#pragma unroll
            for (int o = 1; o < TC_MW; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t excl = inc - pc;
            const int npart = (int)__shfl_sync(0xffffffffu, inc, TC_MW - 1);
            const uint32_t wA = __shfl_sync(0xffffffffu, mwl, wb), wB = __shfl_sync(0xffffffffu, mwl, wb + 4);
            const int preA = (int)__shfl_sync(0xffffffffu, excl, wb), preB = (int)__shfl_sync(0xffffffffu, excl, wb + 4);
            const uint32_t below = (1u << lane) - 1u;
            bool failed = false;
            for (int t0 = 0; t0 < ent.z; t0 += TC_NT, i++) {
                const int so = i % TC_SO, sj = i % TC_SJ;
                const bool bad = !mbar_wait_or_fail(&barAEmpty[so], ((i / TC_SO) & 1) ^ 1, vFail) ||
                                 !mbar_wait_or_fail(&barJEmpty[sj], ((i / TC_SJ) & 1) ^ 1, vFail);
                if (bar1_or_128(bad || *vFail != 0)) {
                    failed = true;
                    break;
                }
                int *map = (int *)(sJ + sj * TC_JSZ + TC_NT * 4);
                if ((wA >> lane) & 1u) map[preA + __popc(wA & below)] = t;
                if ((wB >> lane) & 1u) map[preB + __popc(wB & below)] = t + 128;
                asm volatile("bar.sync 1, 128;" ::: "memory");
                // operand rows: rank r -> M-tile r / 128, row r % 128
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    const int r = t + hh * 128;
                    if (r < npart) {
                        const uint4 *src = (const uint4 *)(sQr + map[r] * TC_ROWB);
                        unsigned char *dst = sA + so * TC_ASZ + hh * (TC_MT * TC_ROWB);
                        const int g = t >> 3, ii = t & 7;
#pragma unroll
                        for (int kg = 0; kg < 6; kg++) *(uint4 *)(dst + ((g * 6 + kg) * 8 + ii) * 16) = src[kg];
                    }
                }
                if (t == 0) sNpart[sj] = npart;
                fence_async_shared();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (t == 0) {
                    mbar_arrive(&barAFull[so]);
                    mbar_arrive(&barJFull[sj]);
                }
            }
            if (failed) {
                if (t == 0) atomicOr(&sFail, 1);
                break;
            }
        }
    } else {
        // ---- epilogue: warp (buffer tb, M-tile mt, lane quarter qd); wait
        // outcomes are made uniform over the warp before any warp-collective
        // TMEM load
        const int e = warp - 6, tb = e >> 3, mt = (e >> 2) & 1, qd = warp & 3;
        const uint32_t taddr = tmem + (uint32_t)(tb * 256 + mt * TC_NT) + ((uint32_t)(qd * 32) << 16);
        int2 *stage = sMay + e * TC_MAYBE;   // this warp's undecided pairs
        int nstage = 0;                      // warp-uniform
        int i = 0, seenT = 0;
        int4 nxt = sidx < nl ? blkEnt[lbase + sidx] : make_int4(0, 0, 0, 0);
        for (int li = sidx; li < nl; li += S) {
            if (__any_sync(0xffffffffu, *vFail != 0)) break;
            const int4 ent = nxt;
            if (li + S < nl) nxt = blkEnt[lbase + li + S];
            bool failed = false;
            for (int t0 = 0; t0 < ent.z; t0 += TC_NT, i++) {
                if ((i & 1) != tb) continue;
                const int sj = i % TC_SJ;
                if (!__all_sync(0xffffffffu, mbar_wait_or_fail(&barTFull[tb], (i >> 1) & 1, vFail))) {
                    failed = true;
                    break;
                }
                seenT++;
                if (!__all_sync(0xffffffffu, mbar_wait_or_fail(&barJFull[sj], (i / TC_SJ) & 1, vFail))) {
                    failed = true;
                    break;
                }
                if (lane == 0) atomicMax(&sSeenJ[sj], i / TC_SJ + 1);
                tc_fence_after();
                const int npart = sNpart[sj];
                const int rows = min(TC_NT, ent.z - t0);
                const int rank0 = mt * TC_MT + qd * 32;
                if (rank0 < npart) {
                    const int rank = rank0 + lane;
                    const bool valid = rank < npart;
                    const float *no = (const float *)(sJ + sj * TC_JSZ);
                    const int j = valid ? ((const int *)(sJ + sj * TC_JSZ + TC_NT * 4))[rank] : 0;
                    float4 P = sPar[j];
                    if (!valid) P.y = P.z = __int_as_float(0x7fffffff);   // NaN: every comparison false
                    int sure = 0;
                    for (int c0 = 0; c0 < rows; c0 += 16) {
                        float v[16];
                        __syncwarp();
                        tmem_ld16(taddr + (uint32_t)c0, v);
                        // branch-free over the 16 columns: padding columns have
                        // NaN norms, so neither test holds for them
                        float nv[16];
#pragma unroll
                        for (int c4 = 0; c4 < 4; c4++) {
                            const float4 n4 = *(const float4 *)(no + c0 + 4 * c4);
                            nv[4 * c4] = n4.x;
                            nv[4 * c4 + 1] = n4.y;
                            nv[4 * c4 + 2] = n4.z;
                            nv[4 * c4 + 3] = n4.w;
                        }
                        uint32_t mb = 0u;   // columns inside the error band
#pragma unroll
                        for (int c = 0; c < 16; c++) {
                            const float vt = __fmaf_rn(-2.f, v[c], __fadd_rn(nv[c], P.x));
                            sure += vt <= P.y ? 1 : 0;
                            mb |= (vt > P.y && vt <= P.z) ? (1u << c) : 0u;
                        }
                        if (__any_sync(0xffffffffu, mb != 0u)) {
                            // warp-aggregated append to the stage (flushed when full)
                            const int cnt = __popc(mb);
                            int incl = cnt;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += y;
                            }
                            const int total = __shfl_sync(0xffffffffu, incl, 31);
                            if (nstage + total > TC_MAYBE) may_flush(stage, nstage, lane, recheckN, recheckCap, recheck);
                            int at = nstage + incl - cnt;
                            while (mb) {
                                const int c = __ffs(mb) - 1;
                                mb &= mb - 1;
                                const int2 rec = make_int2(a0 + j, ent.y + t0 + c0 + c);
                                if (at < TC_MAYBE) {
                                    stage[at] = rec;
                                } else {
                                    // more than a full stage in one chunk (at most 512)
                                    const int g = atomicAdd(recheckN, 1);
                                    if (g < recheckCap) recheck[g] = rec;
                                }
                                at++;
                            }
                            nstage = min(TC_MAYBE, nstage + total);
                            __syncwarp();
                        }
                    }
                    if (valid && sure) atomicAdd(&sCntS[j], sure);
                }
                __syncwarp();
                tc_fence_before();
                if (lane == 0) {
                    mbar_arrive(&barTEmpty[tb]);
                    mbar_arrive(&barJEmpty[sj]);
                }
            }
            if (failed) {
                atomicOr(&sFail, 1);
                break;
            }
        }
        if (lane == 0) atomicMax(&sSeenT[tb], seenT);
        may_flush(stage, nstage, lane, recheckN, recheckCap, recheck);
    }
    __syncthreads();
    if (tid < nb && sCntS[tid]) atomicAdd(&cntSure[a0 + tid], sCntS[tid]);
    if (tid == 0 && sFail) {
        atomicOr(errFlag, 128);
        // nothing may land in shared memory or TMEM after the CTA leaves:
        // wait (bounded) for the copies and MMAs not yet seen complete
        for (int st = 0; st < TC_SO; st++)
            if (sIssB[st] > sSeenB[st]) mbar_wait_bounded(&barBFull[st], (uint32_t)((sIssB[st] - 1) & 1));
        for (int s = 0; s < TC_SJ; s++)
            if (sIssJ[s] > sSeenJ[s]) mbar_wait_bounded(&barJFull[s], (uint32_t)((sIssJ[s] - 1) & 1));
        for (int t = 0; t < 2; t++)
            if (sCommitted[t] > sSeenT[t]) mbar_wait_bounded(&barTFull[t], (uint32_t)((sCommitted[t] - 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// Exact decision of the pairs the tensor-core count left inside its error
// band, in k_count's arithmetic: surely in -> count, band -> band list.
__global__ void k_recheck(const int *__restrict__ recheckN, int recheckCap, const int2 *__restrict__ recheck,
                          const int32_t *__restrict__ act, const Thr *__restrict__ thr,
                          const float *__restrict__ qp32, const float *__restrict__ O32,
                          int *__restrict__ cntSure, int *__restrict__ cntBand, int *__restrict__ bandN, int bandCap,
                          int *__restrict__ bandA, int *__restrict__ bandPos)
{
    const int n = min(*recheckN, recheckCap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int2 rec = recheck[e];
        const int a = rec.x;
        const Thr T = thr[a];
        const int cls = exact_class(O32 + (int64_t)rec.y * PM_MP, qp32 + (int64_t)act[a] * PM_MP, T.lo, T.hi);
        if (cls == 1) {
            atomicAdd(&cntSure[a], 1);
        } else if (cls == 2) {
            atomicAdd(&cntBand[a], 1);
            const int e2 = atomicAdd(bandN, 1);
            if (e2 < bandCap) {
                bandA[e2] = a;
                bandPos[e2] = rec.y;
            }
        }
    }
}

// Empties the results of the listed queries (-1, +inf, 0).
__global__ void k_clear_results(const int32_t *__restrict__ qs, int nn, int k, int64_t *__restrict__ ids,
                                float *__restrict__ dd, float *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    for (int e = 0; e < k; e++) {
        const int64_t o = (int64_t)qs[i] * k + e;
        ids[o] = -1;
        dd[o] = INFINITY;
        err[o] = 0.f;
    }
}

// Sub-batch of the active queries (the ones whose exact range count is
// needed): their query ids and round thresholds.
__global__ void k_gather_sub(const int *__restrict__ idx, int n2, const int32_t *__restrict__ act,
                             const Thr *__restrict__ thr, int32_t *__restrict__ act2, Thr *__restrict__ thr2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    act2[i] = act[idx[i]];
    thr2[i] = thr[idx[i]];
}

// Locality order: counting sort of queries by leaf key.
__global__ void k_hist(const unsigned int *__restrict__ key, int64_t nq, int *__restrict__ h)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nq) atomicAdd(&h[key[q]], 1);
}

__global__ void k_scan_single(int *__restrict__ h, int64_t L)
{
    // one block: exclusive scan of L counters, 1024 at a time
    __shared__ int carry;
    __shared__ int buf[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < L; b0 += 1024) {
        int64_t i = b0 + threadIdx.x;
        int v = i < L ? h[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < L) h[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
}

__global__ void k_scatter_order(const unsigned int *__restrict__ key, int64_t nq, int *__restrict__ h,
                                int32_t *__restrict__ order)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nq) order[atomicAdd(&h[key[q]], 1)] = (int32_t)q;
}

template <class T> T *grow(DevBuf &b, size_t count, pmlsh_status &st)
{
    if (st != PMLSH_OK) return nullptr;
    st = b.reserve(count * sizeof(T));
    return st == PMLSH_OK ? b.as<T>() : nullptr;
}

}  // namespace

namespace {

// Launch shape of the verification for rows of length ld and a top-KP of KP:
// the grouped kernel (verify_group.cu) when its shared memory fits, the
// single-query kernel otherwise.
struct VerifyPlan {
    int nsm = 148;
    int vWarps = 0, vPerSM = 1;   // single-query kernel
    int vPerSMw = 1;              // its register-rich form (for batches that fit one wave of it)
    size_t vsmem = 0;
    int gvTR = 0, gvPerSM = 0;    // grouped kernel
    size_t gvSmem = 0;
    bool grouped = false;
};

pmlsh_status verify_plan(int ld, int KP, VerifyPlan &vp, bool bf16 = false)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&vp.nsm, cudaDevAttrMultiProcessorCount, dev);
    // single-query kernel: one warp per query, as many warps per block as
    // shared memory allows (up to VW_MAXWARPS)
    const size_t vwarp = verify_smem_warp(ld, KP, bf16 ? 1 : 0);
    vp.vWarps = (int)std::min<size_t>(VW_MAXWARPS, (size_t)(227 * 1024) / vwarp);
    if (vp.vWarps < 1) return PMLSH_OK;
    vp.vsmem = (size_t)vp.vWarps * vwarp;
    const void *kn = (const void *)k_verify<false, true>;
    const void *kw = bf16 ? (const void *)k_verify<true, true> : (const void *)k_verify<true, false>;
    PM_TRY(pm_allow_max_dyn_smem(kn));
    PM_TRY(pm_allow_max_dyn_smem(kw));
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&vp.vPerSM, kn, 32 * vp.vWarps, vp.vsmem));
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&vp.vPerSMw, kw, 32 * vp.vWarps, vp.vsmem));
    vp.vPerSM = std::max(1, vp.vPerSM);
    vp.vPerSMw = std::max(1, vp.vPerSMw);
    vp.gvTR = gv_tile_rows(ld);
    vp.gvSmem = vp.gvTR > 0 ? gv_smem_bytes(ld, KP, vp.gvTR) : 0;
    if (vp.gvTR > 0 && vp.gvSmem <= (size_t)pm_max_smem_optin()) PM_TRY(gv_ctas_per_sm(vp.gvSmem, &vp.gvPerSM));
    const char *vsel = std::getenv("PMLSH_VERIFY");
    // (the grouped kernel has no BF16 first pass)
    vp.grouped = !bf16 && vp.gvPerSM > 0 && vsel && std::strcmp(vsel, "group") == 0;
    return PMLSH_OK;
}

}  // namespace

namespace {

// The bytes pm_knn grows each workspace buffer to for a batch of nq queries
// (the largest of the sizes it asks for; the budget selection's key buffers,
// which depend on the data, are left out).
void knn_work_needs(const pmlsh_index *ix, int64_t nq, int k, int precision,
                    std::vector<std::pair<DevBuf KnnWork::*, int64_t>> &out)
{
    const int64_t L = ix->L, ld = ix->ld, W32 = pm_leaf_words(L);
    const bool bfv = (precision & PMLSH_BF16_VERIFY) != 0 && ix->Xr != nullptr;
    const int KP = (k + (bfv ? 64 : 32) + 31) / 32 * 32;
    const bool tc = (precision & PMLSH_BF16_TENSOR) != 0;
    VerifyPlan vp;
    if (verify_plan((int)ld, KP, vp, bfv) != PMLSH_OK)
        vp = VerifyPlan();
    const int64_t nlq = (nq + QB - 1) / QB, nlt = tc ? (nq + TC_QN - 1) / TC_QN : 0;
    const int64_t nlist = std::max(nlq, nlt);
    int64_t vscratch;
    if (vp.grouped) {
        const int64_t grid = std::max<int64_t>(
            1, std::min<int64_t>((nq + GV_WARPS - 1) / GV_WARPS, (int64_t)vp.gvPerSM * vp.nsm));
        vscratch = grid * L * 9 + 64;
    } else {
        const int64_t vw = std::max(1, vp.vWarps);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((nq + vw - 1) / vw, (int64_t)vp.vPerSM * vp.nsm));
        vscratch = grid * vw * L * 8;
    }
    out = {
        {&KnnWork::Qd, nq * ld * 4}, {&KnnWork::qp64, nq * PM_MP * 8}, {&KnnWork::qp32, nq * PM_MP * 4},
        {&KnnWork::qnorm, nq * 8}, {&KnnWork::qpiv, nq * PM_MAX_PIVOTS * 4}, {&KnnWork::keys, nq * 4},
        {&KnnWork::order, nq * 4}, {&KnnWork::qpca, nq * (PM_PCA + 1) * 4}, {&KnnWork::keys2, (L + 1) * 4},
        {&KnnWork::qstate, nq * 8}, {&KnnWork::outIds, nq * k * 8}, {&KnnWork::outD64, nq * k * 4},
        {&KnnWork::outErr, nq * k * 4}, {&KnnWork::active, nq * 4}, {&KnnWork::thr, nq * (int64_t)sizeof(Thr)},
        {&KnnWork::cntSure, nq * 4}, {&KnnWork::cntBand, nq * 4}, {&KnnWork::cntPart, nq * 4},
        {&KnnWork::cntTight, nq * 8},
        {&KnnWork::bandCnt, nq * 4}, {&KnnWork::bandIn, nq * 4}, {&KnnWork::bandInQ, nq * BCAP * 4},
        {&KnnWork::bandQ, ((int64_t)1 << 20) * 4}, {&KnnWork::bandPos, ((int64_t)1 << 20) * 4},
        {&KnnWork::flags, (nq + 8) * 4}, {&KnnWork::dk, nq * 8}, {&KnnWork::leafBits, nq * W32 * 4},
        {&KnnWork::fullBits, nq * W32 * 4},
        {&KnnWork::recheck, tc ? ((int64_t)1 << 23) * 8 : 0},
        {&KnnWork::blkCnt, nlist * 4}, {&KnnWork::blkLeaves, nlist * L * 16},
        {&KnnWork::blkMask, std::max(nlq * L * (QB / 32) * 4, nlt * L * TC_MW * 4)},
        // the straddling sub-batch (at most the whole batch)
        {&KnnWork::subIdx, nq * (12 + BCAP) * 4}, {&KnnWork::subThr, nq * (int64_t)sizeof(Thr)},
        {&KnnWork::subBits, nq * W32 * 4},
        // verification
        {&KnnWork::partSeen, (4 * nq + 8) * 4}, {&KnnWork::partD, vscratch},
    };
}

}  // namespace

int64_t pm_knn_work_bytes(const pmlsh_index *ix, int64_t nq, int k, int precision)
{
    std::vector<std::pair<DevBuf KnnWork::*, int64_t>> need;
    knn_work_needs(ix, nq, k, precision, need);
    int64_t b = 0;
    for (auto &e : need) b += e.second > 0 ? std::max<int64_t>(e.second, 256) : 0;
    return b;
}

int64_t pm_knn_work_growth(const pmlsh_index *ix, int64_t nq, int k, int precision, const KnnWork &w)
{
    std::vector<std::pair<DevBuf KnnWork::*, int64_t>> need;
    knn_work_needs(ix, nq, k, precision, need);
    int64_t b = 0;
    for (auto &e : need) {
        const int64_t want = e.second > 0 ? std::max<int64_t>(e.second, 256) : 0;
        const int64_t have = (int64_t)(w.*(e.first)).bytes;
        if (want > have) b += want;   // the buffer is freed and allocated anew
        if (want > have) b -= have;
    }
    return b;
}

int64_t pm_work_resident(const KnnWork &w)
{
    const DevBuf *bufs[] = {&w.Qd, &w.qp32, &w.qp64, &w.qnorm, &w.qpiv, &w.order, &w.keys, &w.keys2, &w.vals2,
                            &w.sortTmp, &w.qstate, &w.thr, &w.blkCnt, &w.blkLeaves, &w.cntSure, &w.cntBand,
                            &w.bandQ, &w.bandPos, &w.bandIn, &w.bandCnt, &w.partD, &w.partI, &w.partSeen,
                            &w.bandInQ, &w.outD64, &w.outIds, &w.outErr, &w.dk, &w.flags, &w.selBuf, &w.selOff,
                            &w.selCnt, &w.selTau, &w.active, &w.misc, &w.blkMask, &w.recheck, &w.leafBits,
                            &w.fullBits, &w.cntPart, &w.cntTight, &w.subIdx, &w.subThr, &w.subBits, &w.qpca};
    int64_t b = 0;
    for (const DevBuf *p : bufs) b += (int64_t)p->bytes;
    return b;
}

pmlsh_status pm_project_rows(const pmlsh_index *ix, const float *Q, int64_t nq, float *staging,
                             double *out64, float *out32, int ostride, cudaStream_t st)
{
    const int d = ix->d, ld = ix->ld;
    PM_CUDA(cudaMemsetAsync(staging, 0, (size_t)nq * ld * sizeof(float), st));
    PM_CUDA(cudaMemcpy2DAsync(staging, ld * sizeof(float), Q, d * sizeof(float), d * sizeof(float), nq,
                              pm_is_device_ptr(Q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    pm_launch_project64(staging, nq, ld, d, ix->m, ix->A32, out64, out32, nullptr, st, ostride);
    PM_CUDA(cudaGetLastError());
    return PMLSH_OK;
}

pmlsh_status pm_knn(pmlsh_index *ix, const float *Q, int64_t nq, const pmlsh_knn_opts *o,
                    int64_t *ids, float *dists, float *err, pmlsh_query_stats *stats,
                    cudaStream_t st, KnnWork *work, bool rcbc)
{
    const int64_t n = ix->n;
    const int d = ix->d, ld = ix->ld, m = ix->m, k = o->k;
    const int64_t L = ix->L;
    KnnWork &w = work ? *work : ix->work;
    // parameters (Eq. 9; budget of Algorithm 2; r_min rule of Sec. 5.2)
    const double t = o->t > 0.0 ? o->t : std::sqrt(pm_chi2_upper_quantile(o->alpha1, m));
    // Algorithm 2: |C| >= beta n + k; Algorithm 1: |C| >= beta n + 1
    const int64_t B = pmlsh_budget(n, o->beta, rcbc ? 1 : k);
    double rmin = o->r_min;
    if (!(rmin > 0.0)) {
        const std::vector<double> &v = ix->distSample;
        double rstar = 1.0;
        if (!v.empty()) {
            double p = std::min(1.0, (o->beta * (double)n + (double)k) / (double)n);
            int64_t N = (int64_t)v.size();
            int64_t rank = (int64_t)std::ceil(p * (double)N - 1e-9);
            rank = std::max<int64_t>(1, std::min<int64_t>(N, rank));
            rstar = v[rank - 1];
            if (!(rstar > 0.0)) {
                rstar = 0.0;
                for (double x : v) if (x > 0.0) { rstar = x; break; }
            }
            rmin = rstar > 0.0 ? rstar / o->c : 1.0;
        } else {
            rmin = 1.0;
        }
    }
    // top-KP size: KP - k entries beyond the k-th catch the FP32 guard band;
    // the BF16 first pass keeps more, its bounds being wider
    const bool bf16v = (o->precision & PMLSH_BF16_VERIFY) != 0 && ix->Xr != nullptr;
    const int KP = (k + (bf16v ? 64 : 32) + 31) / 32 * 32;
    pmlsh_status s = PMLSH_OK;
    float *Qd = grow<float>(w.Qd, (size_t)nq * ld, s);
    double *qp64 = grow<double>(w.qp64, (size_t)nq * PM_MP, s);
    float *qp32 = grow<float>(w.qp32, (size_t)nq * PM_MP, s);
    double *qnorm = grow<double>(w.qnorm, nq, s);
    float *qpiv = grow<float>(w.qpiv, (size_t)nq * PM_MAX_PIVOTS, s);
    unsigned int *key = grow<unsigned int>(w.keys, nq, s);
    int32_t *order = grow<int32_t>(w.order, nq, s);
    float *qpca = grow<float>(w.qpca, (size_t)nq * (PM_PCA + 1), s);
    float *qnx = qpca + (size_t)nq * PM_PCA;
    int *hist = grow<int>(w.keys2, L + 1, s);
    double *rq = grow<double>(w.qstate, nq, s);
    // results go straight to the caller's arrays when those are in device
    // memory, else to scratch copied out at the end
    const bool idev = pm_is_device_ptr(ids), ddev = pm_is_device_ptr(dists);
    const bool edev = err != nullptr && pm_is_device_ptr(err);
    int64_t *oIds = idev ? ids : grow<int64_t>(w.outIds, (size_t)nq * k, s);
    float *oD = ddev ? dists : grow<float>(w.outD64, (size_t)nq * k, s);
    float *oE = edev ? err : grow<float>(w.outErr, (size_t)nq * k, s);
    if (s != PMLSH_OK) return s;
    PM_TRY(pm_project_rows(ix, Q, nq, Qd, qp64, qp32, PM_MP, st));
    const unsigned gq = (unsigned)((nq + 255) / 256);
    PM_LAUNCH("k_query_aux", st, k_query_aux<<<gq, 256, 0, st>>>(qp64, qp32, nq, ix->piv32, ix->s, qnorm, qpiv));
    PM_LAUNCH("k_query_pca", st, k_query_pca<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(Qd, nq, ld, ix->pcaP32, qpca, qnx));
    PM_LAUNCH("k_leaf_key", st, k_leaf_key<<<gq, 256, 0, st>>>(qp32, nq, ix->treeI, ix->treeV, key));
    PM_CUDA(cudaMemsetAsync(hist, 0, (L + 1) * sizeof(int), st));
    PM_LAUNCH("k_hist", st, k_hist<<<gq, 256, 0, st>>>(key, nq, hist));
    PM_LAUNCH("k_scan_single", st, k_scan_single<<<1, 1024, 0, st>>>(hist, L + 1));
    PM_LAUNCH("k_scatter_order", st, k_scatter_order<<<gq, 256, 0, st>>>(key, nq, hist, order));
    PM_CUDA(cudaGetLastError());
    // pinned staging of the per-round decisions: order [nq], bounds [2 nq],
    // verification outputs (k-th distance [nq] f64, fp64/verified/leaves
    // counts [3 nq], error flag)
    // (plus the radii [nq] f64 and an active or straddling list [nq] sent to
    // the device, so that every copy is asynchronous)
    PM_TRY(w.stage.reserve((size_t)nq * (8 + 4 * 8 + 8 + 8 + 4) + 64));
    double *stDk = (double *)w.stage.p;
    double *stR = stDk + nq;
    int2 *stTight = (int2 *)(stR + nq);
    int32_t *stOrder = (int32_t *)(stTight + nq);
    int *stHs = stOrder + nq, *stHp = stHs + nq, *stFp = stHp + nq, *stNv = stFp + nq, *stNl = stNv + nq,
        *stVo = stNl + nq, *stRedo = stVo + nq, *stList = stRedo + nq, *stErr = stList + nq;
    PM_CUDA(cudaMemcpyAsync(stOrder, order, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> orderH;   // host copy, read after the first round's sync

    // host round state
    std::vector<double> r(nq, rmin);
    std::vector<int32_t> rounds(nq, 0), rule(nq, 0), fp64(nq, 0);
    std::vector<int64_t> ncand(nq, 0), nver(nq, 0);
    std::vector<int32_t> nleaf(nq, 0), fallback(nq, 0);
    std::vector<char> done(nq, 0);
    std::memcpy(stR, r.data(), nq * sizeof(double));
    PM_CUDA(cudaMemcpyAsync(rq, stR, nq * sizeof(double), cudaMemcpyHostToDevice, st));

    const int bandCap = 1 << 20;
    int *actBuf = grow<int32_t>(w.active, nq, s);
    Thr *thr = grow<Thr>(w.thr, nq, s);
    int *cntSure = grow<int>(w.cntSure, nq, s);
    int *cntBand = grow<int>(w.cntBand, nq, s);
    int *cntPart = grow<int>(w.cntPart, nq, s);
    int2 *cntTight = grow<int2>(w.cntTight, nq, s);
    int *inTrue = grow<int>(w.bandCnt, nq, s);
    int *inN = grow<int>(w.bandIn, nq, s);
    int *inPos = grow<int>(w.bandInQ, (size_t)nq * BCAP, s);
    int *bandA = grow<int>(w.bandQ, bandCap, s);
    int *bandPos = grow<int>(w.bandPos, bandCap, s);
    int *fpc = grow<int>(w.flags, nq + 8, s);
    double *dk = grow<double>(w.dk, nq, s);
    if (s != PMLSH_OK) return s;
    int *bandN = fpc + nq;       // counters after the per-query array
    int *errFlag = fpc + nq + 1;
    int *recheckN = fpc + nq + 2;
    const int W32 = (int)pm_leaf_words(L);
    uint32_t *leafBits = grow<uint32_t>(w.leafBits, (size_t)nq * W32, s);
    uint32_t *fullBits = grow<uint32_t>(w.fullBits, (size_t)nq * W32, s);
    if (s != PMLSH_OK) return s;

    VerifyPlan vp;
    PM_TRY(verify_plan(ld, KP, vp, bf16v));
    if (vp.vWarps < 1) {
        pm_set_error("d = %d is too large for the verification kernel's shared memory", d);
        return PMLSH_EINVAL;
    }
    const int nsm = vp.nsm, vWarps = vp.vWarps, vPerSM = vp.vPerSM, gvTR = vp.gvTR, gvPerSM = vp.gvPerSM;
    const int vPerSMw = vp.vPerSMw;
    const size_t vsmem = vp.vsmem, gvSmem = vp.gvSmem;
    const bool grouped = vp.grouped;

    const bool tensor = (o->precision & PMLSH_BF16_TENSOR) != 0;
    // the tensor-core count holds all 512 TMEM columns of its SM; its
    // shared memory (over half the SM's) keeps a second CTA off the SM
    if (tensor) PM_TRY(pm_allow_max_dyn_smem((const void *)k_count_tc));
    // pairs the tensor-core count leaves inside its error band (8 M, 64 MB)
    const int recheckCap = 1 << 23;
    int2 *recheck = tensor ? grow<int2>(w.recheck, recheckCap, s) : nullptr;
    if (s != PMLSH_OK) return s;

    std::vector<int32_t> actH;
    actH.reserve(nq);
    for (int round = 0; round < 100000; round++) {
        // round 0: every query, in the order on the device (its host copy is
        // read after this round's first sync); later rounds: the active ones
        int32_t *act = round == 0 ? order : actBuf;
        int na = (int)nq;
        if (round > 0) {
            actH.clear();
            for (int64_t i = 0; i < nq; i++)
                if (!done[orderH[i]]) actH.push_back(orderH[i]);
            na = (int)actH.size();
            if (na == 0) break;
            std::memcpy(stList, actH.data(), na * sizeof(int32_t));
            PM_CUDA(cudaMemcpyAsync(act, stList, na * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        }
        PM_LAUNCH("k_thresholds", st, k_thresholds<<<(na + 255) / 256, 256, 0, st>>>(act, na, rq, t, ix->maxNorm, qnorm, thr));
        // leaf classification (Eq. 5): bounds of |S_i|, leaf lists with the
        // masks of partially covering queries, per-query leaf bit sets.  The
        // phases run on the active batch or on a gathered sub-batch (io).
        struct CountIO {
            const int32_t *act;
            int na;
            const Thr *thr;
            int *cntSure, *cntPart, *cntBand, *inTrue, *inN, *inPos, *fpc;
            uint32_t *leafBits;
            uint32_t *fullBits;   // whole-leaf bits for the verification, or null
            int2 *cntTight;       // partial leaves' members surely / possibly inside (radial profiles), or null
            const int32_t *amb;   // a gathered sub-batch: its rows in the batch (lists from the batch's bits)
        };
        const int64_t Tdec = std::min<int64_t>(B, n);
        auto class_phase = [&](bool tc, const CountIO &io, ZeroList z) -> pmlsh_status {
            const int nlist = tc ? (io.na + TC_QN - 1) / TC_QN : (io.na + QB - 1) / QB;
            const int mwords = tc ? TC_MW : QB / 32;
            pmlsh_status s2 = PMLSH_OK;
            int *blkCnt = grow<int>(w.blkCnt, nlist, s2);
            int4 *blkEnt = grow<int4>(w.blkLeaves, (size_t)nlist * L, s2);
            uint32_t *blkMask = grow<uint32_t>(w.blkMask, (size_t)nlist * L * mwords, s2);
            if (s2 != PMLSH_OK) return s2;
            // the phase's counters (and the caller's extra arrays) in one launch
            z.add(blkCnt, nlist);
            z.add(io.cntSure, io.na);
            z.add(io.cntPart, io.na);
            z.add(io.cntBand, io.na);
            z.add(io.inTrue, io.na);
            z.add(io.inN, io.na);
            z.add(io.fpc, io.na);
            z.add(bandN, 1);
            z.add(recheckN, 1);
            z.add((int *)io.cntTight, io.cntTight ? 2 * io.na : 0);
            PM_LAUNCH("k_zero", st, k_zero<<<2 * nsm, 256, 0, st>>>(z));
            if (io.amb) {
                // a sub-batch: its block lists from the batch's leaf bits
                const int64_t nch = (W32 + 7) / 8;
                const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(nch, ((int64_t)4 * nsm + nlist - 1) / nlist));
                if (!tc)
                    PM_LAUNCH("k_sublists", st, k_sublists<QB><<<dim3((unsigned)nlist, (unsigned)gy), QB, 0, st>>>(
                                                     io.amb, io.na, leafBits, fullBits, W32, L, ix->leafOff, nullptr,
                                                     cntSure, io.cntSure, blkCnt, blkEnt, blkMask));
                else
                    PM_LAUNCH("k_sublists", st, k_sublists<TC_QN><<<dim3((unsigned)nlist, (unsigned)gy), TC_QN, 0, st>>>(
                                                     io.amb, io.na, leafBits, fullBits, W32, L, ix->leafOff, ix->bOff,
                                                     cntSure, io.cntSure, blkCnt, blkEnt, blkMask));
            } else {
                // query-stationary test: leaf tiles split evenly over enough
                // CTAs per query block to fill the GPU once
                const int64_t nTiles = (L + CQ_LT - 1) / CQ_LT;
                const int perSm = tc ? 4 : 16;
                int64_t gx = std::max<int64_t>(1, std::min<int64_t>(nTiles, ((int64_t)nsm * perSm + nlist - 1) / nlist));
                gx = (nTiles + (nTiles + gx - 1) / gx - 1) / ((nTiles + gx - 1) / gx);
                dim3 gq((unsigned)gx, (unsigned)nlist);
                if (!tc)
                    PM_LAUNCH("k_class", st, k_class<QB><<<gq, QB, 0, st>>>(io.act, io.na, io.thr, qp32, qpiv,
                                                ix->s, ix->leafMeta, ix->leafOff, nullptr, L, io.cntSure, blkCnt,
                                                blkEnt, blkMask, io.leafBits, W32, io.cntPart, io.fullBits));
                else
                    PM_LAUNCH("k_class", st, k_class<TC_QN><<<gq, TC_QN, 0, st>>>(io.act, io.na, io.thr, qp32,
                                                qpiv, ix->s, ix->leafMeta, ix->leafOff, ix->bOff, L, io.cntSure,
                                                blkCnt, blkEnt, blkMask, io.leafBits, W32, io.cntPart, io.fullBits));
            }
            if (io.cntTight)
                PM_LAUNCH("k_tight", st, k_tight<<<(unsigned)io.na, 256, 0, st>>>(io.act, io.na, io.thr,
                                               qp32, ix->leafMeta, ix->leafOff, io.leafBits, io.fullBits, W32, L,
                                               io.cntSure, io.cntPart, Tdec, io.cntTight));
            PM_CUDA(cudaGetLastError());
            return PMLSH_OK;
        };
        // the per-point count in the partially covered leaves (CUDA cores
        // or tensor cores), points inside the FP32 error band listed
        auto point_count = [&](bool tc, const CountIO &io) -> pmlsh_status {
            const int nlist = tc ? (io.na + TC_QN - 1) / TC_QN : (io.na + QB - 1) / QB;
            const int *blkCnt = w.blkCnt.as<int>();
            const int4 *blkEnt = w.blkLeaves.as<int4>();
            const uint32_t *blkMask = w.blkMask.as<uint32_t>();
            if (!tc) {
                int splitC = std::max(1, std::min(64, (4 * nsm + nlist - 1) / nlist));
                PM_LAUNCH("k_count", st, k_count<<<dim3(nlist, splitC), 256, 0, st>>>(io.act, io.na, io.thr, qp32,
                                            ix->O32, blkCnt, blkEnt, blkMask, L, io.cntSure, io.cntBand, bandN,
                                            bandCap, bandA, bandPos));
            } else {
                // one CTA per SM at a time: the fewest waves (of up to four)
                // whose CTAs fill at least 95% of their SM slots, each CTA
                // taking a share of its block's list (the prologue, building
                // the block's query operand rows, is paid once per CTA)
                int splitC = 1;
                for (int wv = 1; wv <= 4; wv++) {
                    splitC = std::max(1, std::min(256, wv * nsm / nlist));
                    const int64_t tot = (int64_t)nlist * splitC, waves = (tot + nsm - 1) / nsm;
                    if ((double)tot >= 0.95 * (double)(waves * nsm)) break;
                }
                PM_LAUNCH("k_count_tc", st, k_count_tc<<<dim3(nlist, splitC), TC_THREADS, TC_SMEM, st>>>(
                                            io.act, io.na, io.thr, qp32, ix->Bsplit, ix->bNorm, blkCnt, blkEnt,
                                            blkMask, L, ix->maxNorm, io.cntSure, recheckN, recheckCap, recheck,
                                            errFlag));
                PM_LAUNCH("k_recheck", st, k_recheck<<<4 * nsm, 256, 0, st>>>(recheckN, recheckCap, recheck, io.act,
                                            io.thr, qp32, ix->O32, io.cntSure, io.cntBand, bandN, bandCap, bandA,
                                            bandPos));
            }
            PM_CUDA(cudaGetLastError());
            return PMLSH_OK;
        };
        // exact count: per-point test, FP64 band resolution; host copies of
        // the sure, band and band-in counts
        auto exact_count = [&](const CountIO &io, std::vector<int> &es, std::vector<int> &eb,
                               std::vector<int> &ein) -> pmlsh_status {
            // count, FP64 decision of the band (the band size is read on the
            // device), and one read of the counters; if the tensor-core
            // count left more undecided pairs than its recheck list holds,
            // the round is counted again on the CUDA cores (same results)
            int hN[3] = {0, 0, 0};   // bandN, errFlag, recheckN
            for (int pass = 0; pass < 2; pass++) {
                const bool tcp = tensor && pass == 0;
                if (pass == 1) PM_TRY(class_phase(false, io, ZeroList()));
                PM_TRY(point_count(tcp, io));
                PM_LAUNCH("k_band64", st, k_band64<<<2 * nsm, 256, 0, st>>>(bandN, bandCap, bandA, bandPos, io.act,
                                                       io.thr, ix->O64, qp64, m, io.inTrue, io.inN, io.inPos,
                                                       io.fpc, errFlag));
                PM_CUDA(cudaGetLastError());
                es.resize(io.na);
                eb.resize(io.na);
                ein.resize(io.na);
                PM_CUDA(cudaMemcpyAsync(hN, bandN, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
                PM_CUDA(cudaMemcpyAsync(es.data(), io.cntSure, io.na * sizeof(int), cudaMemcpyDeviceToHost, st));
                PM_CUDA(cudaMemcpyAsync(eb.data(), io.cntBand, io.na * sizeof(int), cudaMemcpyDeviceToHost, st));
                PM_CUDA(cudaMemcpyAsync(ein.data(), io.inTrue, io.na * sizeof(int), cudaMemcpyDeviceToHost, st));
                PM_CUDA(cudaStreamSynchronize(st));
                if (!(tcp && hN[2] > recheckCap)) break;
            }
            if (hN[0] > bandCap) {
                pm_set_error("more than %d projected distances fell inside the FP32 error band in one round", bandCap);
                return PMLSH_EINTERNAL;
            }
            return PMLSH_OK;
        };
        const CountIO full{act, na, thr, cntSure, cntPart, cntBand, inTrue, inN, inPos, fpc, leafBits, fullBits,
                           stats == nullptr ? cntTight : nullptr, nullptr};
        {
            // this round's per-query counters and the error and list counters
            // after them (fpc [nq + 8]) start at zero
            ZeroList z;
            z.add(fpc, nq + 8);
            PM_TRY(class_phase(tensor, full, z));
        }
        std::vector<int> hs(na), hp(na), hb(na, 0), hin(na, 0);
        std::vector<int2> ht;
        PM_CUDA(cudaMemcpyAsync(stHs, cntSure, na * sizeof(int), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaMemcpyAsync(stHp, cntPart, na * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (full.cntTight) PM_CUDA(cudaMemcpyAsync(stTight, cntTight, na * sizeof(int2), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        std::memcpy(hs.data(), stHs, na * sizeof(int));
        std::memcpy(hp.data(), stHp, na * sizeof(int));
        if (full.cntTight) ht.assign(stTight, stTight + na);
        if (round == 0) {
            orderH.assign(stOrder, stOrder + nq);
            actH.assign(stOrder, stOrder + nq);
        }
        // The decisions of Algorithm 2 compare |S_i| only with min(B, n)
        // (rule 2: |S_i| >= B; rule 3: |S_i| = n).  Whole-leaf counts bound
        // |S_i| from below and whole partial leaves from above.  The exact
        // count runs for every query when the caller asks for the statistics
        // (|C| is one of them), else only for the queries whose bounds
        // straddle min(B, n); for the rest the verification decides the FP32
        // band points it meets in FP64 itself.
        const bool needExact = stats != nullptr;
        // hb: points with FP32 d'^2 <= hi beyond the sure ones (the budget
        // selection's capacity); without the exact count, the partial leaves
        std::vector<int32_t> ambH;
        if (needExact) {
            PM_TRY(exact_count(full, hs, hb, hin));
        } else {
            // the bounds of |S_i| from whole leaves, tightened by the partial
            // leaves' radial profiles; a query whose lower bound reaches
            // min(B, n) counts as min(B, n) (rule 2, or rule 3 when n < B)
            for (int a = 0; a < na; a++) {
                hb[a] = hp[a];
                if (hs[a] >= Tdec) continue;
                const int64_t lo = ht.empty() ? hs[a] : (int64_t)hs[a] + ht[a].x;
                const int64_t up = ht.empty() ? (int64_t)hs[a] + hp[a] : (int64_t)hs[a] + ht[a].y;
                if (lo >= Tdec) hin[a] = (int)(Tdec - hs[a]);
                else if (up >= Tdec) ambH.push_back(a);
            }
        }
        // Verification work order, decided here so that the host's pass runs
        // while the GPU counts the straddling sub-batch: the queries with the
        // most range candidates (their upper bound) first, so that the long ones do not finish last;
        // locality order inside each of 32 logarithmic cost classes.  The
        // grouped kernel takes groups of GV_WARPS consecutive active queries
        // (locality order), a group's cost class being its costliest
        // member's.
        int *nverD = grow<int>(w.partSeen, (size_t)4 * na + 8, s);
        int *vOrder = nverD + 2 * na + 8;
        int *redoD = vOrder + na;   // queries left by the BF16 first pass
        const int ngroups = (na + GV_WARPS - 1) / GV_WARPS;
        {
            const int nunits = grouped ? ngroups : na;
            std::vector<int32_t> cls(nunits, 31);
            int64_t hist[33] = {0};
            for (int a = 0; a < na; a++) {
                const uint64_t c = (uint64_t)((int64_t)hs[a] + hb[a] + 1);
                const int b = std::min(31, 63 - __builtin_clzll(c));   // floor(log2 c)
                const int u = grouped ? a / GV_WARPS : a;
                cls[u] = std::min(cls[u], 31 - b);   // costliest class first
            }
            for (int u = 0; u < nunits; u++) hist[cls[u] + 1]++;
            for (int b = 0; b < 32; b++) hist[b + 1] += hist[b];
            for (int u = 0; u < nunits; u++) stVo[hist[cls[u]]++] = u;
            PM_CUDA(cudaMemcpyAsync(vOrder, stVo, nunits * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        }
        if (!ambH.empty()) {
            // exact count of the sub-batch whose bounds straddle min(B, n)
            const int na2 = (int)ambH.size();
            int *sub = grow<int>(w.subIdx, (size_t)na2 * (12 + BCAP), s);
            Thr *thr2 = grow<Thr>(w.subThr, na2, s);
            uint32_t *bits2 = grow<uint32_t>(w.subBits, (size_t)na2 * W32, s);
            if (s != PMLSH_OK) return s;
            int *amb = sub, *act2 = sub + na2, *s2Sure = sub + 2 * na2, *s2Part = sub + 3 * na2,
                *s2Band = sub + 4 * na2, *s2In = sub + 5 * na2, *s2InN = sub + 6 * na2, *s2Fp = sub + 7 * na2,
                *s2InPos = sub + 12 * na2;
            std::memcpy(stList, ambH.data(), na2 * sizeof(int32_t));   // (the round's active list is on the device)
            PM_CUDA(cudaMemcpyAsync(amb, stList, na2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            PM_LAUNCH("k_gather_sub", st, k_gather_sub<<<(na2 + 255) / 256, 256, 0, st>>>(amb, na2, act, thr, act2, thr2));
            const CountIO subIO{act2, na2, thr2, s2Sure, s2Part, s2Band, s2In, s2InN, s2InPos, s2Fp, bits2, nullptr,
                                nullptr, amb};
            PM_TRY(class_phase(tensor, subIO, ZeroList()));   // zeroes inTrue, inN, fp64 of the sub-batch
            std::vector<int> es, eb, ein;
            PM_TRY(exact_count(subIO, es, eb, ein));
            for (int i = 0; i < na2; i++) {
                const int a = ambH[i];
                hs[a] = es[i];
                hb[a] = eb[i];
                hin[a] = ein[i];
            }
        }
        // which queries reached the budget (rule 2)
        std::vector<int32_t> selH;
        std::vector<int64_t> selOffH;
        std::vector<int64_t> count(na);
        int64_t selTotal = 0;
        for (int a = 0; a < na; a++) {
            count[a] = (int64_t)hs[a] + hin[a];
            if (count[a] >= B && !rcbc) {   // Algorithm 1 keeps the whole range set
                selH.push_back(a);
                selOffH.push_back(selTotal);
                selTotal += (int64_t)hs[a] + hb[a];
            }
        }
        if (!selH.empty()) {
            const int ns = (int)selH.size();
            int32_t *sel = grow<int32_t>(w.selTau, ns, s);
            int64_t *selOff = grow<int64_t>(w.selOff, 2 * ns + 1, s);
            int *selCnt = grow<int>(w.selCnt, ns, s);
            float *selKey = grow<float>(w.selBuf, (size_t)selTotal, s);
            int *selPos = grow<int>(w.misc, (size_t)selTotal, s);
            if (s != PMLSH_OK) return s;
            PM_CUDA(cudaMemcpyAsync(sel, selH.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            selOffH.push_back(selTotal);
            std::vector<int64_t> capH(ns);
            for (int i = 0; i < ns; i++) capH[i] = selOffH[i + 1] - selOffH[i];
            PM_CUDA(cudaMemcpyAsync(selOff, selOffH.data(), (ns + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            PM_CUDA(cudaMemcpyAsync(selOff + ns + 1, capH.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            PM_CUDA(cudaMemsetAsync(selCnt, 0, ns * sizeof(int), st));
            // about eight 256-thread blocks per SM over all budget queries
            const int64_t gyc = std::max<int64_t>(1, std::min<int64_t>((L + 255) / 256, ((int64_t)8 * nsm + ns - 1) / ns));
            PM_LAUNCH("k_collect", st, k_collect<<<dim3(ns, (unsigned)gyc), 256, 0, st>>>(
                sel, act, thr, qp32, qpiv, ix->s, ix->leafMeta, ix->leafOff, L, ix->O32, selOff,
                selOff + ns + 1, selCnt, selKey, selPos, errFlag));
            PM_LAUNCH("k_select", st, k_select<<<ns, 1024, 0, st>>>(sel, act, thr, selOff, selCnt, selKey, selPos, B, ix->maxNorm,
                                          qnorm, ix->O64, qp64, m, ix->perm, inN, inPos, fpc, errFlag));
            PM_CUDA(cudaGetLastError());
        }
        // verification (order uploaded above): best-first over candidate
        // leaves, guard set, FP64
        PM_CUDA(cudaMemsetAsync(nverD + 2 * na, 0, 8 * sizeof(int), st));
        if (grouped) {
            const int gGrid = std::max(1, std::min(ngroups, gvPerSM * nsm));
            uint32_t *ukey = grow<uint32_t>(w.partD, (size_t)gGrid * L * 9 / 4 + 16, s);
            if (s != PMLSH_OK) return s;
            GvArgs ga;
            ga.act = act; ga.na = na; ga.thr = thr; ga.qp32 = qp32; ga.qpiv = qpiv; ga.s = ix->s;
            ga.meta = ix->leafMeta; ga.L = L; ga.O32 = ix->O32; ga.X = ix->X; ga.Qd = Qd;
            ga.ld = ld; ga.d = d; ga.leafMu = ix->leafMu; ga.leafRx = ix->leafRx; ga.leafOff = ix->leafOff;
            ga.KP = KP; ga.k = k;
            ga.inN = inN; ga.inPos = inPos; ga.perm = ix->perm; ga.outIds = oIds; ga.outD = oD; ga.outErr = oE;
            ga.dk = dk; ga.fp64cnt = fpc; ga.nverOut = nverD; ga.nleafOut = nverD + na; ga.errFlag = errFlag;
            ga.workCtr = nverD + 2 * na; ga.dbg = nverD + 2 * na + 1; ga.n = n;
            ga.leafBits = leafBits; ga.W32 = W32;
            ga.O64 = ix->O64; ga.qp64 = qp64; ga.m = m; ga.inlineBand = needExact ? 0 : 1;
            ga.leafPmu = ix->leafPmu; ga.qpca = qpca; ga.qnx = qnx;
            ga.muMax = (float)(ix->muMax * (1.0 + 1e-6)) + 1e-30f;
            ga.gOrder = vOrder; ga.ngroups = ngroups;
            ga.ukey = ukey;
            ga.uleaf = (int32_t *)(ukey + (size_t)gGrid * L);
            ga.umask = (uint8_t *)(ga.uleaf + (size_t)gGrid * L);
            ga.TR = gvTR;
            PM_TRY(gv_launch(ga, gGrid, gvSmem, st));
        } else {
            // a batch that one wave of the register-rich form holds takes it
            // (more loads in flight per lane; resident warps do not limit it)
            const bool wide = na <= vPerSMw * nsm * vWarps;
            const int vGrid = std::max(1, std::min((na + vWarps - 1) / vWarps, (wide ? vPerSMw : vPerSM) * nsm));
            int2 *vLists = grow<int2>(w.partD, (size_t)vGrid * vWarps * L, s);
            if (s != PMLSH_OK) return s;
            VwArgs va;
            va.act = act; va.na = na; va.thr = thr; va.qp32 = qp32; va.qpiv = qpiv; va.s = ix->s;
            va.meta = ix->leafMeta; va.L = L; va.O32 = ix->O32; va.X = ix->X; va.Qd = Qd;
            va.ld = ld; va.d = d; va.leafMu = ix->leafMu; va.leafRx = ix->leafRx; va.chunkOff = ix->chunkOff;
            va.leafChunk = ix->leafChunk; va.chunkMu = ix->chunkMu; va.chunkRx = ix->chunkRx; va.KP = KP; va.k = k;
            va.inN = inN; va.inPos = inPos; va.perm = ix->perm; va.outIds = oIds; va.outD = oD; va.outErr = oE;
            va.dk = dk; va.fp64cnt = fpc; va.nverOut = nverD; va.nleafOut = nverD + na; va.errFlag = errFlag;
            va.workCtr = nverD + 2 * na; va.dbg = nverD + 2 * na + 1; va.n = n; va.lists = vLists;
            va.order = vOrder;
            va.leafBits = leafBits; va.fullBits = fullBits; va.W32 = W32;
            va.O64 = ix->O64; va.qp64 = qp64; va.m = m; va.inlineBand = needExact ? 0 : 1;
            va.leafPmu = ix->leafPmu; va.qpca = qpca; va.qnx = qnx;
            va.muMax = (float)(ix->muMax * (1.0 + 1e-6)) + 1e-30f;
            va.nwork = na;
            va.bf16 = bf16v ? 1 : 0;
            va.Xr = ix->Xr;
            va.rowErr = ix->rowErr;
            va.redo = redoD;
            if (bf16v) PM_CUDA(cudaMemsetAsync(redoD, 0, na * sizeof(int), st));
            if (wide && bf16v)
                PM_LAUNCH("k_verify", st, k_verify<true, true><<<vGrid, 32 * vWarps, vsmem, st>>>(va));
            else if (wide)
                PM_LAUNCH("k_verify", st, k_verify<true, false><<<vGrid, 32 * vWarps, vsmem, st>>>(va));
            else
                PM_LAUNCH("k_verify", st, k_verify<false, true><<<vGrid, 32 * vWarps, vsmem, st>>>(va));
        }
        PM_CUDA(cudaGetLastError());
        if (stats) {
            PM_CUDA(cudaMemcpyAsync(stNl, nverD + na, na * sizeof(int), cudaMemcpyDeviceToHost, st));
            PM_CUDA(cudaMemcpyAsync(stNv, nverD, na * sizeof(int), cudaMemcpyDeviceToHost, st));
            PM_CUDA(cudaMemcpyAsync(stFp, fpc, na * sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        PM_CUDA(cudaMemcpyAsync(stDk, dk, na * sizeof(double), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaMemcpyAsync(stErr, errFlag, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (bf16v) PM_CUDA(cudaMemcpyAsync(stRedo, redoD, na * sizeof(int), cudaMemcpyDeviceToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
        const double *dkH = stDk;
        const int errH = *stErr;
        if (errH) {
            int dbgH[3] = {0, 0, 0};
            cudaMemcpy(dbgH, nverD + 2 * na + 1, sizeof(dbgH), cudaMemcpyDeviceToHost);
            pm_set_error("internal error flags %d (index check %d value %d query %d); flags 2, 4, 8, 16, 32, "
                         "64: more points tied within one FP32 error band than an internal capacity; 128: a "
                         "staged copy timed out; 256/512: layout capacity", errH, dbgH[0], dbgH[1], dbgH[2]);
            return PMLSH_EINTERNAL;
        }
        // stop rules (Algorithm 2, with the readings of pmlsh.h)
        bool changed = false;
        for (int a = 0; a < na; a++) {
            const int q = actH[a];
            rounds[q]++;
            const bool budget = count[a] >= B;
            if (stats) {
                fp64[q] += stFp[a];
                nver[q] += stNv[a];
                nleaf[q] += stNl[a];
                if (bf16v) fallback[q] += stRedo[a];
            }
            if (rcbc) {
                // Algorithm 1: the nearest candidate if |C| >= beta n + 1 or it
                // lies within c r, else nothing
                done[q] = 1;
                ncand[q] = count[a];
                rule[q] = budget ? 2 : (dkH[a] <= o->c * r[q] ? 1 : 0);
                continue;
            }
            if (budget) { done[q] = 1; rule[q] = 2; ncand[q] = B; continue; }
            ncand[q] = count[a];
            if (count[a] == n) { done[q] = 1; rule[q] = 3; continue; }
            if (o->stop_rule == PMLSH_STOP_BC_CONSISTENT) {
                if (dkH[a] <= o->c * r[q]) { done[q] = 1; rule[q] = 1; continue; }
                r[q] = o->c * r[q];
            } else {
                r[q] = o->c * r[q];
                // dk is finite only when C holds at least k points
                if (dkH[a] <= o->c * r[q]) { done[q] = 1; rule[q] = 1; continue; }
            }
            changed = true;
        }
        if (changed) {
            std::memcpy(stR, r.data(), nq * sizeof(double));
            PM_CUDA(cudaMemcpyAsync(rq, stR, nq * sizeof(double), cudaMemcpyHostToDevice, st));
        }
        if (round == 99999) {
            pm_set_error("Algorithm 2 did not stop within 100000 rounds");
            return PMLSH_EINTERNAL;
        }
    }
    if (rcbc) {
        // queries whose answer is "nothing": -1 / +inf
        std::vector<int32_t> none;
        for (int64_t q = 0; q < nq; q++)
            if (rule[q] == 0) none.push_back((int32_t)q);
        if (!none.empty()) {
            int32_t *noneD = grow<int32_t>(w.keys, none.size(), s);
            if (s != PMLSH_OK) return s;
            PM_CUDA(cudaMemcpyAsync(noneD, none.data(), none.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            PM_LAUNCH("k_clear_results", st, k_clear_results<<<(unsigned)((none.size() + 255) / 256), 256, 0, st>>>(
                                                  noneD, (int)none.size(), k, oIds, oD, oE));
        }
    }
    // results held in scratch (host arrays of the caller)
    if (!idev) PM_CUDA(cudaMemcpyAsync(ids, oIds, (size_t)nq * k * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (!ddev) PM_CUDA(cudaMemcpyAsync(dists, oD, (size_t)nq * k * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (err && !edev) PM_CUDA(cudaMemcpyAsync(err, oE, (size_t)nq * k * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats) {
        std::vector<pmlsh_query_stats> sv(nq);
        for (int64_t q = 0; q < nq; q++) {
            sv[q].rounds = rounds[q];
            sv[q].stop_rule = rule[q];
            sv[q].n_cand = ncand[q];
            sv[q].r_final = r[q];
            sv[q].fp64_checks = fp64[q];
            sv[q].leaves_visited = nleaf[q];
            sv[q].n_verified = nver[q];
            sv[q].first_pass_fallbacks = fallback[q];
        }
        PM_CUDA(cudaMemcpyAsync(stats, sv.data(), nq * sizeof(pmlsh_query_stats),
                                pm_is_device_ptr(stats) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
        PM_CUDA(cudaStreamSynchronize(st));
    }
    if (!idev || !ddev || (err && !edev)) PM_CUDA(cudaStreamSynchronize(st));
    return PMLSH_OK;
}

