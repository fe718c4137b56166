// Grouped verification: the verification step of Algorithm 2 (exact
// distances of the candidates, top-k, the k-th distance for stop rule 1)
// for groups of up to eight queries that are neighbours in the locality
// order, so that they share most of the points they have to verify.
//
// One CTA per group, one warp per query.  Every warp keeps its own state as
// the single-query kernel does (its query row, the thresholds of its round,
// its top-KP of FP32 squared distances and the pruning bound that follows
// from it, its guard set and FP64 ranking), so its result is the exact k
// nearest of its own candidate set.  What the warps share is the walk:
//   1. the union of the group's candidate leaves (the leaf bit sets of
//      k_class), each with the mask of the group's queries that list it and
//      the smallest lower bound over them (the cheap principal-direction
//      bound of the single-query kernel);
//   2. the union in ascending order of that group minimum, in windows of
//      256 leaves (radix select of the window's bound, bitonic sort), until
//      the group minimum of the next leaf is pruned for every warp (each
//      warp's own bound is at least the group minimum, so every later leaf
//      is pruned for it too);
//   3. the window in batches of up to 32 leaves: the batch's leaf centres
//      are copied into shared memory (one bulk copy each) and every warp
//      tightens its own bound for each leaf of the batch at once, one leaf
//      per lane (cheap bound, original-space leaf ball, Eq. 5 class); the
//      rows of every leaf some warp still needs are then streamed through
//      shared memory (rows and projected coordinates, bulk copies completing
//      on an mbarrier, two buffers so that the next tile is in flight while
//      the current one is used), and each needing warp computes its
//      candidates' distances from there.
// A row is therefore read from L2/HBM once per group instead of once per
// query, and the latency of the bound steps is paid once per batch.
// Pruning is exact per warp (the guard-set rule of k_verify), so the results
// do not depend on the grouping.
#include <climits>

#include "knn_shared.cuh"

namespace pmk {

namespace {

constexpr int GV_THREADS = 32 * GV_WARPS;
constexpr int GV_WIN = 256;                 // leaves per sorted window
constexpr uint32_t GV_TAKEN = 0xFFFFFFFFu;  // key of a leaf already windowed
constexpr int GV_CTL = 8192;                // control region of shared memory

// Total order of FP32 values as unsigned keys (finite and infinite values).
__device__ __forceinline__ uint32_t f2key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__host__ __device__ __forceinline__ size_t gv_slot_bytes(int ld, int KP)
{
    // gd[KP] f64, gid[KP] i64, q[ld], vals[KP], idxs[KP], gpos[KP], q'[16],
    // pivot distances[8], P q[PM_PCA]
    const size_t b = (size_t)KP * 28 + (size_t)ld * 4 + 96 + PM_PCA * 4;
    return (b + 15) & ~(size_t)15;
}
// Leaves per batch of the walk: their centres fill about 16 KB.
__host__ __device__ __forceinline__ int gv_batch_leaves(int ld)
{
    return max(1, min(32, 4096 / ld));
}
__host__ __device__ __forceinline__ size_t gv_stage_bytes(int ld, int TR)
{
    return ((size_t)TR * ld * 4 + (size_t)TR * PM_MP * 4 + 127) & ~(size_t)127;
}

// Exclusive prefix sum over the CTA's 256 threads (tmp: 8 ints of shared
// memory); *total receives the sum.
__device__ __forceinline__ int cta_excl_scan(int v, int *tmp, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(VW_FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) tmp[w] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int i = 0; i < GV_WARPS; i++) {
        const int t = tmp[i];
        before += i < w ? t : 0;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// The want-th smallest (1-based) of the keys != GV_TAKEN in keys[0, U), by
// four 8-bit histogram passes (want must not exceed their number).
__device__ uint32_t cta_select(const uint32_t *keys, int U, int want, uint32_t *hist, int *ctl)
{
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t prefix = 0, pmask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        hist[tid] = 0u;
        __syncthreads();
        for (int e = tid; e < U; e += GV_THREADS) {
            const uint32_t k = keys[e];
            if (k != GV_TAKEN && (k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
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
            if (lane == fl) {
                uint32_t rem = (uint32_t)want - (incl - sum);
                int j = 0;
                while (j < 7 && rem > h[j]) {
                    rem -= h[j];
                    j++;
                }
                ctl[4] = lane * 8 + j;
                ctl[5] = (int)rem;
            }
        }
        __syncthreads();
        prefix |= (uint32_t)ctl[4] << shift;
        pmask |= 0xFFu << shift;
        want = ctl[5];
    }
    return prefix;
}

// Ascending bitonic sort of GV_WIN (key, index) pairs by the CTA.
__device__ __forceinline__ void cta_sort_win(uint32_t *key, int32_t *idx)
{
    const int i = threadIdx.x;   // GV_WIN == GV_THREADS
    for (int size = 2; size <= GV_WIN; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            const int j = i ^ stride;
            if (j > i) {
                const uint32_t ka = key[i], kb = key[j];
                const int32_t ia = idx[i], ib = idx[j];
                const bool gt = ka > kb || (ka == kb && ia > ib);
                if (gt == ((i & size) == 0)) {
                    key[i] = kb;
                    key[j] = ka;
                    idx[i] = ib;
                    idx[j] = ia;
                }
            }
        }
    __syncthreads();
}

#define GV_CHECK(cond, site, val)                                              \
    (((cond)) ? true                                                           \
              : (atomicCAS(&A.dbg[0], 0, (site)) == 0 ? (A.dbg[1] = (int)(val), A.dbg[2] = a, \
                                                         atomicOr(A.errFlag, 1024), false)    \
                                                      : (atomicOr(A.errFlag, 1024), false)))

__global__ void __launch_bounds__(GV_THREADS, 2)
k_verify_grouped(GvArgs A)
{
    extern __shared__ __align__(128) unsigned char gsm[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int ld = A.ld, KP = A.KP, KPW = A.KP >> 5, k = A.k, s = A.s, nf4 = A.ld >> 2;
    const int64_t L = A.L;
    const int TR = A.TR, LPR = 32 / A.TR, T4 = nf4 / LPR;
    // control region
    uint64_t *bar = (uint64_t *)gsm;                      // [2] tile buffers
    uint64_t *hbar = bar + 2;                             // leaf-centre buffer
    int *ctl = (int *)(gsm + 32);                         // [16]: 0 group, 2/3 gather counts, 4/5 select
    float *sCmax = (float *)(ctl + 16);                   // [8] each warp's pruning value
    uint32_t *sNeedW = (uint32_t *)(sCmax + GV_WARPS);    // [8] leaves of the batch each warp needs
    float *sPsl = (float *)(sNeedW + GV_WARPS);           // [8] slack of each warp's cheap bound
    int *sWalk = (int *)(sPsl + GV_WARPS);                // [8] warp takes part in the walk
    int *sTmp = sWalk + GV_WARPS;                         // [8] scan
    int64_t *sR0 = (int64_t *)(sTmp + GV_WARPS);          // [32] first row of each leaf of the batch
    int *sRn = (int *)(sR0 + 32);                         // [32] its rows
    uint32_t *sHist = (uint32_t *)(sRn + 32);             // [256]
    float *sLb = (float *)(sHist + 256);                  // [8][32] each warp's leaf bounds
    unsigned char *sCl = (unsigned char *)(sLb + GV_WARPS * 32);   // [8][32] each warp's Eq. 5 class
    uint32_t *sWinKey = (uint32_t *)(sCl + GV_WARPS * 32);   // [GV_WIN]
    int32_t *sWinIdx = (int32_t *)(sWinKey + GV_WIN);     // [GV_WIN]
    int32_t *sWinLeaf = sWinIdx + GV_WIN;                 // [GV_WIN]
    int32_t *sWinMask = sWinLeaf + GV_WIN;                // [GV_WIN]
    const size_t stageB = gv_stage_bytes(ld, TR);
    unsigned char *stage = gsm + GV_CTL;
    const int NB = gv_batch_leaves(ld);
    float *head = (float *)(stage + 2 * stageB);          // [NB][ld] leaf centres
    const size_t slotB = gv_slot_bytes(ld, KP);
    unsigned char *slots = stage + 2 * stageB + (size_t)NB * ld * 4;
    auto slot_pq = [&](int v) -> const float * {
        return (const float *)(slots + (size_t)v * slotB + (size_t)KP * 28 + (size_t)ld * 4 + 96);
    };
    // this warp's slot
    unsigned char *wbase = slots + (size_t)w * slotB;
    double *gd = (double *)wbase;
    long long *gid = (long long *)(gd + KP);
    float *qs = (float *)(gid + KP);
    float *vals = qs + ld;
    int *idxs = (int *)(vals + KP);
    int *gpos = idxs + KP;
    float *sq = (float *)(gpos + KP);
    float *sp = sq + PM_MP;
    float *sPq = sp + PM_MAX_PIVOTS;
    const float4 *q4 = (const float4 *)qs;
    uint32_t *ukey = A.ukey + (int64_t)blockIdx.x * L;
    int32_t *uleaf = A.uleaf + (int64_t)blockIdx.x * L;
    uint8_t *umask = A.umask + (int64_t)blockIdx.x * L;

    const double epsv = (double)(ld + 8) * 0x1.0p-24;
    const float lbMulF = __double2float_rd(1.0 - epsv), cutMulF = __double2float_ru(1.0 + 3.0 * epsv);
    const float lbSlack = 1.f - (float)((ld + 8) * 0x1.0p-24) - 1e-6f;
    // pruned for a warp whose KP-th smallest FP32 d^2 is cm (directed
    // rounding: prunes only what the exact test lb^2 (1 - eps_v) >
    // K (1 + 3 eps_v) prunes)
    auto prunedc = [&](float lb, float cm) -> bool {
        return lb > 0.f && __fmul_rd(__fmul_rd(lb, lb), lbMulF) > __fmul_ru(cm, cutMulF);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(hbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0, hph = 0;   // parity of each buffer's next completion
    bool abort = false;

    for (;;) {
        if (tid == 0) ctl[0] = atomicAdd(A.workCtr, 1);
        __syncthreads();
        const int gi = ctl[0];
        if (gi >= A.ngroups) break;
        const int g = A.gOrder[gi];
        const int a0 = g * GV_WARPS;
        const int G = min(GV_WARPS, A.na - a0);
        const bool live = w < G && a0 >= 0;
        int a = live ? a0 + w : 0;
        const int q = live ? A.act[a] : 0;
        Thr T;
        T.R = 0.0;
        T.lo = T.hi = T.lov = -1.f;
        T.pad = 0.f;
        if (live) T = A.thr[a];
        const float lov = T.lov;
        const float Rv = lov > 0.f ? __fsqrt_rn(lov) : -1.f;
        const bool inl = A.inlineBand != 0 && T.pad == 0.f;
        const float Rout = inl ? __fsqrt_rn(T.hi) : Rv;
        const bool walker = live && (Rv > 0.f || inl);
        int nfp = 0;
        if (live) {
            for (int i = lane; i < ld; i += 32) qs[i] = A.Qd[(int64_t)q * ld + i];
            if (lane < PM_MP) sq[lane] = A.qp32[(int64_t)q * PM_MP + lane];
            if (lane < PM_MAX_PIVOTS) sp[lane] = A.qpiv[(int64_t)q * PM_MAX_PIVOTS + lane];
            if (lane < PM_PCA) sPq[lane] = A.qpca[(int64_t)q * PM_PCA + lane];
            for (int e = lane; e < KP; e += 32) {
                vals[e] = INFINITY;
                idxs[e] = 0x7fffffff;
            }
        }
        if (lane == 0) {
            sCmax[w] = INFINITY;
            sWalk[w] = walker ? 1 : 0;
            // slack of the cheap bound (FP32 P q, P mu, difference and sum),
            // rounded generously up
            sPsl[w] = live ? __fmul_ru(1.01f, __fadd_ru(__fmul_ru((float)(4 * (ld + 2)) * 0x1.0p-24f, A.qnx[q]),
                                                         __fmul_ru(0x1.0p-20f, __fadd_ru(A.qnx[q], A.muMax))))
                           : 0.f;
        }
        __syncthreads();
        int walk = 0;
        for (int v = 0; v < GV_WARPS; v++) walk |= sWalk[v] << v;
        // top-KP state (lane owns slots lane, lane + 32, ...)
        float cmax = INFINITY, myMax = INFINITY;
        int cslot = 0, mySlot = lane;
        int seen = 0, leaves = 0;
        auto pruned = [&](float lb) -> bool { return prunedc(lb, cmax); };
        auto offer = [&](bool cand, float v, int pos) {
            unsigned bits = __ballot_sync(VW_FULL, cand && v < cmax);
            while (bits) {
                const int src = __ffs(bits) - 1;
                bits &= bits - 1;
                const float val = __shfl_sync(VW_FULL, v, src);
                const int ps = __shfl_sync(VW_FULL, pos, src);
                if (!(val < cmax)) continue;
                if (lane == (cslot & 31)) {
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

        // 1. union of the walkers' candidate leaves, with masks and the
        // group-minimum cheap bound
        int U = 0;
        if (walk) {
            const int W32 = A.W32;
            const int per = (W32 + GV_THREADS - 1) / GV_THREADS;
            const int w0 = min(W32, tid * per), w1 = min(W32, w0 + per);
            const uint32_t lastMask = (L & 31) ? ((1u << (L & 31)) - 1u) : 0xFFFFFFFFu;
            int cnt = 0;
            for (int i = w0; i < w1; i++) {
                uint32_t u = 0;
                for (int v = 0; v < G; v++)
                    if ((walk >> v) & 1) u |= A.leafBits[(int64_t)(a0 + v) * W32 + i];
                if (i == W32 - 1) u &= lastMask;
                cnt += __popc(u);
            }
            int pos = cta_excl_scan(cnt, sTmp, &U);
            for (int i = w0; i < w1; i++) {
                uint32_t bw[GV_WARPS];
                uint32_t u = 0;
#pragma unroll
                for (int v = 0; v < GV_WARPS; v++) {
                    bw[v] = (v < G && ((walk >> v) & 1)) ? A.leafBits[(int64_t)(a0 + v) * W32 + i] : 0u;
                    u |= bw[v];
                }
                if (i == W32 - 1) u &= lastMask;
                while (u) {
                    const int b = __ffs(u) - 1;
                    u &= u - 1;
                    const int l = i * 32 + b;
                    int mask = 0;
#pragma unroll
                    for (int v = 0; v < GV_WARPS; v++) mask |= (int)((bw[v] >> b) & 1u) << v;
                    const float4 *pm4 = (const float4 *)(A.leafPmu + (int64_t)l * PM_PCA);
                    float pm[PM_PCA];
#pragma unroll
                    for (int r4 = 0; r4 < PM_PCA / 4; r4++) {
                        const float4 t = __ldg(pm4 + r4);
                        pm[4 * r4] = t.x;
                        pm[4 * r4 + 1] = t.y;
                        pm[4 * r4 + 2] = t.z;
                        pm[4 * r4 + 3] = t.w;
                    }
                    const float rx = A.leafRx[l];
                    float gmin = INFINITY;
                    for (int v = 0; v < GV_WARPS; v++) {
                        if (!((mask >> v) & 1)) continue;
                        const float *pq = slot_pq(v);
                        float s2 = 0.f;
#pragma unroll
                        for (int r = 0; r < PM_PCA; r++) {
                            const float d = __fsub_rn(pq[r], pm[r]);
                            s2 = __fmaf_rn(d, d, s2);
                        }
                        const float lbp =
                            __fsub_rn(__fsub_rn(__fmul_rn(__fsqrt_rn(s2), 1.f - 0x1.0p-18f), sPsl[v]), rx);
                        gmin = fminf(gmin, lbp);
                    }
                    uleaf[pos] = l;
                    umask[pos] = (uint8_t)mask;
                    ukey[pos] = f2key(gmin);
                    pos++;
                }
            }
        }
        __syncthreads();

        // 2./3. windows of the union in ascending group minimum
        int remaining = U;
        bool finished = U == 0;
        while (!finished && !abort) {
            const int want = min(GV_WIN, remaining);
            const uint32_t tau = cta_select(ukey, U, want, sHist, ctl);
            if (tid == 0) {
                ctl[2] = 0;
                ctl[3] = 0;
            }
            __syncthreads();
            for (int e = tid; e < U; e += GV_THREADS) {
                const uint32_t kk = ukey[e];
                if (kk < tau) {
                    // fewer than `want` keys lie below the selected one
                    const int p = atomicAdd(&ctl[2], 1);
                    if (p < GV_WIN) {
                        sWinKey[p] = kk;
                        sWinIdx[p] = e;
                        ukey[e] = GV_TAKEN;
                    } else {
                        atomicOr(A.errFlag, 2048);
                    }
                }
            }
            __syncthreads();
            const int nless = min(ctl[2], GV_WIN);
            for (int e = tid; e < U; e += GV_THREADS) {
                const uint32_t kk = ukey[e];
                if (kk == tau) {
                    const int p = nless + atomicAdd(&ctl[3], 1);
                    if (p < GV_WIN) {
                        sWinKey[p] = kk;
                        sWinIdx[p] = e;
                        ukey[e] = GV_TAKEN;
                    }
                }
            }
            __syncthreads();
            const int nwin = min(GV_WIN, nless + ctl[3]);
            remaining -= nwin;
            if (tid >= nwin) {
                sWinKey[tid] = GV_TAKEN;
                sWinIdx[tid] = INT_MAX;
            }
            cta_sort_win(sWinKey, sWinIdx);
            if (tid < nwin) {
                const int e = sWinIdx[tid];
                sWinLeaf[tid] = uleaf[e];
                sWinMask[tid] = umask[e];
            }
            __syncthreads();
            if (nwin == 0) break;
            // batches of up to NB leaves of the window
            for (int i0 = 0; i0 < nwin && !abort && !finished;) {
                // every later leaf's group minimum is at least this one's
                bool unbounded = false;
                {
                    const float g0 = key2f(sWinKey[i0]);
                    bool allp = true;
                    for (int v = 0; v < GV_WARPS; v++)
                        if ((walk >> v) & 1) {
                            if (!prunedc(g0, sCmax[v])) allp = false;
                            if (!(sCmax[v] < INFINITY)) unbounded = true;
                        }
                    if (allp) {
                        finished = true;
                        break;
                    }
                }
                // while some warp has no pruning bound yet (fewer than KP
                // candidates seen), batches of two leaves: a warp without a
                // bound verifies every leaf it lists
                const int nb = min(min(NB, nwin - i0), unbounded ? 2 : NB);
                // this lane's leaf of the batch
                const bool inb = lane < nb;
                const int l = inb ? sWinLeaf[i0 + lane] : 0;
                const int msk = inb ? sWinMask[i0 + lane] : 0;
                const float gmin = inb ? key2f(sWinKey[i0 + lane]) : INFINITY;
                const bool okl = !inb || (l >= 0 && l < L);
                if (!okl) GV_CHECK(false, 11, l);
                if (__syncthreads_or(okl ? 0 : 1)) {
                    abort = true;
                    break;
                }
                // the leaves' original-space centres, one bulk copy each
                if (tid == 0) {
                    fence_async_shared();
                    mbar_expect_tx(hbar, (uint32_t)nb * ld * 4);
                    for (int j = 0; j < nb; j++)
                        bulk_g2s(head + (size_t)j * ld, A.leafMu + (int64_t)sWinLeaf[i0 + j] * ld, ld * 4, hbar);
                }
                // rows of each leaf (warp 0), checked
                if (w == 0 && inb) {
                    const int64_t r0 = A.leafOff[l], r1 = A.leafOff[l + 1];
                    const bool okr = r0 >= 0 && r1 > r0 && r1 <= A.n;
                    if (!okr) GV_CHECK(false, 12, (int)(r1 - r0));
                    sR0[lane] = r0;
                    sRn[lane] = okr ? (int)(r1 - r0 < (1 << 30) ? r1 - r0 : (1 << 30)) : 0;
                }
                // this warp's own bounds, one leaf per lane: the cheap
                // principal-direction bound first
                bool want = inb && ((walk >> w) & 1) && ((msk >> w) & 1) && !pruned(gmin);
                if (want) {
                    const float4 *pm4 = (const float4 *)(A.leafPmu + (int64_t)l * PM_PCA);
                    float s2 = 0.f;
#pragma unroll
                    for (int r4 = 0; r4 < PM_PCA / 4; r4++) {
                        const float4 pmv = __ldg(pm4 + r4);
                        float u = __fsub_rn(sPq[4 * r4], pmv.x);
                        s2 = __fmaf_rn(u, u, s2);
                        u = __fsub_rn(sPq[4 * r4 + 1], pmv.y);
                        s2 = __fmaf_rn(u, u, s2);
                        u = __fsub_rn(sPq[4 * r4 + 2], pmv.z);
                        s2 = __fmaf_rn(u, u, s2);
                        u = __fsub_rn(sPq[4 * r4 + 3], pmv.w);
                        s2 = __fmaf_rn(u, u, s2);
                    }
                    const float lbp =
                        __fsub_rn(__fsub_rn(__fmul_rn(__fsqrt_rn(s2), 1.f - 0x1.0p-18f), sPsl[w]), A.leafRx[l]);
                    want = !pruned(lbp);
                }
                const uint32_t phh = hph;
                const bool okh = __syncthreads_and(mbar_wait_bounded(hbar, phh) ? 1 : 0);
                if (!okh) {
                    if (tid == 0) {
                        // record it and wait (bounded) for the copies in flight
                        atomicOr(A.errFlag, 128);
                        mbar_wait_bounded(hbar, phh);
                    }
                    abort = true;
                    break;
                }
                hph ^= 1u;
                // then the original-space leaf ball ||q - mu_l|| - Rx_l (the
                // centre from shared memory; rotated columns keep the lanes
                // of an 8-lane phase on different banks) and the Eq. 5 class
                float lbf = INFINITY;
                unsigned char cl = CL_OUT;
                if (want) {
                    const float4 *m4 = (const float4 *)(head + (size_t)lane * ld);
                    float acc = 0.f;
                    int f = lane % nf4;
                    for (int t = 0; t < nf4; t++) {
                        const float4 x = m4[f];
                        const float4 qv = q4[f];
                        float u = __fsub_rn(qv.x, x.x);
                        acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(qv.y, x.y);
                        acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(qv.z, x.z);
                        acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(qv.w, x.w);
                        acc = __fmaf_rn(u, u, acc);
                        f = f + 1 == nf4 ? 0 : f + 1;
                    }
                    lbf = __fsub_rn(__fmul_rn(__fsqrt_rn(acc), lbSlack), A.leafRx[l]);
                    if (!pruned(lbf)) cl = leaf_class(sq, sp, s, Rv, Rout, A.meta + (int64_t)l * PM_LEAF_STRIDE);
                }
                const uint32_t needm = __ballot_sync(VW_FULL, want && cl != CL_OUT);
                sLb[w * 32 + lane] = lbf;
                sCl[w * 32 + lane] = cl;
                if (lane == 0) sNeedW[w] = needm;
                leaves += __popc(needm);
                __syncthreads();
                uint32_t uni = 0;
                for (int v = 0; v < GV_WARPS; v++) uni |= sNeedW[v];
                // tiles of the needed leaves: (leaf of the batch, TR rows)
                uint32_t pbits = uni;
                int psub = 0;
                auto issue_next = [&](int buf) -> bool {
                    while (pbits) {
                        const int j = __ffs(pbits) - 1;
                        const int rows = sRn[j];
                        const int nsub = (rows + TR - 1) / TR;
                        if (psub >= nsub) {
                            pbits &= pbits - 1;
                            psub = 0;
                            continue;
                        }
                        const int tr = min(TR, rows - psub * TR);
                        const int64_t p0 = sR0[j] + (int64_t)psub * TR;
                        unsigned char *dst = stage + (size_t)buf * stageB;
                        const uint32_t bx = (uint32_t)tr * ld * 4, bo = (uint32_t)tr * PM_MP * 4;
                        fence_async_shared();
                        mbar_expect_tx(&bar[buf], bx + bo);
                        bulk_g2s(dst, A.X + p0 * ld, bx, &bar[buf]);
                        bulk_g2s(dst + (size_t)TR * ld * 4, A.O32 + p0 * PM_MP, bo, &bar[buf]);
                        psub++;
                        return true;
                    }
                    return false;
                };
                bool pend0 = false, pend1 = false;   // thread 0: copies in flight
                if (tid == 0 && uni) {
                    pend0 = issue_next(0);
                    pend1 = issue_next(1);
                }
                uint32_t cbits = uni;
                int csub = 0, tile = 0;
                while (cbits) {
                    const int j = __ffs(cbits) - 1;
                    const int rows = sRn[j];
                    const int nsub = (rows + TR - 1) / TR;
                    if (csub >= nsub) {
                        cbits &= cbits - 1;
                        csub = 0;
                        continue;
                    }
                    const int buf = tile & 1;
                    const int tr = min(TR, rows - csub * TR);
                    const int64_t p0 = sR0[j] + (int64_t)csub * TR;
                    const uint32_t phw = buf ? ph1 : ph0;
                    // (warp-uniform: the warp's lanes compute together)
                    const bool okw = __all_sync(VW_FULL, mbar_wait_bounded(&bar[buf], phw));
                    if (okw && ((sNeedW[w] >> j) & 1u) && !pruned(sLb[w * 32 + j])) {
                        const unsigned char clj = sCl[w * 32 + j];
                        const float *tX = (const float *)(stage + (size_t)buf * stageB);
                        const float *tO = tX + (size_t)TR * ld;
                        bool cand = false;
                        if (lane < tr) {
                            if (clj == CL_FULL) {
                                cand = true;
                            } else {
                                // pm_pd2_32's arithmetic (the count's decisions)
                                const float4 *o4 = (const float4 *)(tO + lane * PM_MP);
                                float pd = 0.f;
#pragma unroll
                                for (int j4 = 0; j4 < PM_MP / 4; j4++) {
                                    const float4 x = o4[j4];
                                    float t = __fsub_rn(x.x, sq[4 * j4]);
                                    pd = __fmaf_rn(t, t, pd);
                                    t = __fsub_rn(x.y, sq[4 * j4 + 1]);
                                    pd = __fmaf_rn(t, t, pd);
                                    t = __fsub_rn(x.z, sq[4 * j4 + 2]);
                                    pd = __fmaf_rn(t, t, pd);
                                    t = __fsub_rn(x.w, sq[4 * j4 + 3]);
                                    pd = __fmaf_rn(t, t, pd);
                                }
                                cand = pd <= lov;
                                if (!cand && inl && pd <= T.hi) {
                                    // inside the FP32 error band: k_band64's FP64 test
                                    cand = pm_pdist64(A.O64 + (p0 + lane) * PM_MP, A.qp64 + (int64_t)q * PM_MP, A.m) <=
                                           T.R;
                                    nfp++;
                                }
                            }
                        }
                        const uint32_t cbm = __ballot_sync(VW_FULL, cand);
                        if (cbm) {
                            seen += __popc(cbm);
                            const int r = lane / LPR, p = lane % LPR;
                            const bool mine = r < tr && ((cbm >> r) & 1u);
                            float acc = 0.f;
                            if (mine) {
                                // rotated column order: the lanes of one 8-lane
                                // phase read different 16-byte bank groups
                                const float4 *x4 = (const float4 *)(tX + (size_t)r * ld);
                                int jj = r % T4;
                                for (int t = 0; t < T4; t++) {
                                    const int f = p + LPR * jj;
                                    const float4 x = x4[f];
                                    const float4 qv = q4[f];
                                    float u = __fsub_rn(qv.x, x.x);
                                    acc = __fmaf_rn(u, u, acc);
                                    u = __fsub_rn(qv.y, x.y);
                                    acc = __fmaf_rn(u, u, acc);
                                    u = __fsub_rn(qv.z, x.z);
                                    acc = __fmaf_rn(u, u, acc);
                                    u = __fsub_rn(qv.w, x.w);
                                    acc = __fmaf_rn(u, u, acc);
                                    jj = jj + 1 == T4 ? 0 : jj + 1;
                                }
                            }
                            for (int o = 1; o < LPR; o <<= 1) acc = __fadd_rn(acc, __shfl_xor_sync(VW_FULL, acc, o));
                            offer(mine && p == 0, acc, (int)(p0 + r));
                            if (lane == 0) sCmax[w] = cmax;
                        }
                    }
                    // the buffer is free once every warp is past it
                    const int allok = __syncthreads_and(okw ? 1 : 0);
                    if (!allok) {
                        if (tid == 0) {
                            // a wait gave up: record it and wait (bounded)
                            // for the copies still in flight
                            atomicOr(A.errFlag, 128);
                            mbar_wait_bounded(&bar[buf], phw);
                            if (buf ? pend0 : pend1) mbar_wait_bounded(&bar[buf ^ 1], buf ? ph0 : ph1);
                        }
                        abort = true;
                        break;
                    }
                    if (buf) ph1 ^= 1u; else ph0 ^= 1u;
                    if (tid == 0) {
                        const bool more = issue_next(buf);
                        if (buf) pend1 = more; else pend0 = more;
                    }
                    csub++;
                    tile++;
                }
                // the head buffer, sR0/sRn and sNeedW are reused by the next batch
                __syncthreads();
                i0 += nb;
            }
        }
        if (abort) break;

        if (live) {
            // band-in points (FP64-resolved members just inside the radius)
            const int nIn = min(A.inN[a], BCAP);
            for (int e0 = 0; e0 < nIn; e0 += 32) {
                const int e = e0 + lane;
                int pos = e < nIn ? A.inPos[(int64_t)a * BCAP + e] : -1;
                if (e < nIn && !GV_CHECK(pos >= 0 && pos < A.n, 4, pos)) pos = -1;
                const bool cand = pos >= 0;
                const float d2 = warp_d2(q4, cand ? A.X + (int64_t)pos * ld : nullptr, nf4, lane);
                seen += __popc(__ballot_sync(VW_FULL, cand));
                offer(cand, d2, pos);
            }
            __syncwarp();
            // guard set: the k-th smallest (value, position) of the top-KP
            float kth = INFINITY;
            int nfin = 0;
            for (int j = 0; j < KPW; j++) {
                const int e = lane + 32 * j;
                const float v = vals[e];
                const int p = idxs[e];
                int rank = 0;
                for (int f = 0; f < KP; f++) {
                    const float vf = vals[f];
                    rank += (vf < v || (vf == v && idxs[f] < p)) ? 1 : 0;
                }
                if (v < INFINITY && rank == k - 1) kth = v;
                nfin += v < INFINITY ? 1 : 0;
            }
            for (int o = 16; o; o >>= 1) {
                nfin += __shfl_xor_sync(VW_FULL, nfin, o);
                kth = fminf(kth, __shfl_xor_sync(VW_FULL, kth, o));
            }
            const float K32 = nfin >= k ? kth : INFINITY;
            const float thrv = K32 < INFINITY ? (float)((double)K32 * (1.0 + 3.0 * epsv) + 1e-36) : INFINITY;
            // entries dropped from the top-KP are >= its final maximum
            if (lane == 0 && seen > KP && cmax <= thrv) atomicOr(A.errFlag, 16);
            int G2 = 0;
            for (int j = 0; j < KPW; j++) {
                const int e = lane + 32 * j;
                const float v = vals[e];
                const bool in = v <= thrv && v < INFINITY;
                const unsigned m = __ballot_sync(VW_FULL, in);
                if (in) gpos[G2 + __popc(m & ((1u << lane) - 1u))] = idxs[e];
                G2 += __popc(m);
            }
            __syncwarp();
            for (int e = lane; e < G2; e += 32) {
                const int p = gpos[e];
                if (GV_CHECK(p >= 0 && p < A.n, 5, p)) {
                    gd[e] = dist64_widen(A.X + (int64_t)p * ld, qs, A.d);
                    gid[e] = A.perm[p];
                } else {
                    gd[e] = INFINITY;
                    gid[e] = 0x7fffffffffffffffLL;
                }
            }
            __syncwarp();
            // rank by (FP64 distance, id); the k nearest are written in order
            for (int e = lane; e < G2; e += 32) {
                const double dv = gd[e];
                const long long iv = gid[e];
                int rank = 0;
                for (int f = 0; f < G2; f++) rank += (gd[f] < dv || (gd[f] == dv && gid[f] < iv)) ? 1 : 0;
                if (rank < k) {
                    const int64_t o = (int64_t)q * k + rank;
                    const float fv = __double2float_rn(dv);
                    A.outIds[o] = iv;
                    A.outD[o] = fv;
                    A.outErr[o] = (float)fabs((double)fv - dv);
                }
                if (rank == k - 1) A.dk[a] = dv;
            }
            for (int e = G2 + lane; e < k; e += 32) {
                const int64_t o = (int64_t)q * k + e;
                A.outIds[o] = -1;
                A.outD[o] = INFINITY;
                A.outErr[o] = 0.f;
            }
            for (int o = 16; o; o >>= 1) nfp += __shfl_xor_sync(VW_FULL, nfp, o);
            if (lane == 0) {
                if (G2 < k) A.dk[a] = INFINITY;
                atomicAdd(&A.fp64cnt[a], G2 + nfp);
                A.nverOut[a] = seen;
                A.nleafOut[a] = leaves;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int gv_tile_rows(int ld)
{
    if (ld <= 0 || ld % 32 != 0) return 0;
    // about 16 KB of rows per tile, at least 4 rows
    int tr = 32;
    while (tr > 4 && (size_t)tr * ld * 4 > 16384) tr >>= 1;
    return tr;
}

size_t gv_smem_bytes(int ld, int KP, int TR)
{
    return GV_CTL + 2 * gv_stage_bytes(ld, TR) + (size_t)gv_batch_leaves(ld) * ld * 4 +
           GV_WARPS * gv_slot_bytes(ld, KP);
}

pmlsh_status gv_ctas_per_sm(size_t smem, int *out)
{
    PM_TRY(pm_allow_max_dyn_smem((const void *)k_verify_grouped));
    int v = 0;
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_verify_grouped, GV_THREADS, smem));
    *out = v;
    return PMLSH_OK;
}

pmlsh_status gv_launch(const GvArgs &A, int grid, size_t smem, cudaStream_t st)
{
    PM_LAUNCH("k_verify", st, k_verify_grouped<<<grid, GV_THREADS, smem, st>>>(A));
    PM_CUDA(cudaGetLastError());
    return PMLSH_OK;
}

}  // namespace pmk
