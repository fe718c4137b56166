// Device helpers and types shared by the query-path kernels (knn.cu and
// verify_group.cu).  Internal to libpmlsh.
#pragma once

#include "pmlsh_impl.h"

namespace pmk {

constexpr int QB = 64;          // queries per block
constexpr int BCAP = 256;       // band-in entries per query
constexpr int SELBAND = 2048;   // band at the budget cut, per query
constexpr float SLACK = 1e-5f;  // relative slack of the conservative leaf tests

enum : unsigned char { CL_OUT = 0, CL_FULL = 1, CL_PART = 2 };

// Eq. 5 (Sec. 4.2): a leaf can hold a point of B(q', R) only if
// ||q', RO|| <= r + R and, for every pivot p_i,
// ||q', p_i|| - R <= HR[i].max and ||q', p_i|| + R >= HR[i].min.
// CL_OUT: every point certainly has FP32 distance^2 > Rout^2 (out-ball);
// CL_FULL: every point certainly has FP32 distance^2 <= Rin^2;
// otherwise CL_PART.  Slack covers the FP32 rounding of every term.
__device__ __forceinline__ unsigned char leaf_class(const float *q, const float *qpiv, int s,
                                                    float Rin, float Rout, const float *M)
{
    // explicit round-to-nearest intrinsics: never contracted, so every kernel
    // that inlines this test takes the same decision
    const float lo_f = 1.f - SLACK, hi_f = 1.f + SLACK;
    float dc = __fsqrt_rn(pm_pd2_32(q, M));
    float rr = M[16];
    float ro = __fmul_rn(Rout, hi_f);
    if (__fsub_rn(__fmul_rn(dc, lo_f), rr) > ro) return CL_OUT;
    // unrolled over the largest pivot count, so that a register copy of M
    // is indexed by constants
#pragma unroll
    for (int i = 0; i < PM_MAX_PIVOTS; i++) {
        if (i < s) {
            float dq = qpiv[i];
            if (__fsub_rn(__fmul_rn(dq, lo_f), M[32 + i]) > ro) return CL_OUT;
            if (__fsub_rn(M[24 + i], __fmul_rn(dq, hi_f)) > ro) return CL_OUT;
        }
    }
    if (Rin > 0.f && __fadd_rn(__fmul_rn(dc, hi_f), rr) <= __fmul_rn(Rin, lo_f)) return CL_FULL;
    return CL_PART;
}

// |sqrt(FP32 d'^2) - FP64 d'| <= eps: coordinate rounding (2^-24 relative per
// coordinate of o' and q') plus the FP32 sum (<= 9 u relative), doubled.
__device__ __forceinline__ double band_eps(double R, double maxNorm, double qn)
{
    return 0x1.0p-23 * (maxNorm + qn) + 0x1.0p-19 * R + 1e-300;
}

// Per-round thresholds for the active queries.
struct Thr {
    double R;      // t r (FP64, as in the oracle)
    float lo, hi;  // FP32 d'^2 <= lo: surely in; > hi: surely out
    float lov;     // verification threshold (lo, or the budget cut)
    float pad;     // 1: the budget selection listed this query's band-in points
};

// ------------------------------------------------- best-first verification

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// TMA (bulk-copy engine): global -> shared, completion counted in bytes on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Waits for phase `ph` of `bar` with an iteration limit; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t ph)
{
    for (int it = 0; it < (1 << 22); it++)
        if (mbar_try_wait(bar, ph)) return true;
    return false;
}

constexpr unsigned VW_FULL = 0xffffffffu;

// Squared FP32 distances ||q - x_v||^2 of up to 32 rows x_v, one per lane
// (`p`: the lane's row, nullptr: none; the lane then gets 0).  Eight lanes
// share a row and read its float4 columns g, g + 8, ..., so that every load
// instruction of the warp covers whole 128-byte lines of four rows; the
// eight partial sums are added by a butterfly.  Requires ld % 32 == 0 with
// zero padding columns in q and in the rows.
// Prefetch hint for the line holding global address p (no fault, no result).
__device__ __forceinline__ void pm_prefetch_l2(const void *p)
{
    asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tprefetch.global.L2 [ga];\n\t}" ::"l"(p));
}

__device__ __forceinline__ float warp_d2(const float4 *__restrict__ q4, const float *p, int nf4, int lane)
{
    const int grp = lane >> 3, g = lane & 7;
    float keep = 0.f;
    // the loop below reads the 32 rows 4 at a time; an L2 prefetch of every
    // line of the lane's own row first puts all 32 rows' misses in flight at
    // once, so later groups find their lines in L2
    if (p != nullptr) {
        const char *pc = (const char *)p;
        for (int b = 0; b < nf4 * 16; b += 128) pm_prefetch_l2(pc + b);
    }
#pragma unroll 1
    for (int j = 0; j < 8; j++) {
        const float4 *x4 = (const float4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 4 * j);
        float acc = 0.f;
        if (x4 != nullptr) {
            for (int t = g; t < nf4; t += 8) {
                const float4 x = __ldg(x4 + t);
                const float4 qv = q4[t];
                float u = __fsub_rn(qv.x, x.x);
                acc = __fmaf_rn(u, u, acc);
                u = __fsub_rn(qv.y, x.y);
                acc = __fmaf_rn(u, u, acc);
                u = __fsub_rn(qv.z, x.z);
                acc = __fmaf_rn(u, u, acc);
                u = __fsub_rn(qv.w, x.w);
                acc = __fmaf_rn(u, u, acc);
            }
        }
        acc = __fadd_rn(acc, __shfl_xor_sync(VW_FULL, acc, 1));
        acc = __fadd_rn(acc, __shfl_xor_sync(VW_FULL, acc, 2));
        acc = __fadd_rn(acc, __shfl_xor_sync(VW_FULL, acc, 4));
        if (g == j) keep = acc;
    }
    // lane (grp, g) holds row grp + 4 g
    return __shfl_sync(VW_FULL, keep, ((lane & 3) << 3) | (lane >> 2));
}

// Two FP32 values as one 64-bit operand of the packed (f32x2) arithmetic.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi)
{
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// acc += (q - x)^2 for two coordinates at once: each half is a separate
// round-to-nearest subtraction and fused multiply-add (the scalar
// __fsub_rn / __fmaf_rn of that coordinate).
__device__ __forceinline__ void f32x2_sqdiff_acc(unsigned long long &acc, unsigned long long q,
                                                 unsigned long long x)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(q), "l"(x));
    asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(d));
}

// warp_d2 with packed arithmetic: each lane keeps two partial sums (even
// and odd coordinates) and adds them before the butterfly, a different
// order of the same ld non-negative terms (the verification's error bound
// (ld + 8) 2^-24 covers any order).
__device__ __forceinline__ float warp_d2x2(const float4 *__restrict__ q4, const float *p, int nf4, int lane)
{
    const int grp = lane >> 3, g = lane & 7;
    float keep = 0.f;
    if (p != nullptr) {
        const char *pc = (const char *)p;
        for (int b = 0; b < nf4 * 16; b += 128) pm_prefetch_l2(pc + b);
    }
#pragma unroll 1
    for (int j = 0; j < 8; j++) {
        const float4 *x4 = (const float4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 4 * j);
        unsigned long long acc = 0ull;
        if (x4 != nullptr) {
            for (int t = g; t < nf4; t += 8) {
                const float4 x = __ldg(x4 + t);
                const float4 qv = q4[t];
                f32x2_sqdiff_acc(acc, f32x2_pack(qv.x, qv.y), f32x2_pack(x.x, x.y));
                f32x2_sqdiff_acc(acc, f32x2_pack(qv.z, qv.w), f32x2_pack(x.z, x.w));
            }
        }
        float a = __fadd_rn(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 1));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 2));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 4));
        if (g == j) keep = a;
    }
    // lane (grp, g) holds row grp + 4 g
    return __shfl_sync(VW_FULL, keep, ((lane & 3) << 3) | (lane >> 2));
}

// warp_d2x2 with four lanes per row: eight rows per round and four rounds,
// each lane's loads of a round issued together (nf4 / 4 float4 per lane), so
// that half as many dependent load rounds stand between the rows and their
// distances; each lane sums its coordinates in two packed partial sums, the
// four lanes of a row are added by a butterfly.  Requires nf4 % 4 == 0.
__device__ __forceinline__ float warp_d2x4(const float4 *__restrict__ q4, const float *p, int nf4, int lane)
{
    const int grp = lane >> 2, g = lane & 3;
    float keep = 0.f;
#pragma unroll 1
    for (int j = 0; j < 4; j++) {
        const float4 *x4 = (const float4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 8 * j);
        unsigned long long acc = 0ull;
        if (x4 != nullptr) {
            int t = g;
            for (; t + 28 < nf4; t += 32) {
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; u++) x[u] = __ldg(x4 + t + 4 * u);
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float4 qv = q4[t + 4 * u];
                    f32x2_sqdiff_acc(acc, f32x2_pack(qv.x, qv.y), f32x2_pack(x[u].x, x[u].y));
                    f32x2_sqdiff_acc(acc, f32x2_pack(qv.z, qv.w), f32x2_pack(x[u].z, x[u].w));
                }
            }
            for (; t < nf4; t += 4) {
                const float4 x = __ldg(x4 + t);
                const float4 qv = q4[t];
                f32x2_sqdiff_acc(acc, f32x2_pack(qv.x, qv.y), f32x2_pack(x.x, x.y));
                f32x2_sqdiff_acc(acc, f32x2_pack(qv.z, qv.w), f32x2_pack(x.z, x.w));
            }
        }
        float a = __fadd_rn(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 1));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 2));
        if (g == j) keep = a;
    }
    // lane (grp, g) holds row grp + 8 g; row v sits at lane 4 (v % 8) + v / 8
    return __shfl_sync(VW_FULL, keep, ((lane & 7) << 2) | (lane >> 3));
}

// warp_d2x4 with two of its eight-row groups in flight at once (for kernels
// with registers to spare): sixteen 16-byte loads per lane are issued
// together, halving the dependent load rounds again; the same sums per row.
__device__ __forceinline__ float warp_d2x4w(const float4 *__restrict__ q4, const float *p, int nf4, int lane)
{
    const int grp = lane >> 2, g = lane & 3;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float keep = 0.f;
#pragma unroll 1
    for (int j = 0; j < 4; j += 2) {
        const float4 *xa = (const float4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 8 * j);
        const float4 *xb = (const float4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 8 * (j + 1));
        unsigned long long accA = 0ull, accB = 0ull;
        if (xa != nullptr || xb != nullptr) {
            int t = g;
            for (; t + 28 < nf4; t += 32) {
                float4 a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    a[u] = xa != nullptr ? __ldg(xa + t + 4 * u) : zero;
                    b[u] = xb != nullptr ? __ldg(xb + t + 4 * u) : zero;
                }
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float4 qv = q4[t + 4 * u];
                    const unsigned long long q0 = f32x2_pack(qv.x, qv.y), q1 = f32x2_pack(qv.z, qv.w);
                    f32x2_sqdiff_acc(accA, q0, f32x2_pack(a[u].x, a[u].y));
                    f32x2_sqdiff_acc(accA, q1, f32x2_pack(a[u].z, a[u].w));
                    f32x2_sqdiff_acc(accB, q0, f32x2_pack(b[u].x, b[u].y));
                    f32x2_sqdiff_acc(accB, q1, f32x2_pack(b[u].z, b[u].w));
                }
            }
            for (; t < nf4; t += 4) {
                const float4 a = xa != nullptr ? __ldg(xa + t) : zero;
                const float4 b = xb != nullptr ? __ldg(xb + t) : zero;
                const float4 qv = q4[t];
                const unsigned long long q0 = f32x2_pack(qv.x, qv.y), q1 = f32x2_pack(qv.z, qv.w);
                f32x2_sqdiff_acc(accA, q0, f32x2_pack(a.x, a.y));
                f32x2_sqdiff_acc(accA, q1, f32x2_pack(a.z, a.w));
                f32x2_sqdiff_acc(accB, q0, f32x2_pack(b.x, b.y));
                f32x2_sqdiff_acc(accB, q1, f32x2_pack(b.z, b.w));
            }
        }
        float sa = __fadd_rn(__uint_as_float((unsigned)accA), __uint_as_float((unsigned)(accA >> 32)));
        float sb = __fadd_rn(__uint_as_float((unsigned)accB), __uint_as_float((unsigned)(accB >> 32)));
        sa = __fadd_rn(sa, __shfl_xor_sync(VW_FULL, sa, 1));
        sb = __fadd_rn(sb, __shfl_xor_sync(VW_FULL, sb, 1));
        sa = __fadd_rn(sa, __shfl_xor_sync(VW_FULL, sa, 2));
        sb = __fadd_rn(sb, __shfl_xor_sync(VW_FULL, sb, 2));
        if (g == j) keep = sa;
        if (g == j + 1) keep = sb;
    }
    // lane (grp, g) holds row grp + 8 g; row v sits at lane 4 (v % 8) + v / 8
    return __shfl_sync(VW_FULL, keep, ((lane & 7) << 2) | (lane >> 3));
}

// ||u - r~_v||^2 in FP32 of up to 32 BF16 rows r~_v (one per lane, length
// ld; nullptr: none, the lane then gets 0) against the FP32 vector u in
// shared memory: eight lanes share a row (16-byte loads of 8 BF16 values),
// packed arithmetic over coordinate pairs, the eight partial sums added by a
// butterfly.  Requires ld % 32 == 0 with zero padding in u and the rows.
__device__ __forceinline__ float warp_d2_bf16(const float *__restrict__ us, const uint16_t *p, int ld, int lane)
{
    const int grp = lane >> 3, g = lane & 7, nu4 = ld >> 3;
    const float4 *u4 = (const float4 *)us;
    float keep = 0.f;
    if (p != nullptr) {
        const char *pc = (const char *)p;
        for (int b = 0; b < ld * 2; b += 128) pm_prefetch_l2(pc + b);
    }
#pragma unroll 1
    for (int j = 0; j < 8; j++) {
        const uint4 *x4 = (const uint4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 4 * j);
        unsigned long long acc = 0ull;
        if (x4 != nullptr) {
            for (int t = g; t < nu4; t += 8) {
                const uint4 x = __ldg(x4 + t);
                const float4 ua = u4[2 * t], ub = u4[2 * t + 1];
                // a 32-bit word holds two BF16 values, the lower coordinate
                // in its low half; as FP32: the half moved to the top bits
                f32x2_sqdiff_acc(acc, f32x2_pack(ua.x, ua.y),
                                 ((unsigned long long)(x.x & 0xFFFF0000u) << 32) | (x.x << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ua.z, ua.w),
                                 ((unsigned long long)(x.y & 0xFFFF0000u) << 32) | (x.y << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ub.x, ub.y),
                                 ((unsigned long long)(x.z & 0xFFFF0000u) << 32) | (x.z << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ub.z, ub.w),
                                 ((unsigned long long)(x.w & 0xFFFF0000u) << 32) | (x.w << 16));
            }
        }
        float a = __fadd_rn(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 1));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 2));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 4));
        if (g == j) keep = a;
    }
    return __shfl_sync(VW_FULL, keep, ((lane & 3) << 3) | (lane >> 2));
}

// warp_d2_bf16 with four lanes per row (eight rows per round, four rounds),
// each lane's loads of a round issued together.  Requires ld % 32 == 0.
__device__ __forceinline__ float warp_d2_bf16x4(const float *__restrict__ us, const uint16_t *p, int ld, int lane)
{
    const int grp = lane >> 2, g = lane & 3, nu4 = ld >> 3;
    const float4 *u4 = (const float4 *)us;
    float keep = 0.f;
#pragma unroll 1
    for (int j = 0; j < 4; j++) {
        const uint4 *x4 = (const uint4 *)__shfl_sync(VW_FULL, (unsigned long long)p, grp + 8 * j);
        unsigned long long acc = 0ull;
        if (x4 != nullptr) {
            auto step = [&](const uint4 x, int t) {
                const float4 ua = u4[2 * t], ub = u4[2 * t + 1];
                f32x2_sqdiff_acc(acc, f32x2_pack(ua.x, ua.y),
                                 ((unsigned long long)(x.x & 0xFFFF0000u) << 32) | (x.x << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ua.z, ua.w),
                                 ((unsigned long long)(x.y & 0xFFFF0000u) << 32) | (x.y << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ub.x, ub.y),
                                 ((unsigned long long)(x.z & 0xFFFF0000u) << 32) | (x.z << 16));
                f32x2_sqdiff_acc(acc, f32x2_pack(ub.z, ub.w),
                                 ((unsigned long long)(x.w & 0xFFFF0000u) << 32) | (x.w << 16));
            };
            int t = g;
            for (; t + 12 < nu4; t += 16) {
                uint4 x[4];
#pragma unroll
                for (int u = 0; u < 4; u++) x[u] = __ldg(x4 + t + 4 * u);
#pragma unroll
                for (int u = 0; u < 4; u++) step(x[u], t + 4 * u);
            }
            for (; t < nu4; t += 4) step(__ldg(x4 + t), t);
        }
        float a = __fadd_rn(__uint_as_float((unsigned)acc), __uint_as_float((unsigned)(acc >> 32)));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 1));
        a = __fadd_rn(a, __shfl_xor_sync(VW_FULL, a, 2));
        if (g == j) keep = a;
    }
    return __shfl_sync(VW_FULL, keep, ((lane & 7) << 2) | (lane >> 3));
}

// FP32 -> FP64 re-encoded with integer operations (exact, equal to the
// conversion instruction), so that the widening does not occupy the FP64
// pipe; zeros are re-encoded too, subnormals, infinities and NaNs use the
// conversion instruction.
__device__ __forceinline__ double f2d_exact(float f) { return pm_f2d_exact(f); }

// pm_dist64 (FP64 sequential sum of (x_i - y_i)^2, separate multiply and
// add, correctly rounded sqrt) with the inputs widened by f2d_exact.
__device__ __forceinline__ double dist64_widen(const float *x, const float *y, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; i++) {
        const double t = __dsub_rn(f2d_exact(x[i]), f2d_exact(y[i]));
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return __dsqrt_rn(s);
}

// FP32 d'^2 of one projected row against q' (the arithmetic of pm_pd2_32:
// sequential over the 16 coordinates, row minus query), float4 loads.
__device__ __forceinline__ float pd2_row(const float *__restrict__ o, const float *__restrict__ qv)
{
    const float4 *o4 = (const float4 *)o;
    float s = 0.f;
#pragma unroll
    for (int j4 = 0; j4 < PM_MP / 4; j4++) {
        const float4 x = __ldg(o4 + j4);
        float t = __fsub_rn(x.x, qv[4 * j4]);
        s = __fmaf_rn(t, t, s);
        t = __fsub_rn(x.y, qv[4 * j4 + 1]);
        s = __fmaf_rn(t, t, s);
        t = __fsub_rn(x.z, qv[4 * j4 + 2]);
        s = __fmaf_rn(t, t, s);
        t = __fsub_rn(x.w, qv[4 * j4 + 3]);
        s = __fmaf_rn(t, t, s);
    }
    return s;
}


// --------------------------------------------- grouped verification (host)

// Arguments of the grouped verification kernel (verify_group.cu): the
// per-query inputs and outputs of the single-query kernel k_verify, plus the
// grouping of the active queries and the per-CTA scratch.
struct GvArgs {
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
    const int64_t *leafOff;     // [L+1] leaf l holds positions [leafOff[l], leafOff[l+1])
    int KP, k;
    const int *inN, *inPos;
    const int32_t *perm;
    int64_t *outIds;
    float *outD, *outErr;
    double *dk;
    int *fp64cnt, *nverOut, *nleafOut, *errFlag;
    int *workCtr;               // next entry of gOrder to take (persistent CTAs)
    int *dbg;                   // [3]: site, value, query of the first failed index check
    int64_t n;
    const uint32_t *leafBits;   // [na][W32]: leaves Eq. 5 does not exclude (k_class)
    int W32;
    const double *O64, *qp64;
    const float *leafPmu;       // [L][PM_PCA]
    const float *qpca, *qnx;    // [nq][PM_PCA], [nq]
    float muMax;
    int m;
    int inlineBand;
    const int32_t *gOrder;      // [ngroups] group ids, costliest first
    int ngroups;                // group g = active entries [8 g, min(8 g + 8, na))
    uint32_t *ukey;             // [grid][L] scratch: ordered group-minimum bound
    int32_t *uleaf;             // [grid][L] scratch: leaf id
    uint8_t *umask;             // [grid][L] scratch: queries of the group that list the leaf
    int TR;                     // rows per staged tile (power of two, 4..32)
};

// Queries per group (one warp each) of the grouped verification.
constexpr int GV_WARPS = 8;
// Rows per staged tile for row length ld (0: ld too long for the kernel).
int gv_tile_rows(int ld);
// Dynamic shared memory of one CTA.
size_t gv_smem_bytes(int ld, int KP, int TR);
// Launches the grouped verification on `grid` persistent CTAs.
pmlsh_status gv_launch(const GvArgs &A, int grid, size_t smem, cudaStream_t st);
// CTAs per SM the kernel reaches with this shared memory (>= 1).
pmlsh_status gv_ctas_per_sm(size_t smem, int *out);

}  // namespace pmk
