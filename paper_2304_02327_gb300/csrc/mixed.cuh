// Device helpers of the mixed-precision (TF32x3) form.
//
// On GB300 the FP64 pipe issues ~2 operations per clock per SM against 128 for
// FP32, so one FP64 operation per element of a 32.8M-element state costs as much
// as the whole tensor-core contraction of a mode.  The mixed form therefore
// touches the FP64 pipe only for the state update u + tau*y; conversions between
// FP64 and FP32 are done exactly with integer bit manipulation, and everything
// else (K u, g, the split into TF32 parts, partial-sum combination) runs in FP32.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace mm {
namespace mx {

// Exact widening FP32 -> FP64 by bit manipulation (FP32 subnormals flush to 0), on
// the two 32-bit words with selects (no branch): the exponent rebased by 896 (0x7ff
// for inf / nan), the 23 mantissa bits shifted up by 29 across the two words.
__device__ __forceinline__ double f2d(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t m = b & 0x7fffffu;
    const uint32_t eh = e == 0xffu ? 0x7ffu : e + 896u;
    const uint32_t hi = (b & 0x80000000u) | (e == 0 ? 0u : (eh << 20) | (m >> 3));
    const uint32_t lo = e == 0 ? 0u : m << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// x ~ hi + lo with hi = x truncated to 24 significant bits and lo = the next 23
// bits (|x - hi - lo| <= 2^-46 |x|), from the bits of x, without FP64 arithmetic.
// |x| < 2^-103 gives lo = 0; |x| < 2^-126 gives hi = lo = 0; inf/nan map to inf/nan.
__device__ __forceinline__ void d2ff_general(double x, float& hi, float& lo) {
    // branch-free: every case is computed and the right one selected, so a warp never
    // diverges on the exponent
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t s = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const uint64_t m = b & 0xfffffffffffffull;
    const int ef = e - 896;                     // FP32 exponent field of x
    const uint32_t hn = s | ((uint32_t)ef << 23) | (uint32_t)(m >> 29);
    // overflow -> inf; nan stays nan
    const uint32_t hs = s | 0x7f800000u | ((e == 0x7ff && m) ? 0x400000u : 0u);
    hi = __uint_as_float(ef <= 0 ? s : (ef >= 255 ? hs : hn));
    // remainder = (m mod 2^29) * 2^(e-1075); its top 23 bits as P - Q with
    // Q = 2^(ef-23-127), P = Q (1 + r/2^23): exact by Sterbenz.  Below FP32's
    // normal range (ef < 24) and for inf / nan the low part is 0.
    const uint32_t r = (uint32_t)((m & 0x1fffffffull) >> 6);
    const uint32_t E0 = (uint32_t)(ef - 23) & 0xffu;
    const float P = __uint_as_float((E0 << 23) | r);
    const float Q = __uint_as_float(E0 << 23);
    lo = __uint_as_float((ef >= 24 && ef < 255) ? (__float_as_uint(P - Q) | s) : 0u);
}

// The same split with a short path for the values the state holds in practice
// (2^-103 <= |x| < 2^128, where both parts are FP32 normals, and zero), bit for bit
// the general split's result there: hi is the sign and the exponent rebased by
// 896 with the top 23 mantissa bits shifted in (one funnel shift), lo is P - Q as
// above with P's exponent taken from hi.  Anything else takes d2ff_general.
__device__ __forceinline__ void d2ff(double x, float& hi, float& lo) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
    const uint32_t e = (h >> 20) & 0x7ffu;
    const uint32_t sg = h & 0x80000000u;
    const bool zero = ((h & 0x7fffffffu) | l) == 0u;
    if (e - 920u <= 230u || zero) {
        const uint32_t hb = __funnelshift_l(l, h - (896u << 20), 3) | sg;
        const uint32_t qb = (hb & 0x7f800000u) - (23u << 23);
        const float P = __uint_as_float(qb | ((l >> 6) & 0x7fffffu));
        const float Q = __uint_as_float(qb);
        hi = __uint_as_float(zero ? sg : hb);
        lo = __uint_as_float(zero ? 0u : (__float_as_uint(P - Q) | sg));
    } else {
        d2ff_general(x, hi, lo);
    }
}

// Round-to-nearest (ties away) FP32 -> TF32, kept in an FP32 container.
__device__ __forceinline__ float tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// x = hi + lo with hi, lo TF32 (|x - hi - lo| <= 2^-22 |x|).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = tf32(x);
    lo = tf32(x - hi);
}
__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
    float a, b;
    d2ff(x, a, b);
    hi = tf32(a);
    lo = tf32((a - hi) + b);
}

// Pointwise g in FP32 at (t, u): cubic or the manufactured ADR term.
__device__ __forceinline__ float g32(const PointwiseG& g, float u, float t, int64_t idx) {
    if (g.kind == MM_G_CUBIC) {
        return fmaf(fmaf(fmaf(g.f3, u, g.f2), u, g.f1), u, g.f0);
    } else if (g.kind == MM_G_ADR_MANUFACTURED) {
        const float et = __expf(t);
        float ah, al, bh, bl;
        d2ff(g.psi_a[idx], ah, al);
        d2ff(g.psi_b[idx], bh, bl);
        return 1.f / (1.f + u * u) + et * ah - 1.f / (1.f + et * et * bh * bh);
    }
    return 0.f;
}

// g(t1, u + delta) - g(t0, u) in FP32 with relative accuracy in the difference
// itself: for the cubic c0 + c1 u + c2 u^2 + c3 u^3 the difference is written as
// delta (c1 + c2 (2u + delta) + c3 (3u^2 + 3u delta + delta^2)), with no
// cancellation between two nearby values of g.
__device__ __forceinline__ float dg32(const PointwiseG& g, float u, float delta, float t0, float t1,
                                      int64_t idx) {
    if (g.kind == MM_G_CUBIC) {
        const float q = fmaf(3.f * u, u + delta, delta * delta);
        return delta * fmaf(g.f3, q, fmaf(g.f2, 2.f * u + delta, g.f1));
    } else if (g.kind == MM_G_ADR_MANUFACTURED) {
        return g32(g, u + delta, t1, idx) - g32(g, u, t0, idx);
    }
    return 0.f;
}

// Finite test of a double from its exponent bits (no FP64 pipe).
__device__ __forceinline__ bool finite_bits(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

}  // namespace mx
}  // namespace mm
