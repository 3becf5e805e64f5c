// The two split-precision forms of the mixed path and the operand layout they share.
//
// An operand of mode mu is stored already split into parts, each part an array of
// rows ("fibres") of n_mu values at a row pitch p_mu (p_mu * element size a
// multiple of 16 bytes, so a TMA map can address the rows); element (j, row) of
// part q sits at q * part_pitch + row * p_mu + j.
//   TF32x3: two TF32 parts (4-byte containers), x = a0 + a1, residual <= 2^-22 |x|
//   BF16x3: three BF16 parts, x = a0 + a1 + a2, residual ~2^-25 |x|
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "mixed.cuh"

namespace mm {

// kBK: values of one pipeline stage along K (one 128-byte swizzle row: four MMAs).
struct FormTF32 {
    static constexpr int kElem = 4, kBK = 32, kAParts = 2;
    static constexpr int kCorr = 3;   // a1 b0, a0 b1, a0 b2
    __host__ __device__ static constexpr int corr_a(int c) { return c == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int corr_b(int c) { return c == 0 ? 0 : c; }
};
struct FormBF16 {
    static constexpr int kElem = 2, kBK = 64, kAParts = 3;
    static constexpr int kCorr = 5;   // a1 b0, a0 b1, a2 b0, a1 b1, a0 b2
    __host__ __device__ static constexpr int corr_a(int c) { return c == 0 ? 1 : c == 2 ? 2 : c == 3 ? 1 : 0; }
    __host__ __device__ static constexpr int corr_b(int c) { return c == 1 ? 1 : c == 3 ? 1 : c == 4 ? 2 : 0; }
};

// Split x (+ a lower-order correction xl, e.g. the low half of a double) into the
// form's parts, as 32-bit patterns (TF32 in an FP32 container) or 16-bit patterns
// (BF16, low half), each rounded to nearest in turn.
template <class F> __device__ __forceinline__ void split_parts(float x, float xl, uint32_t (&p)[3]);
template <> __device__ __forceinline__ void split_parts<FormTF32>(float x, float xl, uint32_t (&p)[3]) {
    const float h = mx::tf32(x);
    const float l = mx::tf32((x - h) + xl);
    p[0] = __float_as_uint(h); p[1] = __float_as_uint(l); p[2] = 0;
}
template <> __device__ __forceinline__ void split_parts<FormBF16>(float x, float xl, uint32_t (&p)[3]) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
    const float r1 = (x - __bfloat162float(b0)) + xl;
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    p[0] = __bfloat16_as_ushort(b0); p[1] = __bfloat16_as_ushort(b1); p[2] = __bfloat16_as_ushort(b2);
}

// Write the parts of value (x + xl) at element position pos of a part array.
template <class F>
__device__ __forceinline__ void store_parts(uint8_t* base, int64_t part_pitch, int64_t pos, float x, float xl) {
    uint32_t pp[3];
    split_parts<F>(x, xl, pp);
#pragma unroll
    for (int q = 0; q < F::kAParts; ++q) {
        if (F::kElem == 4) ((uint32_t*)base)[q * part_pitch + pos] = pp[q];
        else ((uint16_t*)base)[q * part_pitch + pos] = (uint16_t)pp[q];
    }
}

// Three parts of (x + xl) in both forms (the operand that every product multiplies
// with all of the other side's parts: a phi matrix, a remainder of A, the state as
// the matrix side of a Riccati product).  The first kAParts parts equal those of
// split_parts, so one three-part array also serves as a kAParts-part operand.
template <class F> __device__ __forceinline__ void split_parts3(float x, float xl, uint32_t (&p)[3]);
template <> __device__ __forceinline__ void split_parts3<FormTF32>(float x, float xl, uint32_t (&p)[3]) {
    const float h = mx::tf32(x);
    const float r = (x - h) + xl;
    const float l = mx::tf32(r);
    p[0] = __float_as_uint(h); p[1] = __float_as_uint(l); p[2] = __float_as_uint(mx::tf32(r - l));
}
template <> __device__ __forceinline__ void split_parts3<FormBF16>(float x, float xl, uint32_t (&p)[3]) {
    split_parts<FormBF16>(x, xl, p);
}

// Runtime dispatch on the plan's precision for elementwise writers.
__device__ __forceinline__ void store_parts_prec(int prec, uint8_t* base, int64_t part_pitch, int64_t pos,
                                                 float x, float xl) {
    if (prec == MM_BF16X3) store_parts<FormBF16>(base, part_pitch, pos, x, xl);
    else store_parts<FormTF32>(base, part_pitch, pos, x, xl);
}

}  // namespace mm
