// Pointwise prepasses of the integrators (FP64, HBM-bound).
//
//   PRE_KU_G     W = sum_mu U x_mu A_mu + g(t, U)     for tridiagonal A_mu (the
//                centred-difference operators of Section 4.2): K u is formed
//                without assembling K (Section 3.2) as a 3-point stencil per
//                direction, read from the diagonals of A_mu.
//   PRE_G        W = g(t, U)                           (dense A_mu: the mode
//                products then accumulate K u into W)
//   PRE_LAWSON   W = U + a g(t, U);  W2 = U + b g(t, U) (if W2 != NULL)
//
// One CTA walks rows of the fastest index i_1, so loads and stores are
// coalesced and the neighbours along i_2.. i_d come from L1/L2.
#include "common.cuh"
#include "stencil.cuh"
#include "trace.cuh"
#include "forms.cuh"
#include "mixed.cuh"

#include <algorithm>

namespace mm {

namespace {

__global__ void __launch_bounds__(256) prepass_kernel(StencilArgs a) {
    const int64_t rows = a.N / a.n[0];
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        // multi-index of this row in directions 2..d
        int idx[MM_MAX_D];
        int64_t rem = row;
        for (int mu = 1; mu < a.d; ++mu) { idx[mu] = (int)(rem % a.n[mu]); rem /= a.n[mu]; }
        const int64_t base = row * a.n[0];
        for (int i1 = threadIdx.x; i1 < a.n[0]; i1 += blockDim.x) {
            const int64_t off = base + i1;
            const double u = a.U[off];
            const double g = g_point(a.g, u, a.t, off);
            if (a.mode == PRE_KU_G) {
                double acc = g;
                idx[0] = i1;
                for (int mu = 0; mu < a.d; ++mu) {
                    const int i = idx[mu];
                    const int nm = (int)a.n[mu];
                    const double* dg = a.diag3[mu];
                    acc = fma(dg[nm + i], u, acc);
                    if (i > 0) acc = fma(dg[i], a.U[off - a.stride[mu]], acc);
                    if (i + 1 < nm) acc = fma(dg[2 * nm + i], a.U[off + a.stride[mu]], acc);
                }
                a.W[off] = acc;
            } else if (a.mode == PRE_G) {
                a.W[off] = g;
            } else {
                a.W[off] = fma(a.ca, g, u);
                if (a.W2) a.W2[off] = fma(a.cb, g, u);
            }
        }
    }
}

// U -> (hi, lo) FP32 pairs, exact to 2^-46, one conversion per element.
__global__ void __launch_bounds__(256) split_pairs_kernel(const double* __restrict__ U,
                                                           float2* __restrict__ P, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        mx::d2ff(__ldg(U + i), h, l);
        P[i] = make_float2(h, l);
    }
}

// One thread per element (flat index, i_1 fastest); the neighbours' pairs come
// from L1/L2, differences are taken pairwise so they keep their own accuracy.
__global__ void __launch_bounds__(256, 6) prepass_mixed_kernel(StencilArgsMixed a) {
    for (int64_t off = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; off < a.N;
         off += (int64_t)gridDim.x * blockDim.x) {
        float uh, ul;
        if (a.mode == PRE_KU_G) {
            const float2 pu = __ldg(a.Up + off);
            uh = pu.x; ul = pu.y;
        } else {
            mx::d2ff(__ldg(a.U + off), uh, ul);
        }
        const float u = uh + ul;
        const float g = mx::g32(a.g, u, a.t, off);
        if (a.mode == PRE_KU_G) {
            float acc = g;
            const bool small = a.N < (int64_t(1) << 31);
            int64_t rem = off;
            uint32_t rem32 = (uint32_t)off;
            for (int mu = 0; mu < a.d; ++mu) {
                const int nm = (int)a.n[mu];
                int i;
                if (small) { i = (int)(rem32 % (uint32_t)nm); rem32 /= (uint32_t)nm; }
                else { i = (int)(rem % nm); rem /= nm; }
                const float* cf = a.coef[mu];
                acc = fmaf(cf[2 * nm + i], u, acc);
                if (i > 0) {
                    const float2 v = __ldg(a.Up + off - a.stride[mu]);
                    acc = fmaf(cf[i], (v.x - uh) + (v.y - ul), acc);
                }
                if (i + 1 < nm) {
                    const float2 v = __ldg(a.Up + off + a.stride[mu]);
                    acc = fmaf(cf[nm + i], (v.x - uh) + (v.y - ul), acc);
                }
            }
            if (a.yadd) acc += __ldg(a.yadd + off);
            if (a.yadd2) acc += __ldg(a.yadd2 + off);
            if (a.cadd) {
                float ch, cl;
                mx::d2ff(__ldg(a.cadd + off), ch, cl);
                acc += ch + cl;
            }
            const int64_t pos = (off % a.n[0]) + (int64_t)a.p1 * (off / a.n[0]);
            store_parts_prec(a.prec, a.Wp, a.part_pitch, pos, acc, 0.f);
        } else {
            // u + c g as (uh + c g) + ul: the low part of u enters the split exactly
            const int64_t pos = (off % a.n[0]) + (int64_t)a.p1 * (off / a.n[0]);
            store_parts_prec(a.prec, a.Wp, a.part_pitch, pos, fmaf(a.ca, g, uh), ul);
            if (a.W2p) store_parts_prec(a.prec, a.W2p, a.part_pitch, pos, fmaf(a.cb, g, uh), ul);
        }
    }
}

__global__ void stencil_coef_kernel(const double* __restrict__ A, int n, float* coef) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = i > 0 ? A[i + (int64_t)n * (i - 1)] : 0.0;
        const double b = A[i + (int64_t)n * i];
        const double c = i + 1 < n ? A[i + (int64_t)n * (i + 1)] : 0.0;
        coef[i] = (float)a;
        coef[n + i] = (float)c;
        coef[2 * n + i] = (float)((a + b) + c);
    }
}

}  // namespace

int launch_prepass_mixed(const StencilArgsMixed& a0, float2* Up, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((a0.N + 255) / 256, (int64_t)num_sms() * 16);
    StencilArgsMixed a = a0;
    if (a.mode == PRE_KU_G) {
        TraceScope tr(KC_SPLIT, s);
        split_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(a.U, Up, a.N);
        MM_LAUNCH_CHECK();
        a.Up = Up;
    }
    TraceScope tr(KC_PREPASS, s);
    prepass_mixed_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int build_stencil_coef(const double* A, int n, float* coef, cudaStream_t s) {
    stencil_coef_kernel<<<(n + 255) / 256, 256, 0, s>>>(A, n, coef);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int launch_prepass(const StencilArgs& a, cudaStream_t s) {
    const int64_t rows = a.N / a.n[0];
    int64_t grid = rows < 65535LL * 16 ? rows : 65535LL * 16;
    int block = a.n[0] >= 256 ? 256 : (a.n[0] >= 128 ? 128 : (a.n[0] >= 64 ? 64 : 32));
    TraceScope tr(KC_PREPASS, s);
    prepass_kernel<<<(unsigned)grid, block, 0, s>>>(a);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

}  // namespace mm
