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
#include "tcgen05.cuh"
#include "tf32.cuh"

#include <algorithm>
#include <type_traits>

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

// K u + g of the mixed prepass for d = 2 and d = 3 in one pass: the state is read
// once and split once into (hi, lo) pairs held in shared memory, the stencil reads
// its neighbours there (same operations, in the same order, as
// prepass_mixed_kernel).  d = 2: one 32 x 32 tile and its halo per step of the
// block loop.  d = 3: a 32 x 32 tile of (i_1, i_2) marches along i_3 through a
// ring of three planes, so every plane is split once per tile.
constexpr int kT1 = 32;

__device__ __forceinline__ float stencil_extras(const StencilArgsMixed& a, float acc, int64_t off) {
    if (a.yadd) acc += __ldg(a.yadd + off);
    if (a.yadd2) acc += __ldg(a.yadd2 + off);
    if (a.cadd) {
        float ch, cl;
        mx::d2ff(__ldg(a.cadd + off), ch, cl);
        acc += ch + cl;
    }
    return acc;
}

__device__ __forceinline__ float stencil_dir(const float* __restrict__ cf, int nm, int i, float u, float uh, float ul,
                                             float2 lo_nb, float2 hi_nb, float acc) {
    acc = fmaf(__ldg(cf + 2 * nm + i), u, acc);
    if (i > 0) acc = fmaf(__ldg(cf + i), (lo_nb.x - uh) + (lo_nb.y - ul), acc);
    if (i + 1 < nm) acc = fmaf(__ldg(cf + nm + i), (hi_nb.x - uh) + (hi_nb.y - ul), acc);
    return acc;
}

__global__ void __launch_bounds__(256) stencil2d_kernel(StencilArgsMixed a) {
    __shared__ float2 sp[kT1 + 2][kT1 + 2];
    const int n1 = (int)a.n[0], n2 = (int)a.n[1];
    const int t1 = (n1 + kT1 - 1) / kT1, t2 = (n2 + kT1 - 1) / kT1;
    for (int T = blockIdx.x; T < t1 * t2; T += gridDim.x) {
        const int a1 = (T % t1) * kT1, a2 = (T / t1) * kT1;
        for (int e = threadIdx.x; e < (kT1 + 2) * (kT1 + 2); e += blockDim.x) {
            const int r = e / (kT1 + 2), c = e % (kT1 + 2);
            const int i1 = a1 - 1 + c, i2 = a2 - 1 + r;
            float2 v = make_float2(0.f, 0.f);
            if (i1 >= 0 && i1 < n1 && i2 >= 0 && i2 < n2) mx::d2ff(__ldg(a.U + i1 + (int64_t)n1 * i2), v.x, v.y);
            sp[r][c] = v;
        }
        __syncthreads();
        const int c = threadIdx.x % kT1;
        const int i1 = a1 + c;
#pragma unroll
        for (int q = 0; q < kT1 / 8; ++q) {
            const int r = threadIdx.x / kT1 + 8 * q;
            const int i2 = a2 + r;
            if (i1 >= n1 || i2 >= n2) continue;
            const float uh = sp[r + 1][c + 1].x, ul = sp[r + 1][c + 1].y;
            const float u = uh + ul;
            const int64_t off = i1 + (int64_t)n1 * i2;
            float acc = mx::g32(a.g, u, a.t, off);
            acc = stencil_dir(a.coef[0], n1, i1, u, uh, ul, sp[r + 1][c], sp[r + 1][c + 2], acc);
            acc = stencil_dir(a.coef[1], n2, i2, u, uh, ul, sp[r][c + 1], sp[r + 2][c + 1], acc);
            acc = stencil_extras(a, acc, off);
            store_parts_prec(a.prec, a.Wp, a.part_pitch, i1 + (int64_t)a.p1 * i2, acc, 0.f);
        }
        __syncthreads();
    }
}

constexpr int kT2 = 32;      // i_2 extent of a 3D tile
constexpr int kZ = 32;       // most planes per block of the 3D march
constexpr int kHalo3 = (kT2 + 2) * (kT1 + 2);      // 1156 values of a plane with its halo
constexpr int kPer3 = (kHalo3 + 255) / 256;         // of them per thread

// The coefficient of the missing neighbour at a grid edge is exactly zero and the
// halo there holds zeros, so the edge terms add exact zeros and need no branch.
__device__ __forceinline__ float stencil_term(float a, float2 nb, float uh, float ul, float acc) {
    return fmaf(a, (nb.x - uh) + (nb.y - ul), acc);
}

// zc planes per block (<= kZ): small grids march in shorter chunks so that every SM
// gets blocks.
__global__ void __launch_bounds__(256, 4) stencil3d_kernel(StencilArgsMixed a, int zc) {
    __shared__ float2 sp[3][kT2 + 2][kT1 + 2];
    const int n1 = (int)a.n[0], n2 = (int)a.n[1], n3 = (int)a.n[2];
    const int t1 = (n1 + kT1 - 1) / kT1, t2 = (n2 + kT2 - 1) / kT2, tz = (n3 + zc - 1) / zc;
    const int64_t plane = (int64_t)n1 * n2;
    const float* cf1 = a.coef[0];
    const float* cf2 = a.coef[1];
    const float* cf3 = a.coef[2];
    const int c = threadIdx.x % kT1;
    for (int T = blockIdx.x; T < t1 * t2 * tz; T += gridDim.x) {
        const int a1 = (T % t1) * kT1, a2 = ((T / t1) % t2) * kT2, z0 = (T / (t1 * t2)) * zc;
        const int z1 = min(n3, z0 + zc);
        // this thread's share of a plane's halo region: offsets, validity
        int64_t goff[kPer3];
        bool gin[kPer3];
#pragma unroll
        for (int k = 0; k < kPer3; ++k) {
            const int e = threadIdx.x + 256 * k;
            const int r = e / (kT1 + 2), cc = e % (kT1 + 2);
            const int i1 = a1 - 1 + cc, i2 = a2 - 1 + r;
            gin[k] = e < kHalo3 && i1 >= 0 && i1 < n1 && i2 >= 0 && i2 < n2;
            goff[k] = gin[k] ? i1 + (int64_t)n1 * i2 : 0;
        }
        double raw[kPer3];
        auto fetch = [&](int z) {           // global loads of plane z, left in flight
#pragma unroll
            for (int k = 0; k < kPer3; ++k)
                raw[k] = (gin[k] && z >= 0 && z < n3) ? __ldg(a.U + goff[k] + plane * z) : 0.0;
        };
        auto deposit = [&](int z) {         // split them into ring slot z mod 3
            float2* dst = &sp[(z + 3) % 3][0][0];
#pragma unroll
            for (int k = 0; k < kPer3; ++k) {
                const int e = threadIdx.x + 256 * k;
                if (e < kHalo3) {
                    float2 v;
                    mx::d2ff(raw[k], v.x, v.y);
                    dst[e] = v;
                }
            }
        };
        fetch(z0 - 1);
        deposit(z0 - 1);
        fetch(z0);
        deposit(z0);
        fetch(z0 + 1);
        // coefficients along i_1 and i_2 are fixed for this thread's outputs
        const int i1 = a1 + c;
        const bool in1 = i1 < n1;
        const float a1a = in1 ? __ldg(cf1 + i1) : 0.f, a1c = in1 ? __ldg(cf1 + n1 + i1) : 0.f,
                    a1s = in1 ? __ldg(cf1 + 2 * n1 + i1) : 0.f;
        float a2a[kT2 / 8], a2c[kT2 / 8], a2s[kT2 / 8];
#pragma unroll
        for (int q = 0; q < kT2 / 8; ++q) {
            const int i2 = a2 + threadIdx.x / kT1 + 8 * q;
            const bool in2 = i2 < n2;
            a2a[q] = in2 ? __ldg(cf2 + i2) : 0.f;
            a2c[q] = in2 ? __ldg(cf2 + n2 + i2) : 0.f;
            a2s[q] = in2 ? __ldg(cf2 + 2 * n2 + i2) : 0.f;
        }
        for (int z = z0; z < z1; ++z) {
            deposit(z + 1);
            fetch(z + 2);                   // in flight during this plane's stencil
            __syncthreads();
            const float2(*pm)[kT1 + 2] = sp[(z + 2) % 3];
            const float2(*p0)[kT1 + 2] = sp[z % 3];
            const float2(*pp)[kT1 + 2] = sp[(z + 1) % 3];
            const float a3a = __ldg(cf3 + z), a3c = __ldg(cf3 + n3 + z), a3s = __ldg(cf3 + 2 * n3 + z);
#pragma unroll
            for (int q = 0; q < kT2 / 8; ++q) {
                const int r = threadIdx.x / kT1 + 8 * q;
                const int i2 = a2 + r;
                if (!in1 || i2 >= n2) continue;
                const float uh = p0[r + 1][c + 1].x, ul = p0[r + 1][c + 1].y;
                const float u = uh + ul;
                const int64_t off = i1 + (int64_t)n1 * i2 + plane * z;
                float acc = mx::g32(a.g, u, a.t, off);
                acc = fmaf(a1s, u, acc);
                acc = stencil_term(a1a, p0[r + 1][c], uh, ul, acc);
                acc = stencil_term(a1c, p0[r + 1][c + 2], uh, ul, acc);
                acc = fmaf(a2s[q], u, acc);
                acc = stencil_term(a2a[q], p0[r][c + 1], uh, ul, acc);
                acc = stencil_term(a2c[q], p0[r + 2][c + 1], uh, ul, acc);
                acc = fmaf(a3s, u, acc);
                acc = stencil_term(a3a, pm[r + 1][c + 1], uh, ul, acc);
                acc = stencil_term(a3c, pp[r + 1][c + 1], uh, ul, acc);
                acc = stencil_extras(a, acc, off);
                store_parts_prec(a.prec, a.Wp, a.part_pitch,
                                 i1 + (int64_t)a.p1 * (i2 + (int64_t)n2 * z), acc, 0.f);
            }
            __syncthreads();
        }
    }
}

// The 3D K u + g prepass fed from registers, taken when the state admits no TMA map
// (odd n_1; the TMA-fed march below is the usual one).  No Riccati or dense terms
// (d = 3 has neither); N < 2^31, so 32-bit offsets.  The same
// arithmetic as stencil3d_kernel: g, the row sums times u and the six differences
// of the double-float split, in FP32, then the form's split of the result.  It
// marches a 32 x 32 tile of (i_1, i_2) along i_3 with two shared-memory planes:
// plane z (with its halo) supplies the in-plane neighbours, the centres of planes
// z - 1 and z + 1 live in registers (the z + 1 centre is read once from the next
// plane's buffer and then rotated), and the next plane's loads are in flight while
// plane z is computed.  Templated on the form and on the manufactured g (which
// needs the element's offset), so no per-element branch on either remains.
constexpr int kRows3 = kT2 / 8;                      // outputs per thread and plane

// Work balance: the (tile, plane) steps, tile-major, are cut into gridDim.x equal
// contiguous ranges, one per block of a grid sized to the resident blocks, so every
// SM marches the same number of planes (a range that crosses a tile boundary
// restarts the march there).
template <class F, bool MANUF>
__global__ void __launch_bounds__(256, 3) stencil3d_reg_kernel(StencilArgsMixed a) {
    __shared__ float2 sp[2][kT2 + 2][kT1 + 2];
    using T = typename std::conditional<F::kElem == 4, uint32_t, uint16_t>::type;
    const int n1 = (int)a.n[0], n2 = (int)a.n[1], n3 = (int)a.n[2];
    const int t1 = (n1 + kT1 - 1) / kT1, t2 = (n2 + kT2 - 1) / kT2;
    const uint32_t plane = (uint32_t)n1 * (uint32_t)n2;
    const uint32_t pplane = (uint32_t)a.p1 * (uint32_t)n2;       // one plane in the mode-1 layout
    const uint32_t pp = (uint32_t)a.part_pitch;
    const float* cf1 = a.coef[0];
    const float* cf2 = a.coef[1];
    const float* cf3 = a.coef[2];
    const int c = threadIdx.x % kT1, ty = threadIdx.x / kT1;
    const int64_t total = (int64_t)t1 * t2 * n3;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t s_end = min(total, (int64_t)(blockIdx.x + 1) * per);
    for (int64_t s0 = (int64_t)blockIdx.x * per; s0 < s_end;) {
        const int T0 = (int)(s0 / n3);
        const int a1 = (T0 % t1) * kT1, a2 = (T0 / t1) * kT2, z0 = (int)(s0 % n3);
        const int z1 = (int)min((int64_t)n3, z0 + (s_end - s0));
        s0 += z1 - z0;
        // this thread's share of a plane's halo region
        uint32_t goff[kPer3];
        bool gin[kPer3];
#pragma unroll
        for (int k = 0; k < kPer3; ++k) {
            const int e = threadIdx.x + 256 * k;
            const int r = e / (kT1 + 2), cc = e % (kT1 + 2);
            const int i1 = a1 - 1 + cc, i2 = a2 - 1 + r;
            gin[k] = e < kHalo3 && i1 >= 0 && i1 < n1 && i2 >= 0 && i2 < n2;
            goff[k] = gin[k] ? (uint32_t)i1 + (uint32_t)n1 * (uint32_t)i2 : 0u;
        }
        double raw[kPer3];
        auto fetch = [&](int z) {           // global loads of plane z, left in flight
            const bool zin = z >= 0 && z < n3;
            const double* Uz = a.U + (zin ? plane * (uint32_t)z : 0u);
#pragma unroll
            for (int k = 0; k < kPer3; ++k) raw[k] = (gin[k] && zin) ? __ldg(Uz + goff[k]) : 0.0;
        };
        auto deposit = [&](int buf) {       // split them into plane buffer buf
            float2* dst = &sp[buf][0][0];
#pragma unroll
            for (int k = 0; k < kPer3; ++k) {
                const int e = threadIdx.x + 256 * k;
                if (e < kHalo3) {
                    float2 v;
                    mx::d2ff(raw[k], v.x, v.y);
                    dst[e] = v;
                }
            }
        };
        // coefficients along i_1 and i_2 are fixed for this thread's outputs
        const int i1 = a1 + c;
        const bool in1 = i1 < n1;
        const float a1a = in1 ? __ldg(cf1 + i1) : 0.f, a1c = in1 ? __ldg(cf1 + n1 + i1) : 0.f;
        const float a1s = in1 ? __ldg(cf1 + 2 * n1 + i1) : 0.f;
        float a2a[kRows3], a2c[kRows3], s12[kRows3];
#pragma unroll
        for (int q = 0; q < kRows3; ++q) {
            const int i2 = a2 + ty + 8 * q;
            const bool in2 = i2 < n2;
            a2a[q] = in2 ? __ldg(cf2 + i2) : 0.f;
            a2c[q] = in2 ? __ldg(cf2 + n2 + i2) : 0.f;
            s12[q] = a1s + (in2 ? __ldg(cf2 + 2 * n2 + i2) : 0.f);
        }
        // centres of planes z - 1 (cm) and z (c0) of this thread's outputs
        float2 cm[kRows3], c0[kRows3];
        fetch(z0 - 1);
        deposit((z0 + 1) & 1);
        fetch(z0);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRows3; ++q) cm[q] = sp[(z0 + 1) & 1][ty + 8 * q + 1][c + 1];
        deposit(z0 & 1);
        fetch(z0 + 1);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRows3; ++q) c0[q] = sp[z0 & 1][ty + 8 * q + 1][c + 1];
        for (int z = z0; z < z1; ++z) {
            const int b = z & 1, bn = b ^ 1;
            deposit(bn);                    // plane z + 1 (its buffer held z - 1, read)
            fetch(z + 2);                   // in flight during this plane's stencil
            __syncthreads();
            const float a3a = __ldg(cf3 + z), a3c = __ldg(cf3 + n3 + z), a3s = __ldg(cf3 + 2 * n3 + z);
            uint32_t pos = (uint32_t)i1 + (uint32_t)a.p1 * (uint32_t)(a2 + ty) + pplane * (uint32_t)z;
#pragma unroll
            for (int q = 0; q < kRows3; ++q, pos += 8u * (uint32_t)a.p1) {
                const int r = ty + 8 * q;
                const float2 cp = sp[bn][r + 1][c + 1];
                const float uh = c0[q].x, ul = c0[q].y;
                const float u = uh + ul;
                if (in1 && a2 + r < n2) {
                    float acc;
                    if (MANUF) {
                        acc = mx::g32(a.g, u, a.t, (int64_t)i1 + (int64_t)n1 * (a2 + r) + (int64_t)plane * z);
                    } else {
                        acc = fmaf(fmaf(fmaf(a.g.f3, u, a.g.f2), u, a.g.f1), u, a.g.f0);
                    }
                    acc = fmaf(s12[q] + a3s, u, acc);
                    acc = stencil_term(a1a, sp[b][r + 1][c], uh, ul, acc);
                    acc = stencil_term(a1c, sp[b][r + 1][c + 2], uh, ul, acc);
                    acc = stencil_term(a2a[q], sp[b][r][c + 1], uh, ul, acc);
                    acc = stencil_term(a2c[q], sp[b][r + 2][c + 1], uh, ul, acc);
                    acc = stencil_term(a3a, cm[q], uh, ul, acc);
                    acc = stencil_term(a3c, cp, uh, ul, acc);
                    uint32_t v[3];
                    split_parts<F>(acc, 0.f, v);
                    T* w = (T*)a.Wp + pos;
                    w[0] = (T)v[0];
                    w[pp] = (T)v[1];
                    if (F::kAParts == 3) w[2 * pp] = (T)v[2];
                }
                cm[q] = c0[q];
                c0[q] = cp;
            }
            __syncthreads();                // before the next deposit overwrites plane z
        }
    }
}

// The same march with the planes brought in by TMA: a ring of kTmaStages raw FP64
// planes (each the 36 x 34 box at (a1 - 2, a2 - 1, z), so that the box starts on a
// 16-byte boundary; rows and planes outside the array read zeros, which is the
// Dirichlet halo), filled up to kTmaStages planes ahead by thread 0, so that many
// loads are in flight per block without holding them in registers.  The arithmetic of
// every output and its order are stencil3d_reg_kernel's, and so is the work balance;
// the work is laid out for fewer instructions per element: each thread owns two
// adjacent columns (i_1 = a1 + 2 cp, + 1; n1 is even on this path) of two rows, so it
// reads its neighbours with 16-byte shared loads and writes two parts per 32-bit
// (BF16) or 64-bit (TF32) store; the split planes keep the raw box's column index
// (column i_1 at i_1 - a1 + 2) and are split two values at a time.  Every wait on a
// plane is bounded: on timeout the status word gets MM_STATUS_TIMEOUT, the block stops
// after its next barrier, and thread 0 waits (bounded) for its copies in flight.
constexpr int kTmaStages = 4;
constexpr int kRawX = kT1 + 4;                                   // 36 doubles: a1 - 2 .. a1 + 33
constexpr int kRawY = kT2 + 2;                                   // 34 rows: a2 - 1 .. a2 + 32
constexpr uint32_t kRawBytes = kRawX * kRawY * 8;                // 9792 bytes per plane
constexpr uint32_t kRawStride = (kRawBytes + 127) / 128 * 128;
constexpr int kPairs = kRawY * (kRawX / 2);                      // 612 value pairs per plane
constexpr int kPairsPer = (kPairs + 255) / 256;
constexpr uint32_t kPlaneBytes = kRawY * kRawX * sizeof(float2);  // one split plane, 36 columns
constexpr size_t kTmaSmem = 128 + kTmaStages * kRawStride + 2 * kPlaneBytes + kTmaStages * 8;

template <class F>
__device__ __forceinline__ void store_pair(uint8_t* W, uint32_t pos, uint32_t pp, float x0, float x1) {
    uint32_t v0[3], v1[3];
    split_parts<F>(x0, 0.f, v0);
    split_parts<F>(x1, 0.f, v1);
    if (F::kElem == 2) {
        uint32_t* w = (uint32_t*)((uint16_t*)W + pos);
        const uint32_t step = pp >> 1;                           // parts pp elements apart
        w[0] = v0[0] | (v1[0] << 16);
        w[step] = v0[1] | (v1[1] << 16);
        if (F::kAParts == 3) w[2 * step] = v0[2] | (v1[2] << 16);
    } else {
        uint2* w = (uint2*)((uint32_t*)W + pos);
        const uint32_t step = pp >> 1;
        w[0] = make_uint2(v0[0], v1[0]);
        w[step] = make_uint2(v0[1], v1[1]);
        if (F::kAParts == 3) w[2 * step] = make_uint2(v0[2], v1[2]);
    }
}

template <class F, bool MANUF>
__global__ void __launch_bounds__(256, 3) stencil3d_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                               StencilArgsMixed a) {
    extern __shared__ uint8_t smem_raw[];
    // 128-byte aligned, by an offset on the shared array itself so that the compiler
    // keeps shared-memory instructions for the accesses below
    uint8_t* sm = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    float2(*sp)[kRawY][kRawX] = (float2(*)[kRawY][kRawX])(sm + kTmaStages * kRawStride);
    uint64_t* bars = (uint64_t*)(sm + kTmaStages * kRawStride + 2 * kPlaneBytes);
    __shared__ int fail;
    const int n1 = (int)a.n[0], n2 = (int)a.n[1], n3 = (int)a.n[2];
    const int t1 = (n1 + kT1 - 1) / kT1, t2 = (n2 + kT2 - 1) / kT2;
    const uint32_t plane = (uint32_t)n1 * (uint32_t)n2;
    const uint32_t p1 = (uint32_t)a.p1;
    const uint32_t pplane = p1 * (uint32_t)n2;
    const uint32_t pp = (uint32_t)a.part_pitch;
    uint8_t* const Wp = a.Wp;
    const float gf0 = a.g.f0, gf1 = a.g.f1, gf2 = a.g.f2, gf3 = a.g.f3;
    const float* cf1 = a.coef[0];
    const float* cf2 = a.coef[1];
    const float* cf3 = a.coef[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cp = lane & 15;                 // column pair: tile columns 2 cp, 2 cp + 1
    const int r0 = (lane >> 4) + 2 * w;       // rows r0 and r0 + 16 of the tile
    const int j0 = 2 * cp + 2;                // their index in the split planes
    if (threadIdx.x == 0) {
        for (int st = 0; st < kTmaStages; ++st) tc::mbar_init(tc::smem_u32(bars + st), 1);
        tc::fence_mbar_init();
        fail = 0;
    }
    __syncthreads();
    int64_t issued = 0, consumed = 0;    // planes loaded / taken from the ring by this block
    const int64_t total = (int64_t)t1 * t2 * n3;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t s_end = min(total, (int64_t)(blockIdx.x + 1) * per);
    for (int64_t s0 = (int64_t)blockIdx.x * per; s0 < s_end;) {
        const int T0 = (int)(s0 / n3);
        const int a1 = (T0 % t1) * kT1, a2 = (T0 / t1) * kT2, z0 = (int)(s0 % n3);
        const int z1 = (int)min((int64_t)n3, z0 + (s_end - s0));
        s0 += z1 - z0;
        // planes z0 - 1 .. z1 of this segment, loaded in order into the ring
        const int64_t first = issued, nplanes = z1 - z0 + 2;
        auto issue = [&](int64_t k) {        // thread 0: plane z0 - 1 + (k - first)
            const int st = (int)(k % kTmaStages);
            const uint32_t bar = tc::smem_u32(bars + st);
            tc::mbar_arrive_expect_tx(bar, kRawBytes);
            tc::tma_load_3d(tc::smem_u32(sm + st * kRawStride), &map, a1 - 2, a2 - 1, z0 - 1 + (int)(k - first), bar);
        };
        if (threadIdx.x == 0) {
            tc::fence_proxy_async_smem();
            for (; issued < first + min((int64_t)kTmaStages, nplanes); ++issued) issue(issued);
        }
        // take the next plane from the ring and split it, two values at a time, into
        // float2 plane buf (the raw box's column index kept)
        auto take = [&](int buf) -> bool {
            const int st = (int)(consumed % kTmaStages);
            if (!tc::mbar_wait(tc::smem_u32(bars + st), (uint32_t)(consumed / kTmaStages) & 1, a.status)) fail = 1;
            const double2* rp = (const double2*)(sm + st * kRawStride);
            float4* dst = (float4*)&sp[buf][0][0];
#pragma unroll
            for (int k = 0; k < kPairsPer; ++k) {
                const int e = threadIdx.x + 256 * k;
                if (e < kPairs) {
                    const double2 v = rp[e];
                    float4 h;
                    mx::d2ff(v.x, h.x, h.y);
                    mx::d2ff(v.y, h.z, h.w);
                    dst[e] = h;
                }
            }
            ++consumed;
            __syncthreads();
            if (threadIdx.x == 0 && issued < first + nplanes && !fail) {   // refill the stage just read
                tc::fence_proxy_async_smem();
                issue(issued++);
            }
            return fail == 0;
        };
        // coefficients along i_1 and i_2 are fixed for this thread's outputs
        const int i1 = a1 + 2 * cp;
        const bool in1 = i1 < n1;               // n1 even: both columns, or neither
        float c1a[2], c1c[2], c1s[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            c1a[j] = in1 ? __ldg(cf1 + i1 + j) : 0.f;
            c1c[j] = in1 ? __ldg(cf1 + n1 + i1 + j) : 0.f;
            c1s[j] = in1 ? __ldg(cf1 + 2 * n1 + i1 + j) : 0.f;
        }
        float c2a[2], c2c[2], s12[2][2];
        bool in2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i2 = a2 + r0 + 16 * q;
            in2[q] = i2 < n2;
            c2a[q] = in2[q] ? __ldg(cf2 + i2) : 0.f;
            c2c[q] = in2[q] ? __ldg(cf2 + n2 + i2) : 0.f;
            const float c2s = in2[q] ? __ldg(cf2 + 2 * n2 + i2) : 0.f;
            s12[q][0] = c1s[0] + c2s;
            s12[q][1] = c1s[1] + c2s;
        }
        // centres of planes z - 1 (cm) and z (c0) of this thread's outputs, [q][column]
        float4 cm[2], c0[2];
        if (!take((z0 + 1) & 1)) break;
#pragma unroll
        for (int q = 0; q < 2; ++q) cm[q] = *(const float4*)&sp[(z0 + 1) & 1][r0 + 16 * q + 1][j0];
        if (!take(z0 & 1)) break;
#pragma unroll
        for (int q = 0; q < 2; ++q) c0[q] = *(const float4*)&sp[z0 & 1][r0 + 16 * q + 1][j0];
        bool ok = true;
        for (int z = z0; z < z1 && ok; ++z) {
            const int b = z & 1, bn = b ^ 1;
            ok = take(bn);                      // plane z + 1 (its buffer held z - 1, read)
            if (!ok) break;
            const float a3a = __ldg(cf3 + z), a3c = __ldg(cf3 + n3 + z), a3s = __ldg(cf3 + 2 * n3 + z);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int r = r0 + 16 * q;
                const float4 cpn = *(const float4*)&sp[bn][r + 1][j0];           // plane z + 1
                if (in1 && in2[q]) {
                    const float2 lft = sp[b][r + 1][j0 - 1], rgt = sp[b][r + 1][j0 + 2];
                    const float4 up = *(const float4*)&sp[b][r][j0];
                    const float4 dn = *(const float4*)&sp[b][r + 2][j0];
                    const float2 ctr[2] = {make_float2(c0[q].x, c0[q].y), make_float2(c0[q].z, c0[q].w)};
                    const float2 nbl[2] = {lft, ctr[0]}, nbr[2] = {ctr[1], rgt};
                    const float2 nbu[2] = {make_float2(up.x, up.y), make_float2(up.z, up.w)};
                    const float2 nbd[2] = {make_float2(dn.x, dn.y), make_float2(dn.z, dn.w)};
                    const float2 nbm[2] = {make_float2(cm[q].x, cm[q].y), make_float2(cm[q].z, cm[q].w)};
                    const float2 nbp[2] = {make_float2(cpn.x, cpn.y), make_float2(cpn.z, cpn.w)};
                    float out[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float uh = ctr[j].x, ul = ctr[j].y;
                        const float u = uh + ul;
                        float acc;
                        if (MANUF) {
                            acc = mx::g32(a.g, u, a.t, (int64_t)(i1 + j) + (int64_t)n1 * (a2 + r) + (int64_t)plane * z);
                        } else {
                            acc = fmaf(fmaf(fmaf(gf3, u, gf2), u, gf1), u, gf0);
                        }
                        acc = fmaf(s12[q][j] + a3s, u, acc);
                        acc = stencil_term(c1a[j], nbl[j], uh, ul, acc);
                        acc = stencil_term(c1c[j], nbr[j], uh, ul, acc);
                        acc = stencil_term(c2a[q], nbu[j], uh, ul, acc);
                        acc = stencil_term(c2c[q], nbd[j], uh, ul, acc);
                        acc = stencil_term(a3a, nbm[j], uh, ul, acc);
                        acc = stencil_term(a3c, nbp[j], uh, ul, acc);
                        out[j] = acc;
                    }
                    store_pair<F>(Wp, (uint32_t)i1 + p1 * (uint32_t)(a2 + r) + pplane * (uint32_t)z, pp, out[0], out[1]);
                }
                cm[q] = c0[q];
                c0[q] = cpn;
            }
            __syncthreads();                    // before the next take overwrites plane z
        }
        if (!ok) break;
    }
    // never leave the block with copies in flight
    if (threadIdx.x == 0)
        for (int64_t k = consumed; k < issued; ++k)
            tc::mbar_wait(tc::smem_u32(bars + (int)(k % kTmaStages)), (uint32_t)(k / kTmaStages) & 1, a.status);
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
    if (a.mode == PRE_KU_G && (a.d == 2 || a.d == 3)) {
        const int64_t t1 = (a.n[0] + kT1 - 1) / kT1;
        const int64_t target = (int64_t)num_sms() * 8;
        int zc = kZ;
        int64_t tiles;
        if (a.d == 2) {
            tiles = t1 * ((a.n[1] + kT1 - 1) / kT1);
        } else {
            const int64_t t12 = t1 * ((a.n[1] + kT2 - 1) / kT2);
            const int64_t want_tz = (target + t12 - 1) / t12;            // chunks to fill the SMs
            zc = (int)std::max<int64_t>(4, std::min<int64_t>(kZ, (a.n[2] + want_tz - 1) / want_tz));
            tiles = t12 * ((a.n[2] + zc - 1) / zc);
        }
        if (tiles > 0x7fffffffLL) return MM_ERR_SHAPE;
        const unsigned grid = (unsigned)std::min<int64_t>(tiles, target);
        TraceScope tr(KC_PREPASS, s);
        if (a.d == 2) stencil2d_kernel<<<grid, 256, 0, s>>>(a);
        else if (!a.yadd && !a.yadd2 && !a.cadd && a.N < (int64_t(1) << 31) &&
                 (int64_t)a.part_pitch * (a.prec == MM_BF16X3 ? 3 : 2) < (int64_t(1) << 31)) {
            const bool manuf = a.g.kind == MM_G_ADR_MANUFACTURED;
            // TMA-fed march when the state admits a 3-D FP64 tensor map (16-byte aligned
            // base, even n1), else the register-prefetch march
            CUtensorMap map;
            const uint32_t box[3] = {(uint32_t)kRawX, (uint32_t)kRawY, 1};
            if (encode_f64_box3(&map, a.U, a.n, box) == MM_OK) {
                auto tk = a.prec == MM_BF16X3 ? (manuf ? stencil3d_tma_kernel<FormBF16, true>
                                                       : stencil3d_tma_kernel<FormBF16, false>)
                                              : (manuf ? stencil3d_tma_kernel<FormTF32, true>
                                                       : stencil3d_tma_kernel<FormTF32, false>);
                int per_sm = 0;
                MM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tk, 256, kTmaSmem));
                const int64_t steps = ((a.n[0] + kT1 - 1) / kT1) * ((a.n[1] + kT2 - 1) / kT2) * a.n[2];
                const unsigned g3 =
                    (unsigned)std::max<int64_t>(1, std::min<int64_t>(steps, (int64_t)num_sms() * std::max(per_sm, 1)));
                tk<<<g3, 256, kTmaSmem, s>>>(map, a);
                MM_LAUNCH_CHECK();
                return MM_OK;
            }
            auto kern = a.prec == MM_BF16X3 ? (manuf ? stencil3d_reg_kernel<FormBF16, true>
                                                     : stencil3d_reg_kernel<FormBF16, false>)
                                            : (manuf ? stencil3d_reg_kernel<FormTF32, true>
                                                     : stencil3d_reg_kernel<FormTF32, false>);
            int per_sm = 0;
            MM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
            const int64_t steps = ((a.n[0] + kT1 - 1) / kT1) * ((a.n[1] + kT2 - 1) / kT2) * a.n[2];
            const unsigned g3 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(steps, (int64_t)num_sms() * std::max(per_sm, 1)));
            kern<<<g3, 256, 0, s>>>(a);
        } else {
            stencil3d_kernel<<<grid, 256, 0, s>>>(a, zc);
        }
        MM_LAUNCH_CHECK();
        return MM_OK;
    }
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

int configure_prepass_kernels() {
    static bool done = false;
    if (done) return MM_OK;
    MM_CUDA_TRY(cudaFuncSetAttribute(stencil3d_tma_kernel<FormBF16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTmaSmem));
    MM_CUDA_TRY(cudaFuncSetAttribute(stencil3d_tma_kernel<FormBF16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTmaSmem));
    MM_CUDA_TRY(cudaFuncSetAttribute(stencil3d_tma_kernel<FormTF32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTmaSmem));
    MM_CUDA_TRY(cudaFuncSetAttribute(stencil3d_tma_kernel<FormTF32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTmaSmem));
    done = true;
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
