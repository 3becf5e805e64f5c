// Time steppers of the mixed-precision forms (MM_TF32X3, MM_BF16X3), Section 3.2
// eq. (17)-(20).
//
// Same schemes and PHISPLIT factors as the FP64 form (expint.cu); the arithmetic
// placement differs: the prepass writes the Tucker input K u + g already split into
// the form's parts (from exact FP32 differences of the FP64 state), the Tucker
// chain runs on tcgen05 fed by TMA, each mode writing the next mode's split
// operand, the last mode writes FP32, and one elementwise pass with every SM fully
// occupied performs the FP64 update u + tau*y (one DFMA per element) and, for
// ETD2RK, writes the split stage-2 input g(U2) - g(U) (formed in FP32 from its
// difference expansion).
//
// Dense A_mu (d = 2) and the Riccati G (even d; U the n1 x n2 column-major matrix view
// of the state, n1 the product of the first d/2 sizes; Section 1 eq. (2)):
// K u is split into the tridiagonal band of each A_mu, evaluated by the stencil
// prepass from differences of the state, plus the remainders R_mu = A_mu - band:
//   R1 U = X M^T with X = R1, M = U^T;    U R2^T with X = U, M = R2,
// and U B U as (U B) U: first T = B^T U^T (X = B^T, M = U), written as parts of
// U B with the contraction index fastest, then T U (X = U B, M = U^T).  The state
// is split twice per evaluation (as M = U and as M = U^T); B once per call.  The
// products land in FP32 (yk: the remainders, yq: U B U) and the prepass adds them
// and C to the band stencil.  The tridiagonal band stays out of the tensor-core
// products because its entries (~h^-2) would make their rounding dominate the
// K u + G difference.
//
// Workspace, with S = part_set_bytes (one operand buffer) and N the state size,
// every piece 256-byte aligned:
//   [IN: S][P1: S][P2: S][IN2: S (Lawson2b)][y: 4N][pairs: 8N][U2: 8N]
//   dense / Riccati: [Ut: U 3 parts][Un: U^T 3 parts][T: U B parts][Bx: B^T parts]
//                    [yk: 4N][yq: 4N]
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "forms.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "stencil.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

namespace {

// Position of natural-order element i in the mode-1 layout (fibres of n at pitch
// p): 32-bit division when the tensor allows it.
__device__ __forceinline__ int64_t mode1_pos(int64_t i, int n, int p, int64_t N) {
    if (N < (int64_t(1) << 31)) {
        const uint32_t q = (uint32_t)i / (uint32_t)n;
        return ((uint32_t)i - q * (uint32_t)n) + (int64_t)p * q;
    }
    return (i % n) + (int64_t)p * (i / n);
}

__device__ __forceinline__ void flag_nonfinite_bits(const Epi& e, double v) {
    if (!mx::finite_bits(v) && e.status) atomicOr(e.status, MM_STATUS_NONFINITE);
}

// The integrator epilogue of the mixed forms, element i.
__device__ __forceinline__ void update_one(const Epi& e, int64_t i, float yi, double ui, int64_t N, float alphaf,
                                           float t0f, float t1f) {
    switch (e.kind) {
    case EPI_STORE:
        e.C[i] = e.alpha * mx::f2d(yi);
        break;
    case EPI_EE: {
        const double v = fma(e.alpha, mx::f2d(yi), ui);
        flag_nonfinite_bits(e, v);
        e.U[i] = v;
        break;
    }
    case EPI_ETD_S1: {
        e.U2[i] = fma(e.alpha, mx::f2d(yi), ui);
        float uh, ul;
        mx::d2ff(ui, uh, ul);
        const float w2 = mx::dg32(e.g, uh + ul, alphaf * yi, t0f, t1f, i);
        store_parts_prec(e.prec, e.W2p, e.w2_pitch, mode1_pos(i, e.w2_n, e.w2_p, N), w2, 0.f);
        break;
    }
    case EPI_ETD_S1_NOG:
        e.U2[i] = fma(e.alpha, mx::f2d(yi), ui);
        break;
    case EPI_ETD_S2: {
        const double v = fma(e.alpha, mx::f2d(yi), ui);
        flag_nonfinite_bits(e, v);
        e.U[i] = v;
        break;
    }
    case EPI_LAWSON2: {
        float uh, ul;
        mx::d2ff(ui, uh, ul);
        const float gv = (float)e.beta * mx::g32(e.g, uh + ul, t1f, i);
        const double v = fma(e.alpha, mx::f2d(yi), mx::f2d(gv));
        flag_nonfinite_bits(e, v);
        e.U[i] = v;
        break;
    }
    default: break;
    }
}

// Four elements per thread and pass, their loads issued together (the pass is
// bound by memory latency otherwise); the state read is U (exp. Euler, ETD2RK
// stage 1) or U2 (stage 2, Lawson2b).
__global__ void __launch_bounds__(256) mixed_update_kernel(const float* __restrict__ y, Epi e,
                                                           int64_t N, float alphaf, float t0f, float t1f) {
    const double* src = (e.kind == EPI_ETD_S2 || e.kind == EPI_LAWSON2) ? e.U2 : e.U;
    const bool reads = e.kind != EPI_STORE;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        float yv[4];
        double uv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * stride;
            yv[k] = i < N ? __ldg(y + i) : 0.f;
            uv[k] = (reads && i < N) ? __ldg(src + i) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * stride;
            if (i < N) update_one(e, i, yv[k], uv[k], N, alphaf, t0f, t1f);
        }
    }
}

// The same epilogue for the common case of 16-byte aligned arrays and N a multiple
// of 4: each thread takes four consecutive elements with 16-byte loads and stores
// (y as one float4, the states as two double2), the kind and the form are template
// parameters, and for ETD2RK stage 1 with unpadded fibres (p_1 = n_1, the stage-2
// input's positions are the elements' own) the parts go out as one vector per part.
// Element for element the arithmetic of update_one.
template <class F, int KIND>
__global__ void __launch_bounds__(256) update4_kernel(const float* __restrict__ y, Epi e, int64_t N, float alphaf,
                                                      float t0f, float t1f) {
    using PT = typename std::conditional<F::kElem == 4, uint32_t, uint16_t>::type;
    const double* src = (KIND == EPI_ETD_S2 || KIND == EPI_LAWSON2) ? e.U2 : e.U;
    const int64_t N4 = N >> 2;
    const bool flat = e.w2_p == e.w2_n;
    bool bad = false;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N4; g += (int64_t)gridDim.x * blockDim.x) {
        const float4 yq = __ldg((const float4*)y + g);
        const float yv[4] = {yq.x, yq.y, yq.z, yq.w};
        double uv[4] = {0.0, 0.0, 0.0, 0.0};
        if (KIND != EPI_STORE) {
            const double2 a = __ldg((const double2*)src + 2 * g), b = __ldg((const double2*)src + 2 * g + 1);
            uv[0] = a.x; uv[1] = a.y; uv[2] = b.x; uv[3] = b.y;
        }
        const int64_t i0 = 4 * g;
        double out[4];
        uint32_t parts[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (KIND == EPI_STORE) {
                out[j] = e.alpha * mx::f2d(yv[j]);
            } else if (KIND == EPI_EE || KIND == EPI_ETD_S2 || KIND == EPI_ETD_S1 || KIND == EPI_ETD_S1_NOG) {
                out[j] = fma(e.alpha, mx::f2d(yv[j]), uv[j]);
            } else {   // EPI_LAWSON2
                float uh, ul;
                mx::d2ff(uv[j], uh, ul);
                const float gv = (float)e.beta * mx::g32(e.g, uh + ul, t1f, i0 + j);
                out[j] = fma(e.alpha, mx::f2d(yv[j]), mx::f2d(gv));
            }
            if (KIND == EPI_ETD_S1) {
                float uh, ul;
                mx::d2ff(uv[j], uh, ul);
                split_parts<F>(mx::dg32(e.g, uh + ul, alphaf * yv[j], t0f, t1f, i0 + j), 0.f, parts[j]);
            }
            if (KIND == EPI_EE || KIND == EPI_ETD_S2 || KIND == EPI_LAWSON2) bad |= !mx::finite_bits(out[j]);
        }
        double* dst = (KIND == EPI_STORE) ? e.C : (KIND == EPI_ETD_S1 || KIND == EPI_ETD_S1_NOG) ? e.U2 : e.U;
        ((double2*)dst)[2 * g] = make_double2(out[0], out[1]);
        ((double2*)dst)[2 * g + 1] = make_double2(out[2], out[3]);
        if (KIND == EPI_ETD_S1) {
            if (flat) {
#pragma unroll
                for (int q = 0; q < F::kAParts; ++q) {
                    if (F::kElem == 4) {
                        ((uint4*)((uint32_t*)e.W2p + q * e.w2_pitch))[g] =
                            make_uint4(parts[0][q], parts[1][q], parts[2][q], parts[3][q]);
                    } else {
                        ((uint2*)((uint16_t*)e.W2p + q * e.w2_pitch))[g] =
                            make_uint2(parts[0][q] | (parts[1][q] << 16), parts[2][q] | (parts[3][q] << 16));
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t pos = mode1_pos(i0 + j, e.w2_n, e.w2_p, N);
#pragma unroll
                    for (int q = 0; q < F::kAParts; ++q) ((PT*)e.W2p)[q * e.w2_pitch + pos] = (PT)parts[j][q];
                }
            }
        }
    }
    if (bad && e.status) atomicOr(e.status, MM_STATUS_NONFINITE);
}

template <class F>
int launch_update4(const float* y, const Epi& e, int64_t N, cudaStream_t s) {
    const unsigned grid = (unsigned)std::min<int64_t>((N / 4 + 255) / 256, (int64_t)num_sms() * 8);
    const float af = (float)e.alpha, t0f = (float)e.t0, t1f = (float)e.t1;
    switch (e.kind) {
    case EPI_STORE: update4_kernel<F, EPI_STORE><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    case EPI_EE: update4_kernel<F, EPI_EE><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    case EPI_ETD_S1: update4_kernel<F, EPI_ETD_S1><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    case EPI_ETD_S1_NOG: update4_kernel<F, EPI_ETD_S1_NOG><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    case EPI_ETD_S2: update4_kernel<F, EPI_ETD_S2><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    case EPI_LAWSON2: update4_kernel<F, EPI_LAWSON2><<<grid, 256, 0, s>>>(y, e, N, af, t0f, t1f); break;
    default: return MM_ERR_ARG;
    }
    MM_LAUNCH_CHECK();
    return MM_OK;
}

// Whether the vector epilogue applies: N a multiple of 4, every array it touches
// 16-byte aligned (and the stage-2 part arrays' pitch a multiple of 4 elements).
bool update4_ok(const float* y, const Epi& e, int64_t N) {
    auto al = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
    if (N % 4 || !al(y) || !al(e.U) || !al(e.U2) || !al(e.C) || !al(e.W2p)) return false;
    if (e.kind == EPI_ETD_S1 && (e.w2_pitch % 4)) return false;
    return e.kind != EPI_STORE || (e.D1 == nullptr && e.D2 == nullptr && e.D3 == nullptr);
}

__global__ void __launch_bounds__(256) split_input_kernel(const double* __restrict__ V, uint8_t* parts,
                                                          int64_t pitch, int n1, int p1, int prec, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        mx::d2ff(__ldg(V + i), h, l);
        store_parts_prec(prec, parts, pitch, mode1_pos(i, n1, p1, N), h, l);
    }
}

// W2 = ya - yb as parts in the mode-1 layout (the Riccati stage-2 input).
__global__ void __launch_bounds__(256) diff_split_kernel(const float* __restrict__ ya, const float* __restrict__ yb,
                                                         uint8_t* parts, int64_t pitch, int n1, int p1, int prec,
                                                         int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        store_parts_prec(prec, parts, pitch, mode1_pos(i, n1, p1, N), __ldg(ya + i) - __ldg(yb + i), 0.f);
}

int64_t grid_of(int64_t N) { return std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 16); }

struct Carve {
    uint8_t* p;
    size_t used = 0;
    uint8_t* take(size_t bytes) {
        uint8_t* q = p ? p + used : nullptr;
        used += (bytes + 255) / 256 * 256;
        return q;
    }
};

// The workspace pieces of expint_mixed (see the layout above).
struct MixedWs {
    uint8_t *IN, *P1, *P2, *IN2;
    float* y;
    float2* pairs;
    double* U2;
    uint8_t *Ut, *Un, *T, *Bx;
    float *yk, *yq;
    size_t bytes;
};

MixedWs carve_ws(const mm_plan_s* p, bool dense, uint8_t* base) {
    // the base is 16-byte aligned; start the pieces on a 256-byte boundary
    uint8_t* b0 = base ? (uint8_t*)(((uintptr_t)base + 255) & ~(uintptr_t)255) : nullptr;
    Carve c{b0};
    MixedWs w{};
    const size_t S = part_set_bytes(p);
    const size_t N = (size_t)p->N;
    w.IN = c.take(S); w.P1 = c.take(S); w.P2 = c.take(S); w.IN2 = c.take(S);
    w.y = (float*)c.take(4 * N);
    w.pairs = (float2*)c.take(8 * N);
    w.U2 = (double*)c.take(8 * N);
    if (dense) {
        const int n1 = (int)riccati_rows(p), n2 = (int)(p->N / n1);
        w.Ut = c.take(matrix_parts_bytes(p->prec, n1, n2, 3));
        w.Un = c.take(matrix_parts_bytes(p->prec, n2, n1, 3));
        w.T = c.take(matrix_parts_bytes(p->prec, n1, n1, 3));
        w.Bx = c.take(matrix_parts_bytes(p->prec, n1, n2, 3));
        w.yk = (float*)c.take(4 * N);
        w.yq = (float*)c.take(4 * N);
    }
    w.bytes = c.used + 256;
    return w;
}

// For the state U: yk = R1 U + U R2^T (rem) and yq = U B U (ubu).
int dense_products(mm_plan_s* p, const double* U, bool rem, bool ubu, float* yk, float* yq, const MixedWs& w,
                   cudaStream_t s) {
    const int prec = p->prec;
    const int n1 = (int)riccati_rows(p), n2 = (int)(p->N / n1);
    const PartView Ut = matrix_view(prec, w.Ut, n1, n2);     // M = U   (rows i1, k = i2)
    const PartView Un = matrix_view(prec, w.Un, n2, n1);     // M = U^T (rows i2, k = i1)
    int rc = split_matrix(prec, U, n1, 1, 0, Ut, 3, s);
    if (!rc) rc = split_matrix(prec, U, n1, 0, 0, Un, 3, s);
    if (rc) return rc;
    TcOut o{};
    o.last = 1; o.ldy = n1;
    if (rem) {
        o.y = yk; o.accum = 0;
        rc = tc_product(prec, Ut, matrix_view(prec, (uint8_t*)p->rem_split[1], n2, n2), o, p->status, s);
        if (rc) return rc;
        o.accum = 1;
        rc = tc_product(prec, matrix_view(prec, (uint8_t*)p->rem_split[0], n1, n1), Un, o, p->status, s);
        if (rc) return rc;
    }
    if (ubu) {
        const PartView T = matrix_view(prec, w.T, n1, n1);    // U B, rows i1
        TcOut ot{};
        ot.last = 0; ot.parts = w.T; ot.part_pitch = T.part_pitch;
        ot.next_n = n1; ot.next_p = T.p; ot.next_rows_per_i = 1;
        rc = tc_product(prec, matrix_view(prec, w.Bx, n1, n2), Ut, ot, p->status, s);
        if (rc) return rc;
        o.y = yq; o.accum = 0;
        rc = tc_product(prec, T, Un, o, p->status, s);
    }
    return rc;
}

}  // namespace

int mixed_split_input(const mm_plan_s* p, const double* V, uint8_t* parts, cudaStream_t s) {
    const PartView v = mode_input_view(p, 1, parts);
    TraceScope tr(KC_SPLIT, s);
    split_input_kernel<<<(unsigned)grid_of(p->N), 256, 0, s>>>(V, parts, v.part_pitch, v.n, v.p, p->prec, p->N);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int mixed_tucker(mm_plan_s* p, int ell, uint8_t* in_parts, uint8_t* P1, uint8_t* P2, float* y,
                 const Epi& last0, cudaStream_t s) {
    uint8_t* cur = in_parts;
    for (int mu = 1; mu <= p->d; ++mu) {
        uint8_t* out = (mu & 1) ? P1 : P2;
        int rc = tc_mode_product(p, ell, mu, mode_input_view(p, mu, cur), out, y, s);
        if (rc) return rc;
        cur = out;
    }
    Epi last = last0;
    last.prec = p->prec;
    TraceScope tr(KC_SPLIT, s);
    if (update4_ok(y, last, p->N))
        return p->prec == MM_BF16X3 ? launch_update4<FormBF16>(y, last, p->N, s) : launch_update4<FormTF32>(y, last, p->N, s);
    mixed_update_kernel<<<(unsigned)grid_of(p->N), 256, 0, s>>>(y, last, p->N, (float)last.alpha,
                                                                 (float)last.t0, (float)last.t1);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

size_t mixed_mumode_workspace_bytes(const mm_plan_s* p) {
    return 3 * part_set_bytes(p) + (size_t)p->N * sizeof(float) + 256;
}

size_t mixed_workspace_bytes(const mm_plan_s* p, int scheme, int gkind) {
    (void)scheme;
    return carve_ws(p, !p->tridiag || gkind == MM_G_RICCATI, nullptr).bytes;
}

int mixed_expint(mm_plan_s* p, int scheme, const mm_nonlin* gd, double* U, double t0, int nsteps,
                 uint8_t* ws, cudaStream_t s) {
    const bool riccati = gd && gd->kind == MM_G_RICCATI;
    const bool dense = !p->tridiag || riccati;
    if (!p->tridiag && (p->d != 2 || !p->rem_split[0])) return MM_ERR_UNSUPPORTED;
    if (riccati && p->d % 2 != 0) return MM_ERR_UNSUPPORTED;
    if (riccati && scheme != MM_EXPEULER && scheme != MM_ETD2RK) return MM_ERR_UNSUPPORTED;
    const PointwiseG pg = pointwise_of(gd);
    const MixedWs w = carve_ws(p, dense, ws);
    uint8_t* IN = w.IN;
    uint8_t* P1 = w.P1;
    uint8_t* P2 = w.P2;
    uint8_t* IN2 = w.IN2;
    float* y = w.y;
    float2* pairs = w.pairs;
    double* U2 = w.U2;
    const int64_t N = p->N;
    int rc = MM_OK;
    if (riccati) {   // X = B^T: B is n2 x n1 column-major
        const int64_t m1 = riccati_rows(p), m2 = p->N / m1;    // B is m2 x m1
        rc = split_matrix(p->prec, gd->B, m2, 0, 0, matrix_view(p->prec, w.Bx, m1, (int)m2), form_parts(p->prec), s);
        if (rc) return rc;
    }
    const double tau = p->tau;
    const int d = p->d;
    const PartView in1 = mode_input_view(p, 1, IN);

    StencilArgsMixed a{};
    a.d = d; a.N = N; a.U = U; a.g = pg;
    a.yadd = !p->tridiag ? w.yk : nullptr;
    a.yadd2 = riccati ? w.yq : nullptr;
    a.cadd = riccati ? gd->C : nullptr;
    a.part_pitch = in1.part_pitch; a.p1 = in1.p; a.prec = p->prec;
    a.status = p->status;
    int64_t st = 1;
    for (int mu = 0; mu < d; ++mu) {
        a.n[mu] = p->n[mu];
        a.stride[mu] = st;
        st *= p->n[mu];
        a.coef[mu] = p->coef3f[mu];
    }

    for (int k = 0; k < nsteps && rc == MM_OK; ++k) {
        const double t = t0 + k * tau;
        a.t = (float)t;
        if (dense && (scheme == MM_EXPEULER || scheme == MM_ETD2RK)) {
            rc = dense_products(p, U, !p->tridiag, riccati, w.yk, w.yq, w, s);
            if (rc) break;
        }
        switch (scheme) {
        case MM_EXPEULER: {
            a.mode = PRE_KU_G; a.Wp = IN; a.W2p = nullptr;
            rc = launch_prepass_mixed(a, pairs, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_EE; e.alpha = tau; e.U = U; e.status = p->status;
            rc = mixed_tucker(p, 1, IN, P1, P2, y, e, s);
            break;
        }
        case MM_ETD2RK: {
            a.mode = PRE_KU_G; a.Wp = IN; a.W2p = nullptr;
            rc = launch_prepass_mixed(a, pairs, s);
            if (rc) break;
            Epi e1{};
            e1.kind = riccati ? EPI_ETD_S1_NOG : EPI_ETD_S1; e1.alpha = tau; e1.U = U; e1.U2 = U2;
            e1.W2p = IN; e1.w2_pitch = in1.part_pitch; e1.w2_n = in1.n; e1.w2_p = in1.p;
            e1.t0 = t; e1.t1 = t + tau; e1.g = pg; e1.status = p->status;
            rc = mixed_tucker(p, 1, IN, P1, P2, y, e1, s);
            if (rc) break;
            if (riccati) {   // W2 = G(U2) - G(U) = U2 B U2 - U B U
                // U2 B U2 into yk (the remainders in it are used up)
                rc = dense_products(p, U2, false, true, nullptr, w.yk, w, s);
                if (rc) break;
                TraceScope tr(KC_SPLIT, s);
                diff_split_kernel<<<(unsigned)grid_of(N), 256, 0, s>>>(w.yk, w.yq, IN, in1.part_pitch, in1.n,
                                                                        in1.p, p->prec, N);
                MM_LAUNCH_CHECK();
            }
            Epi e2{};
            e2.kind = EPI_ETD_S2; e2.alpha = tau * pow(2.0, d - 1); e2.U = U; e2.U2 = U2;
            e2.status = p->status;
            rc = mixed_tucker(p, 2, IN, P1, P2, y, e2, s);
            break;
        }
        case MM_LAWSON_EULER: {
            a.mode = PRE_LAWSON; a.Wp = IN; a.W2p = nullptr; a.ca = (float)tau;
            rc = launch_prepass_mixed(a, pairs, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_STORE; e.alpha = 1.0; e.C = U;
            rc = mixed_tucker(p, 0, IN, P1, P2, y, e, s);
            break;
        }
        case MM_LAWSON2B: {
            a.mode = PRE_LAWSON; a.Wp = IN; a.W2p = IN2; a.ca = (float)tau; a.cb = (float)(0.5 * tau);
            rc = launch_prepass_mixed(a, pairs, s);
            if (rc) break;
            Epi e1{};
            e1.kind = EPI_STORE; e1.alpha = 1.0; e1.C = U2;
            rc = mixed_tucker(p, 0, IN, P1, P2, y, e1, s);
            if (rc) break;
            Epi e2{};
            e2.kind = EPI_LAWSON2; e2.alpha = 1.0; e2.beta = 0.5 * tau; e2.U = U; e2.U2 = U2;
            e2.t1 = t + tau; e2.g = pg; e2.status = p->status;
            rc = mixed_tucker(p, 0, IN2, P1, P2, y, e2, s);
            break;
        }
        default: rc = MM_ERR_ARG;
        }
    }
    return rc;
}

}  // namespace mm
