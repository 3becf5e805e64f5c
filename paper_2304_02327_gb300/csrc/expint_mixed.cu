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
// Workspace, with S = part_set_bytes (one operand buffer) and N the state size:
//   [IN: S][P1: S][P2: S][IN2: S (Lawson2b)][y: 4N][pairs: 8N][U2: 8N]
#include <math.h>

#include <algorithm>

#include "forms.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "stencil.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

namespace {

__device__ __forceinline__ void flag_nonfinite_bits(const Epi& e, double v) {
    if (!mx::finite_bits(v) && e.status) atomicOr(e.status, MM_STATUS_NONFINITE);
}

// The integrator epilogue of the mixed forms.
__global__ void __launch_bounds__(256) mixed_update_kernel(const float* __restrict__ y, Epi e,
                                                           int64_t N, float alphaf, float t0f, float t1f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float yi = __ldg(y + i);
        switch (e.kind) {
        case EPI_STORE:
            e.C[i] = e.alpha * mx::f2d(yi);
            break;
        case EPI_EE: {
            const double v = fma(e.alpha, mx::f2d(yi), e.U[i]);
            flag_nonfinite_bits(e, v);
            e.U[i] = v;
            break;
        }
        case EPI_ETD_S1: {
            const double u = e.U[i];
            e.U2[i] = fma(e.alpha, mx::f2d(yi), u);
            float uh, ul;
            mx::d2ff(u, uh, ul);
            const float w2 = mx::dg32(e.g, uh + ul, alphaf * yi, t0f, t1f, i);
            const int64_t pos = (i % e.w2_n) + (int64_t)e.w2_p * (i / e.w2_n);
            store_parts_prec(e.prec, e.W2p, e.w2_pitch, pos, w2, 0.f);
            break;
        }
        case EPI_ETD_S2: {
            const double v = fma(e.alpha, mx::f2d(yi), e.U2[i]);
            flag_nonfinite_bits(e, v);
            e.U[i] = v;
            break;
        }
        case EPI_LAWSON2: {
            float uh, ul;
            mx::d2ff(e.U2[i], uh, ul);
            const float gv = (float)e.beta * mx::g32(e.g, uh + ul, t1f, i);
            const double v = fma(e.alpha, mx::f2d(yi), mx::f2d(gv));
            flag_nonfinite_bits(e, v);
            e.U[i] = v;
            break;
        }
        default: break;
        }
    }
}

__global__ void __launch_bounds__(256) split_input_kernel(const double* __restrict__ V, uint8_t* parts,
                                                          int64_t pitch, int n1, int p1, int prec, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        mx::d2ff(__ldg(V + i), h, l);
        store_parts_prec(prec, parts, pitch, (i % n1) + (int64_t)p1 * (i / n1), h, l);
    }
}

int64_t grid_of(int64_t N) { return std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 16); }

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
    mixed_update_kernel<<<(unsigned)grid_of(p->N), 256, 0, s>>>(y, last, p->N, (float)last.alpha,
                                                                 (float)last.t0, (float)last.t1);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

size_t mixed_mumode_workspace_bytes(const mm_plan_s* p) {
    return 3 * part_set_bytes(p) + (size_t)p->N * sizeof(float) + 256;
}

size_t mixed_workspace_bytes(const mm_plan_s* p, int scheme) {
    const size_t S = part_set_bytes(p);
    const size_t N = (size_t)p->N;
    return 4 * S + N * (4 + 8 + 8) + 1024;
}

int mixed_expint(mm_plan_s* p, int scheme, const PointwiseG& pg, double* U, double t0, int nsteps,
                 uint8_t* ws, cudaStream_t s) {
    if (!p->tridiag) return MM_ERR_UNSUPPORTED;
    const int64_t N = p->N;
    const size_t S = part_set_bytes(p);
    uint8_t* IN = ws;
    uint8_t* P1 = IN + S;
    uint8_t* P2 = P1 + S;
    uint8_t* IN2 = P2 + S;
    float* y = (float*)(IN2 + S);
    float2* pairs = (float2*)(((uintptr_t)(y + N) + 255) & ~(uintptr_t)255);
    double* U2 = (double*)(pairs + N);
    const double tau = p->tau;
    const int d = p->d;
    const PartView in1 = mode_input_view(p, 1, IN);

    StencilArgsMixed a{};
    a.d = d; a.N = N; a.U = U; a.g = pg;
    a.part_pitch = in1.part_pitch; a.p1 = in1.p; a.prec = p->prec;
    int64_t st = 1;
    for (int mu = 0; mu < d; ++mu) {
        a.n[mu] = p->n[mu];
        a.stride[mu] = st;
        st *= p->n[mu];
        a.coef[mu] = p->coef3f[mu];
    }

    int rc = MM_OK;
    for (int k = 0; k < nsteps && rc == MM_OK; ++k) {
        const double t = t0 + k * tau;
        a.t = (float)t;
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
            e1.kind = EPI_ETD_S1; e1.alpha = tau; e1.U = U; e1.U2 = U2;
            e1.W2p = IN; e1.w2_pitch = in1.part_pitch; e1.w2_n = in1.n; e1.w2_p = in1.p;
            e1.t0 = t; e1.t1 = t + tau; e1.g = pg; e1.status = p->status;
            rc = mixed_tucker(p, 1, IN, P1, P2, y, e1, s);
            if (rc) break;
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
