// Time steppers of the mixed-precision form (MM_TF32X3), Section 3.2 eq. (17)-(20).
//
// Same schemes and the same PHISPLIT factors as the FP64 form (expint.cu); the
// differences are the arithmetic placement: the prepass writes the Tucker input
// K u + g in FP32 (from exact FP32 differences of the FP64 state), the Tucker
// chain runs on tcgen05 with FP32 intermediates, and the last mode's epilogue
// updates the FP64 state with one DFMA per element (the stage value g(U2) - g(U)
// of ETD2RK is formed in FP32 from its difference expansion).
//
// Workspace (N = state size; buffer k = doubles [kN, (k+1)N)):
//   buffer 0: FP32 Tucker inputs (Wf, then W2f or Zf) -- 2N floats
//   buffer 1: FP32 mode intermediates F1, F2          -- 2N floats
//   buffer 2: FP64 stage value U2 (ETD2RK, Lawson2b)
#include <math.h>

#include "plan.cuh"
#include "stencil.cuh"
#include "tf32.cuh"

namespace mm {

int mixed_tucker(mm_plan_s* p, int ell, const void* in, bool in64, float* F1, float* F2,
                 const Epi& last, cudaStream_t s) {
    const void* cur = in;
    bool cur64 = in64;
    for (int mu = 1; mu < p->d; ++mu) {
        float* out = (mu & 1) ? F1 : F2;
        int rc = tf32_mode_product(p, ell, mu, cur, cur64, out, nullptr, s);
        if (rc) return rc;
        cur = out;
        cur64 = false;
    }
    return tf32_mode_product(p, ell, p->d, cur, cur64, nullptr, &last, s);
}

int mixed_expint(mm_plan_s* p, int scheme, const PointwiseG& pg, double* U, double t0, int nsteps,
                 double* ws, cudaStream_t s) {
    if (!p->tridiag) return MM_ERR_UNSUPPORTED;
    const int64_t N = p->N;
    float* Wf = (float*)ws;
    float* W2f = Wf + N;
    float* F1 = (float*)(ws + N);
    float* F2 = F1 + N;
    double* U2 = ws + 2 * N;
    const double tau = p->tau;
    const int d = p->d;

    StencilArgsMixed a{};
    a.d = d; a.N = N; a.U = U; a.g = pg;
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
            a.mode = PRE_KU_G; a.Wf = Wf; a.W2f = nullptr;
            rc = launch_prepass_mixed(a, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_EE; e.alpha = tau; e.U = U; e.status = p->status;
            rc = mixed_tucker(p, 1, Wf, false, F1, F2, e, s);
            break;
        }
        case MM_ETD2RK: {
            a.mode = PRE_KU_G; a.Wf = Wf; a.W2f = nullptr;
            rc = launch_prepass_mixed(a, s);
            if (rc) break;
            Epi e1{};
            e1.kind = EPI_ETD_S1; e1.alpha = tau; e1.U = U; e1.U2 = U2; e1.W2f = W2f;
            e1.t0 = t; e1.t1 = t + tau; e1.g = pg; e1.status = p->status;
            rc = mixed_tucker(p, 1, Wf, false, F1, F2, e1, s);
            if (rc) break;
            Epi e2{};
            e2.kind = EPI_ETD_S2; e2.alpha = tau * pow(2.0, d - 1); e2.U = U; e2.U2 = U2;
            e2.status = p->status;
            rc = mixed_tucker(p, 2, W2f, false, F1, F2, e2, s);
            break;
        }
        case MM_LAWSON_EULER: {
            a.mode = PRE_LAWSON; a.Wf = Wf; a.W2f = nullptr; a.ca = (float)tau;
            rc = launch_prepass_mixed(a, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_STORE; e.alpha = 1.0; e.C = U;
            rc = mixed_tucker(p, 0, Wf, false, F1, F2, e, s);
            break;
        }
        case MM_LAWSON2B: {
            a.mode = PRE_LAWSON; a.Wf = Wf; a.W2f = W2f; a.ca = (float)tau; a.cb = (float)(0.5 * tau);
            rc = launch_prepass_mixed(a, s);
            if (rc) break;
            Epi e1{};
            e1.kind = EPI_STORE; e1.alpha = 1.0; e1.C = U2;
            rc = mixed_tucker(p, 0, Wf, false, F1, F2, e1, s);
            if (rc) break;
            Epi e2{};
            e2.kind = EPI_LAWSON2; e2.alpha = 1.0; e2.beta = 0.5 * tau; e2.U = U; e2.U2 = U2;
            e2.t1 = t + tau; e2.g = pg; e2.status = p->status;
            rc = mixed_tucker(p, 0, W2f, false, F1, F2, e2, s);
            break;
        }
        default: rc = MM_ERR_ARG;
        }
    }
    return rc;
}

}  // namespace mm
