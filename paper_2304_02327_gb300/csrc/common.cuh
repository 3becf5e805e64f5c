// Shared definitions of the PHISPLIT CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/phisplit.h"

#define MM_MAX_D 8

#define MM_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) { return MM_ERR_CUDA; }     \
    } while (0)

#define MM_LAUNCH_CHECK() MM_CUDA_TRY(cudaGetLastError())

namespace mm {

// Nonlinearity as the kernels see it (pointwise kinds only; Riccati is
// evaluated with GEMMs by the host orchestration).
struct PointwiseG {
    int kind;                 // MM_G_NONE / MM_G_CUBIC / MM_G_ADR_MANUFACTURED
    double c0, c1, c2, c3;
    float f0, f1, f2, f3;     // the same coefficients rounded to FP32 (mixed form)
    const double* psi_a;
    const double* psi_b;
};

__device__ __forceinline__ double g_point(const PointwiseG& g, double u, double t, int64_t idx) {
    if (g.kind == MM_G_CUBIC) {
        return fma(fma(fma(g.c3, u, g.c2), u, g.c1), u, g.c0);
    } else if (g.kind == MM_G_ADR_MANUFACTURED) {
        double et = exp(t);
        double b = g.psi_b[idx];
        return 1.0 / (1.0 + u * u) + et * g.psi_a[idx] - 1.0 / (1.0 + et * et * b * b);
    }
    return 0.0;
}

// Epilogue of the contraction kernels.  acc is the FP64 (or FP32-accumulated)
// sum for output element C(m, n); `off` is its linear offset in the output
// tensor, which is also its offset in the state-shaped arrays U, U2, W2.
enum EpiKind : int {
    EPI_STORE = 0,      // C = alpha*acc + beta*D1 + gamma*D2 + delta*D3 + diag*[m==n]
    EPI_EE = 1,         // U = U + alpha*acc                      (exp. Euler)
    EPI_ETD_S1 = 2,     // U2 = U + alpha*acc; W2 = g(U2,t1) - g(U,t0)
    EPI_ETD_S1_NOG = 3, // U2 = U + alpha*acc                     (non-pointwise g)
    EPI_ETD_S2 = 4,     // U = U2 + alpha*acc
    EPI_LAWSON2 = 5,    // U = alpha*acc + beta*g(U2, t1)
};

struct Epi {
    int kind;
    double alpha, beta, gamma, delta, diag;
    const double* D1;   // same layout as C (EPI_STORE)
    const double* D2;
    const double* D3;
    double* C;          // output for EPI_STORE
    double* U;
    double* U2;
    double* W2;
    float* W2f;         // (unused by the current forms)
    uint8_t* W2p;       // mixed form: parts of the stage-2 input g(U2) - g(U), mode-1 layout
    int64_t w2_pitch;   //   elements per part
    int w2_n, w2_p;     //   fibre length and row pitch of the mode-1 layout
    int prec;           //   the plan's precision form
    double t0, t1;
    PointwiseG g;
    unsigned int* status;
};

__device__ __forceinline__ void flag_nonfinite(const Epi& e, double v) {
    if (!isfinite(v) && e.status) atomicOr(e.status, MM_STATUS_NONFINITE);
}

__device__ __forceinline__ void apply_epilogue(const Epi& e, double acc, int64_t off, int m, int n) {
    switch (e.kind) {
    case EPI_STORE: {
        double v = e.alpha * acc;
        if (e.D1) v = fma(e.beta, e.D1[off], v);
        if (e.D2) v = fma(e.gamma, e.D2[off], v);
        if (e.D3) v = fma(e.delta, e.D3[off], v);
        if (m == n) v += e.diag;
        e.C[off] = v;
        break;
    }
    case EPI_EE: {
        double v = fma(e.alpha, acc, e.U[off]);
        flag_nonfinite(e, v);
        e.U[off] = v;
        break;
    }
    case EPI_ETD_S1: {
        double u = e.U[off];
        double u2 = fma(e.alpha, acc, u);
        e.U2[off] = u2;
        e.W2[off] = g_point(e.g, u2, e.t1, off) - g_point(e.g, u, e.t0, off);
        break;
    }
    case EPI_ETD_S1_NOG: {
        e.U2[off] = fma(e.alpha, acc, e.U[off]);
        break;
    }
    case EPI_ETD_S2: {
        double v = fma(e.alpha, acc, e.U2[off]);
        flag_nonfinite(e, v);
        e.U[off] = v;
        break;
    }
    case EPI_LAWSON2: {
        double v = fma(e.beta, g_point(e.g, e.U2[off], e.t1, off), e.alpha * acc);
        flag_nonfinite(e, v);
        e.U[off] = v;
        break;
    }
    default: break;
    }
}

// One contraction C(m, n) = sum_k A(m, k) B(k, n), batched:
//   A(m, k) = A[m + lda*k + b*sA]                       (m contiguous)
//   B(k, n) = B[k + ldb*n + b*sB]  if b_kcontig, else B[n + ldb*k + b*sB]
//   C(m, n) -> offset m + ldc*n + b*sC
struct Gemm {
    int M, N, K, batch;
    const double* A; int64_t lda, sA;
    const double* B; int64_t ldb, sB;
    int64_t ldc, sC;
    int b_kcontig;
    int two_level;      // sum each K-tile's chain apart (plan-time products)
};

int num_sms();

// FP64 contraction with epilogue (dgemm.cu).
int launch_dgemm(const Gemm& g, const Epi& e, cudaStream_t s);

// mu-mode product geometry for a tensor of sizes n[0..d-1] (i_1 fastest):
// (V x_mu M)[l, i, r] = sum_j M[i, j] V[l, j, r], L = prod_{nu<mu} n_nu,
// R = prod_{nu>mu} n_nu.  Fills a Gemm for input V and matrix M (column-major).
Gemm mode_gemm(int d, const int64_t* n, int mu, const double* M, const double* V);

}  // namespace mm
