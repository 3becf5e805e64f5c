// Arguments of the pointwise / stencil prepass (stencil.cu).
#pragma once

#include "common.cuh"

namespace mm {

enum PrepassMode : int { PRE_KU_G = 0, PRE_G = 1, PRE_LAWSON = 2 };

struct StencilArgs {
    int mode;
    int d;
    int64_t N;
    int64_t n[MM_MAX_D];
    int64_t stride[MM_MAX_D];
    const double* diag3[MM_MAX_D];
    const double* U;
    double* W;
    double* W2;
    double t, ca, cb;
    PointwiseG g;
};

int launch_prepass(const StencilArgs& a, cudaStream_t s);

// Mixed-precision prepass (split-operand output from the FP64 state, no FP64
// arithmetic; element idx goes to position (idx mod n_1) + p_1 (idx div n_1)):
//   PRE_KU_G:   W = K u + g(t, u) (+ yadd + yadd2 + cadd), K's tridiagonal band as
//               sum_mu a (u_{i-1} - u_i) + c (u_{i+1} - u_i) + s u_i with the row
//               sums s = a + b + c, the differences taken from the double-float
//               split of the state (so they keep their own relative accuracy)
//   PRE_LAWSON: W = u + ca g(t, u);  W2 = u + cb g(t, u) (if W2p != NULL)
struct StencilArgsMixed {
    int mode;
    int d;
    int64_t N;
    int64_t n[MM_MAX_D];
    int64_t stride[MM_MAX_D];
    const float* coef[MM_MAX_D];    // [a | c | s] per direction, 3 n floats
    const double* U;
    const float* yadd;              // PRE_KU_G: FP32 terms added to W, or NULL (dense
    const float* yadd2;             //   parts of K u, U B U of a Riccati G)
    const double* cadd;             // PRE_KU_G: FP64 term added to W (Riccati C), or NULL
    const float2* Up;               // U split once into (hi, lo) FP32 pairs (PRE_KU_G)
    uint8_t* Wp;                    // output parts (mode-1 layout)
    uint8_t* W2p;                   // second output parts (PRE_LAWSON), or NULL
    int64_t part_pitch;             // elements per part
    int p1;                         // row pitch of the mode-1 layout (fibre length n[0])
    int prec;
    float t, ca, cb;
    PointwiseG g;
    unsigned int* status;           // the plan's status word (a bounded wait that ran out)
};

// Runs split_pairs (U -> Up) and then the stencil; Up must hold N float2.
int launch_prepass_mixed(const StencilArgsMixed& a, float2* Up, cudaStream_t s);

// [a | c | s] floats of a column-major tridiagonal n x n matrix (plan set-up).
int build_stencil_coef(const double* A, int n, float* coef, cudaStream_t s);

// Shared-memory attributes of the prepass kernels, set once outside any stream capture.
int configure_prepass_kernels();

}  // namespace mm
