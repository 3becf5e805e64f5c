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

}  // namespace mm
