// TF32x3 tensor-core mu-mode products (tf32.cu).
#pragma once

#include "plan.cuh"

namespace mm {
// One mu-mode product with phi_ell of direction mu on tcgen05 tensor cores with
// 3xTF32 split operands.  `in` holds N doubles (in_fp64) or N floats; with
// last == NULL the FP32 result goes to `out` (N floats), otherwise the FP64
// epilogue `*last` consumes it.
int tf32_mode_product(mm_plan_s* p, int ell, int mu, const void* in, bool in_fp64, float* out,
                      const Epi* last, cudaStream_t s);
// MM_OK if a direction of size n is supported by the TF32x3 kernel.
int tf32_supported(int prec, int n);
// Tucker chain of the mixed form: FP64 (in64) or FP32 input, FP32 intermediates
// in F1/F2 (N floats each), FP64 epilogue `last` on the last mode (expint_mixed.cu).
int mixed_tucker(mm_plan_s* p, int ell, const void* in, bool in64, float* F1, float* F2,
                 const Epi& last, cudaStream_t s);
// nsteps of `scheme` in the mixed form; ws as laid out in expint_mixed.cu.
int mixed_expint(mm_plan_s* p, int scheme, const PointwiseG& pg, double* U, double t0, int nsteps,
                 double* ws, cudaStream_t s);
}  // namespace mm
