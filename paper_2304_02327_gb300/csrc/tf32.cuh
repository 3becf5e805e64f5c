// TF32x3 tensor-core mu-mode products (tf32.cu).
#pragma once

#include "plan.cuh"

namespace mm {
// One mu-mode product of the Tucker chain with phi_ell of direction mu, on
// tcgen05 tensor cores with 3xTF32 split operands; the epilogue runs in FP64.
int tf32_mode_product(mm_plan_s* p, int ell, int mu, const double* in, const Epi& e, cudaStream_t s);
}  // namespace mm
