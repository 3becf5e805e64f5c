// Split-precision tensor-core mu-mode products (tf32.cu) and the mixed-form
// steppers (expint_mixed.cu).
#pragma once

#include "plan.cuh"

namespace mm {

// One operand of a mode: `parts` split arrays of `rows` fibres of n values at row
// pitch p; part q starts part_pitch elements after part q-1.
struct PartView {
    uint8_t* base;
    int n, p;
    int64_t rows, part_pitch;
};

int form_elem_bytes(int prec);
int form_parts(int prec);
int form_pitch(int prec, int n);
// Layout of the operand of mode mu (fibres along i_mu, rotated order).
PartView mode_input_view(const mm_plan_s* p, int mu, uint8_t* base);
// Bytes of one operand buffer large enough for every mode of the plan.
size_t part_set_bytes(const mm_plan_s* p);

// Mode mu with phi_ell: reads operand `in`, writes the next mode's operand parts to
// out_parts (mu < d) or the FP32 result in natural order to yout (mu == d).
int tc_mode_product(mm_plan_s* p, int ell, int mu, const PartView& in, uint8_t* out_parts, float* yout,
                    cudaStream_t s);
// MM_OK if a direction of size n is supported by the form `prec`.
int tf32_supported(int prec, int n);

// Tucker chain of the mixed form: input parts in mode-1 layout, operand buffers
// P1/P2 (part_set_bytes each), FP32 result y (N floats), then the FP64 epilogue
// `last` as one elementwise pass.
int mixed_tucker(mm_plan_s* p, int ell, uint8_t* in_parts, uint8_t* P1, uint8_t* P2, float* y,
                 const Epi& last, cudaStream_t s);
// FP64 tensor (natural order) -> its parts in mode-1 layout.
int mixed_split_input(const mm_plan_s* p, const double* V, uint8_t* parts, cudaStream_t s);
// Workspace of mixed_expint / the mixed mumode_phi_apply.
size_t mixed_workspace_bytes(const mm_plan_s* p, int scheme);
size_t mixed_mumode_workspace_bytes(const mm_plan_s* p);
// nsteps of `scheme` in the mixed form; ws laid out as in expint_mixed.cu.
int mixed_expint(mm_plan_s* p, int scheme, const PointwiseG& pg, double* U, double t0, int nsteps,
                 uint8_t* ws, cudaStream_t s);
}  // namespace mm
