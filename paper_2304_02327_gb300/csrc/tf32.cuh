// Split-precision tensor-core mu-mode products (tf32.cu) and the mixed-form
// steppers (expint_mixed.cu).
#pragma once

#include <cuda.h>

#include <vector>

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
// A 3-D TMA map of a contiguous FP64 array with sizes dims[0] (fastest) x dims[1] x
// dims[2], box box[0] x box[1] x box[2], no swizzle; loads past the array read zeros.
// MM_ERR_ARG if the base is not 16-byte aligned or a row / plane pitch or the box's
// rows are not a multiple of 16 bytes.
int encode_f64_box3(CUtensorMap* map, const double* base, const int64_t* dims, const uint32_t* box);
int form_parts(int prec);
int form_pitch(int prec, int n);
// Layout of the operand of mode mu (fibres along i_mu, rotated order).
PartView mode_input_view(const mm_plan_s* p, int mu, uint8_t* base);
// Bytes of one operand buffer large enough for every mode of the plan.
size_t part_set_bytes(const mm_plan_s* p);

// A matrix M (rows x K) as a part array: M[i][k] at k + p i of each part.
PartView matrix_view(int prec, uint8_t* base, int64_t rows, int K);
// Bytes of nparts parts of a rows x K matrix (rounded to 256).
size_t matrix_parts_bytes(int prec, int64_t rows, int K, int nparts);
// Parts of the FP64 matrix M into dst (layout of matrix_view): src holds M
// column-major (colmajor = 1, M[i][k] = src[i + ld k]) or M^T column-major
// (colmajor = 0, M[i][k] = src[k + ld i]); zero_band drops the tridiagonal band.
int split_matrix(int prec, const double* src, int64_t ld, int colmajor, int zero_band, const PartView& dst,
                 int nparts, cudaStream_t s);

// Output of one tensor-core product D = X M^T (D[q][i], q < X.rows, i < M.rows):
//   last = 1: FP32, y[q + ldy i] = D (accum = 0) or += D (accum = 1)
//   last = 0: parts of D at next_n-fibre layout position
//             (q mod next_n) + next_p ((q div next_n) + next_rows_per_i i)
struct TcOut {
    int last, accum;
    float* y;
    int64_t ldy;
    uint8_t* parts;
    int64_t part_pitch;
    int next_n, next_p;
    int64_t next_rows_per_i;
};
// D = X M^T on the tensor cores: X with the form's kAParts parts, M with 3 parts,
// both with the contraction index fastest (X.n == M.n).
int tc_product(int prec, const PartView& X, const PartView& M, const TcOut& out, unsigned int* status,
               cudaStream_t s);

// Grouped products: up to MM_TC_MAX_CLASSES classes of `count` equal-shape
// instances each, operands packed instance after instance (X rows j * rows..,
// M rows j * ncols..), outputs at per-instance strides (y_stride floats for FP32,
// p_stride elements within each part for split output).
#define MM_TC_MAX_CLASSES 32
struct TcClassSpec {
    PartView X;             // rows = rows * count
    int rows;
    PartView M;             // rows = ncols * count
    int ncols;
    int count;
    TcOut out;
    int64_t y_stride, p_stride;
};
// The tile list of a grouped product, tiles of decreasing cost (nc per class from
// nc_cap[c], a multiple of 16 <= 128).
int tc_group_tiles(int prec, const TcClassSpec* cls, int ncls, const int* nc_cap, std::vector<int4>& tiles);
// One persistent launch over the tiles (device array of tc_group_tiles' output).
int tc_group_product(int prec, const TcClassSpec* cls, int ncls, const int* nc_cap, const int4* dev_tiles,
                     int64_t ntiles, unsigned int* status, cudaStream_t s);

// Mode mu with phi_ell: reads operand `in`, writes the next mode's operand parts to
// out_parts (mu < d) or the FP32 result in natural order to yout (mu == d).
int tc_mode_product(mm_plan_s* p, int ell, int mu, const PartView& in, uint8_t* out_parts, float* yout,
                    cudaStream_t s);

// Tucker chain of the mixed form: input parts in mode-1 layout, operand buffers
// P1/P2 (part_set_bytes each), FP32 result y (N floats), then the FP64 epilogue
// `last` as one elementwise pass.
int mixed_tucker(mm_plan_s* p, int ell, uint8_t* in_parts, uint8_t* P1, uint8_t* P2, float* y,
                 const Epi& last, cudaStream_t s);
// FP64 tensor (natural order) -> its parts in mode-1 layout.
int mixed_split_input(const mm_plan_s* p, const double* V, uint8_t* parts, cudaStream_t s);
// Workspace of mixed_expint / the mixed mumode_phi_apply.
size_t mixed_workspace_bytes(const mm_plan_s* p, int scheme, int gkind);
size_t mixed_mumode_workspace_bytes(const mm_plan_s* p);
// The pointwise part of a nonlinearity descriptor (expint.cu).
PointwiseG pointwise_of(const mm_nonlin* g);
// nsteps of `scheme` in the mixed form; ws laid out as in expint_mixed.cu.
int mixed_expint(mm_plan_s* p, int scheme, const mm_nonlin* g, double* U, double t0, int nsteps,
                 uint8_t* ws, cudaStream_t s);
}  // namespace mm
