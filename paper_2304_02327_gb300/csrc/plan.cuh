// The plan object behind the opaque mm_plan handle.
#pragma once

#include <vector>

#include "common.cuh"

// One captured run of expint_step: the CUDA graph of its nsteps steps, valid for
// exactly these arguments (every pointer and coefficient is baked into the nodes).
struct mm_graph_cache {
    cudaGraphExec_t exec = nullptr;
    int scheme = -1, nsteps = 0;
    const void* U = nullptr;
    const void* ws = nullptr;
    mm_nonlin g{};
    int has_g = 0;
    double t0 = 0.0;                   // part of the key only for a time-dependent g
    long long launches[MM_KC_COUNT] = {};
};

struct mm_plan_s {
    int d = 0;
    int64_t n[MM_MAX_D] = {};
    int64_t N = 0;
    int ell_max = 0;
    int prec = MM_FP64;
    double tau = 0.0;
    int owner[MM_MAX_D] = {};          // direction whose phi set is shared
    int squarings[MM_MAX_D] = {};
    int tridiag = 1;                   // every A_mu has band width <= 1
    double* A[MM_MAX_D] = {};          // device copy of A_mu (column-major)
    double* diag3[MM_MAX_D] = {};      // [sub | main | super] of A_mu
    double* phi[MM_MAX_D][4] = {};     // phi_l(tau A_mu), FP64, column-major
    // Mixed forms: per direction and l, phi_l(tau A_mu) split into three parts
    // (matrix operand layout of tf32.cuh).
    float* phi_split[MM_MAX_D][4] = {};
    float* coef3f[MM_MAX_D] = {};      // mixed K u stencil: [a | c | row sum] per direction
    float* rem_split[MM_MAX_D] = {};   // mixed, dense A (d = 2): parts of A_mu minus its band
    unsigned int* status = nullptr;    // device status word (MM_STATUS_* bits)
    int use_graphs = 1;                // expint_step replays captured graphs
    cudaStream_t cap = nullptr;        // capture stream of those graphs
    std::vector<mm_graph_cache> graphs;
    std::vector<void*> owned;

    bool alloc(void** p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; return false; }
        owned.push_back(*p);
        return true;
    }
    ~mm_plan_s() {
        for (auto& e : graphs)
            if (e.exec) cudaGraphExecDestroy(e.exec);
        if (cap) cudaStreamDestroy(cap);
        for (void* q : owned) cudaFree(q);
        if (status) cudaFree(status);
    }
};

namespace mm {
// Rows of the matrix view of a state for the Riccati term: the first d/2 directions
// (d = 2: U is n1 x n2; d = 4, the order-4 form of the LQ problem: n1 n2 x n3 n4).
inline int64_t riccati_rows(const mm_plan_s* p) {
    int64_t m = 1;
    for (int mu = 0; mu < p->d / 2; ++mu) m *= p->n[mu];
    return m;
}
// Builds the TF32x3 operand images of the plan's phi matrices (tf32.cu).
int plan_prepare_tf32(mm_plan_s* p, cudaStream_t s);
// phi_0 .. phi_L of tau*A (n x n, column-major, device) into out[0..L] by scaling,
// Taylor series and the squaring recurrence eq. (16) (plan.cu).  colsum_dev: n
// doubles, band_dev: one int (device); *s_out receives the squarings, *band_out the
// band width of A.  scratch: (L + 3) n^2 device doubles, or NULL to allocate.
// Synchronises `s` (the scaling is chosen from the norm on the host).
int form_phis(int n, const double* A, double tau, int L, double* const* out, double* colsum_dev,
              int* band_dev, int* s_out, int* band_out, cudaStream_t s, double* scratch);
}  // namespace mm
