// phi_plan: FP64 formation of phi_l(tau A_mu), l = 0..ell_max, on the GPU.
//
// Section 3.1 forms phi_l of the small matrices by scaling X = tau A to
// X / 2^s, evaluating there, and undoing the scaling with the squaring
// recurrence eq. (16),
//     phi_l(2z) = 2^-l [ e^z phi_l(z) + sum_{k=1..l} phi_k(z) / (l-k)! ],
// which needs all phi_j, j <= l, at every squaring and so yields them all.
// The paper evaluates the scaled functions by Gauss-Lobatto quadrature of
// eq. (4a); here the scaled phi_L (L = ell_max) is the truncated Taylor series
// of eq. (4b), evaluated by Paterson-Stockmeyer blocks of four (Horner for L = 0),
// and phi_{l-1}(Y) = Y phi_l(Y) + I/(l-1)! gives the lower ones.  With ||Y||_1 <= 1 and 18 Taylor terms the truncation is below
// 1/19! ~ 8e-18 relative to ||phi_L||, so every phi_l(Y) is exact to rounding
// (the terms Y^i/(i+L)! never exceed 1/L!, so the alternating sum of a
// dissipative Y cancels little).  Scaling to 1 rather than lower keeps the
// number of squarings, whose rounding the later squarings amplify, to the
// minimum; all products run through the FP64 contraction kernel with two-level
// summation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "plan.cuh"
#include "trace.cuh"

namespace mm {

namespace {

constexpr int kTaylorTerms = 18;

__global__ void scale_copy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                  double a, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = a * src[i];
}

// dst = w1 D1 + w2 D2 + diag I (n x n)
__global__ void lincomb_kernel(double* __restrict__ dst, const double* __restrict__ D1, double w1,
                               const double* __restrict__ D2, double w2, double diag, int n) {
    int64_t count = (int64_t)n * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = w1 * D1[i] + w2 * D2[i] + ((i % n == i / n) ? diag : 0.0);
}

__global__ void fill_identity_kernel(double* dst, int n, double v) {
    int64_t count = (int64_t)n * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (i % n == i / n) ? v : 0.0;
}

// Column j: colsum[j] = sum_i |A(i, j)|; band = max |i - j| over A(i, j) != 0.
__global__ void colsum_band_kernel(const double* __restrict__ A, int n, double* colsum, int* band) {
    int j = blockIdx.x;
    double s = 0.0;
    int b = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = A[i + (int64_t)n * j];
        s += fabs(v);
        if (v != 0.0) b = max(b, abs(i - j));
    }
    __shared__ double ss[256];
    __shared__ int sb[256];
    ss[threadIdx.x] = s;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sb[threadIdx.x] = max(sb[threadIdx.x], sb[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        colsum[j] = ss[0];
        atomicMax(band, sb[0]);
    }
}

__global__ void compare_kernel(const double* __restrict__ a, const double* __restrict__ b,
                               int64_t count, int* differ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) *differ = 1;
}

// diag3 = [sub | main | super] of a column-major n x n matrix (zero-padded ends).
__global__ void extract_tridiag_kernel(const double* __restrict__ A, int n, double* diag3) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        diag3[i] = i > 0 ? A[i + (int64_t)n * (i - 1)] : 0.0;
        diag3[n + i] = A[i + (int64_t)n * i];
        diag3[2 * n + i] = i + 1 < n ? A[i + (int64_t)n * (i + 1)] : 0.0;
    }
}

int grid_for(int64_t count) {
    int64_t b = (count + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// C = alpha*A*B + beta*D1 + gamma*D2 + delta*D3 + diag*I for n x n column-major.
int square_gemm(int n, const double* A, const double* B, double* C, double alpha,
                const double* D1, double beta, const double* D2, double gamma,
                const double* D3, double delta, double diag, cudaStream_t s) {
    Gemm g{};
    g.M = n; g.N = n; g.K = n; g.batch = 1;
    g.A = A; g.lda = n;
    g.B = B; g.ldb = n; g.b_kcontig = 1;
    g.ldc = n;
    g.two_level = 1;
    Epi e{};
    e.kind = EPI_STORE;
    e.alpha = alpha; e.beta = beta; e.gamma = gamma; e.delta = delta; e.diag = diag;
    e.D1 = D1; e.D2 = D2; e.D3 = D3; e.C = C;
    return launch_dgemm(g, e, s);
}

double fact(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

}  // namespace

// phi_0..phi_L of X = tau*A (A column-major n x n on the device) into out[0..L].
// scratch: (L + 3) n^2 doubles of device memory, or NULL to allocate them here.
int form_phis(int n, const double* A, double tau, int L, double* const* out, double* colsum_dev,
              int* band_dev, int* s_out, int* band_out, cudaStream_t s, double* scratch) {
    const int64_t nn = (int64_t)n * n;
    std::vector<double*> tmp(L + 3, nullptr);
    const bool own = scratch == nullptr;
    for (int i = 0; i < L + 3; ++i) {
        if (!own) {
            tmp[i] = scratch + i * nn;
        } else if (cudaMalloc(&tmp[i], nn * sizeof(double)) != cudaSuccess) {
            for (auto q : tmp) if (q) cudaFree(q);
            return MM_ERR_NOMEM;
        }
    }
    int rc = MM_OK;
    double* Y = tmp[L + 1];
    double* H = tmp[L + 2];
    std::vector<double> colsum(n);
    int band = 0;
    // 1-norm of tau*A and the band width of A.
    MM_CUDA_TRY(cudaMemsetAsync(band_dev, 0, sizeof(int), s));
    colsum_band_kernel<<<n, 256, 0, s>>>(A, n, colsum_dev, band_dev);
    MM_LAUNCH_CHECK();
    MM_CUDA_TRY(cudaMemcpyAsync(colsum.data(), colsum_dev, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    MM_CUDA_TRY(cudaMemcpyAsync(&band, band_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    MM_CUDA_TRY(cudaStreamSynchronize(s));
    double norm1 = 0.0;
    for (int j = 0; j < n; ++j) norm1 = fmax(norm1, colsum[j]);
    norm1 *= fabs(tau);
    if (!isfinite(norm1)) { rc = MM_ERR_ARG; goto done; }
    {
        int sq = 0;
        while (sq < 1000 && ldexp(norm1, -sq) > 1.0) ++sq;
        *s_out = sq;
        *band_out = band;
        // Y = tau A / 2^s
        scale_copy_kernel<<<grid_for(nn), 256, 0, s>>>(A, Y, ldexp(tau, -sq), nn);
        MM_LAUNCH_CHECK();
        // phi_L(Y) = sum_{i=0}^{T} c_i Y^i, c_i = 1/(i+L)!
        double* P = out[L];
        if (L == 0) {
            // Horner: P <- Y P + c_i I
            fill_identity_kernel<<<grid_for(nn), 256, 0, s>>>(P, n, 1.0 / fact(kTaylorTerms + L));
            MM_LAUNCH_CHECK();
            for (int i = kTaylorTerms - 1; i >= 0; --i) {
                rc = square_gemm(n, Y, P, H, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 1.0 / fact(i + L), s);
                if (rc) goto done;
                double* t = P; P = H; H = t;
            }
        } else {
            // Paterson-Stockmeyer in blocks of four (7 products instead of 18): with
            // B_j = sum_{k<4} c_{4j+k} Y^k, phi_L = B_0 + Y^4 (B_1 + Y^4 (B_2 + Y^4 (B_3 + Y^4 B_4))),
            // each step one product whose epilogue adds B_j.  Y^2, Y^3, Y^4 live in buffers
            // free until the lower phi are formed (tmp[0], tmp[1], and tmp[2] or out[0]).
            static_assert(kTaylorTerms == 18, "the blocks below cover c_0 .. c_18");
            double* Y2 = tmp[0];
            double* Y3 = tmp[1];
            double* Y4 = L >= 2 ? tmp[2] : out[0];
            auto c = [&](int i) { return i <= kTaylorTerms ? 1.0 / fact(i + L) : 0.0; };
            rc = square_gemm(n, Y, Y, Y2, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0.0, s);
            if (!rc) rc = square_gemm(n, Y, Y2, Y3, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0.0, s);
            if (!rc) rc = square_gemm(n, Y2, Y2, Y4, 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 0.0, s);
            if (rc) goto done;
            lincomb_kernel<<<grid_for(nn), 256, 0, s>>>(P, Y, c(17), Y2, c(18), c(16), n);   // B_4
            MM_LAUNCH_CHECK();
            for (int j = 3; j >= 0; --j) {
                rc = square_gemm(n, Y4, P, H, 1.0, Y, c(4 * j + 1), Y2, c(4 * j + 2), Y3, c(4 * j + 3),
                                 c(4 * j), s);
                if (rc) goto done;
                double* t = P; P = H; H = t;
            }
        }
        if (P != out[L]) {
            MM_CUDA_TRY(cudaMemcpyAsync(out[L], P, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
            H = P;
        }
        // phi_{l-1}(Y) = Y phi_l(Y) + I/(l-1)!
        for (int l = L; l >= 1; --l) {
            rc = square_gemm(n, Y, out[l], out[l - 1], 1.0, nullptr, 0, nullptr, 0, nullptr, 0, 1.0 / fact(l - 1), s);
            if (rc) goto done;
        }
        // s squarings, eq. (16): new phi_l = 2^-l [phi_0 phi_l + sum_{k=1}^{l} phi_k/(l-k)!]
        double* cur[4];
        double* nxt[4];
        for (int l = 0; l <= L; ++l) { cur[l] = out[l]; nxt[l] = tmp[l]; }
        for (int it = 0; it < sq; ++it) {
            for (int l = 0; l <= L; ++l) {
                const double sc = ldexp(1.0, -l);
                // the sum has l terms phi_k/(l-k)!, k = 1..l; with L <= 3 at most three
                const double* D[3] = {nullptr, nullptr, nullptr};
                double w[3] = {0, 0, 0};
                for (int k = 1; k <= l; ++k) { D[k - 1] = cur[k]; w[k - 1] = sc / fact(l - k); }
                rc = square_gemm(n, cur[0], cur[l], nxt[l], sc, D[0], w[0], D[1], w[1], D[2], w[2], 0.0, s);
                if (rc) goto done;
            }
            for (int l = 0; l <= L; ++l) { double* t = cur[l]; cur[l] = nxt[l]; nxt[l] = t; }
        }
        for (int l = 0; l <= L; ++l)
            if (cur[l] != out[l])
                MM_CUDA_TRY(cudaMemcpyAsync(out[l], cur[l], nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
        MM_CUDA_TRY(cudaStreamSynchronize(s));
    }
done:
    if (own)
        for (auto p : tmp) cudaFree(p);
    return rc;
}

}  // namespace mm

using namespace mm;

extern "C" int phi_plan_create(mm_plan* out, int d, const int64_t* n, const double* const* A,
                               double tau, int ell_max, int prec, void* stream) {
    NvtxScope nv("phi_plan_create");
    if (!out) return MM_ERR_ARG;
    *out = nullptr;
    if (!n || !A || d < 1 || d > MM_MAX_D || ell_max < 0 || ell_max > 3 || !isfinite(tau))
        return MM_ERR_ARG;
    if (prec != MM_FP64 && prec != MM_TF32X3 && prec != MM_BF16X3) return MM_ERR_ARG;
    int64_t N = 1;
    for (int mu = 0; mu < d; ++mu) {
        if (n[mu] < 1 || n[mu] > 8192) return MM_ERR_SHAPE;
        if (!A[mu]) return MM_ERR_ARG;
        N *= n[mu];
    }
    if (N >= (int64_t(1) << 40)) return MM_ERR_SHAPE;
    cudaStream_t s = (cudaStream_t)stream;

    mm_plan_s* p = new mm_plan_s();
    p->d = d; p->N = N; p->ell_max = ell_max; p->prec = prec; p->tau = tau;
    for (int mu = 0; mu < d; ++mu) p->n[mu] = n[mu];
    int rc = MM_OK;
    int64_t nmax = 0;
    for (int mu = 0; mu < d; ++mu) nmax = n[mu] > nmax ? n[mu] : nmax;
    double* colsum = nullptr;
    int* flag = nullptr;
    if (cudaMalloc(&colsum, nmax * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&flag, 2 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->status, sizeof(unsigned int)) != cudaSuccess) {
        rc = MM_ERR_NOMEM;
        goto fail;
    }
    if (cudaMemsetAsync(p->status, 0, sizeof(unsigned int), s) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
    p->tridiag = 1;
    for (int mu = 0; mu < d; ++mu) {
        const int64_t nn = n[mu] * n[mu];
        // Share the phi matrices of an earlier direction with a bitwise-equal A.
        int owner = mu;
        for (int nu = 0; nu < mu && owner == mu; ++nu) {
            if (p->owner[nu] != nu || n[nu] != n[mu]) continue;
            if (A[nu] == A[mu]) { owner = nu; break; }
            int differ = 0;
            if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
            compare_kernel<<<grid_for(nn), 256, 0, s>>>(A[nu], A[mu], nn, flag);
            if (cudaMemcpyAsync(&differ, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
            if (!differ) owner = nu;
        }
        p->owner[mu] = owner;
        if (owner != mu) {
            p->A[mu] = p->A[owner];
            p->diag3[mu] = p->diag3[owner];
            for (int l = 0; l <= ell_max; ++l) p->phi[mu][l] = p->phi[owner][l];
            p->squarings[mu] = p->squarings[owner];
            continue;
        }
        if (!p->alloc((void**)&p->A[mu], nn * sizeof(double)) ||
            !p->alloc((void**)&p->diag3[mu], 3 * n[mu] * sizeof(double))) { rc = MM_ERR_NOMEM; goto fail; }
        if (cudaMemcpyAsync(p->A[mu], A[mu], nn * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = MM_ERR_CUDA; goto fail;
        }
        for (int l = 0; l <= ell_max; ++l)
            if (!p->alloc((void**)&p->phi[mu][l], nn * sizeof(double))) { rc = MM_ERR_NOMEM; goto fail; }
        int band = 0;
        rc = form_phis((int)n[mu], p->A[mu], tau, ell_max, p->phi[mu], colsum, flag + 1,
                       &p->squarings[mu], &band, s, nullptr);
        if (rc) goto fail;
        if (band > 1) p->tridiag = 0;
        extract_tridiag_kernel<<<grid_for(n[mu]), 256, 0, s>>>(p->A[mu], (int)n[mu], p->diag3[mu]);
        if (cudaGetLastError() != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
    }
    if (prec == MM_TF32X3 || prec == MM_BF16X3) {
        rc = plan_prepare_tf32(p, s);
        if (rc) goto fail;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
    cudaFree(colsum);
    cudaFree(flag);
    *out = p;
    return MM_OK;
fail:
    if (colsum) cudaFree(colsum);
    if (flag) cudaFree(flag);
    delete p;
    return rc;
}

extern "C" int phi_plan_destroy(mm_plan p) {
    if (!p) return MM_OK;
    cudaDeviceSynchronize();
    delete p;
    return MM_OK;
}

extern "C" int phi_plan_info(mm_plan p, int* d, int64_t* n, int* ell_max, int* prec,
                             int* squarings, int* tridiagonal) {
    if (!p) return MM_ERR_ARG;
    if (d) *d = p->d;
    if (n) for (int mu = 0; mu < p->d; ++mu) n[mu] = p->n[mu];
    if (ell_max) *ell_max = p->ell_max;
    if (prec) *prec = p->prec;
    if (squarings) for (int mu = 0; mu < p->d; ++mu) squarings[mu] = p->squarings[mu];
    if (tridiagonal) *tridiagonal = p->tridiag;
    return MM_OK;
}

extern "C" int phi_plan_get_phi(mm_plan p, int ell, int mu, double* dst, void* stream) {
    if (!p || !dst || ell < 0 || ell > p->ell_max || mu < 1 || mu > p->d) return MM_ERR_ARG;
    const int64_t nn = p->n[mu - 1] * p->n[mu - 1];
    MM_CUDA_TRY(cudaMemcpyAsync(dst, p->phi[mu - 1][ell], nn * sizeof(double),
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MM_OK;
}

extern "C" int phi_plan_status(mm_plan p, int reset, void* stream) {
    if (!p) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int v = 0;
    MM_CUDA_TRY(cudaMemcpyAsync(&v, p->status, sizeof(v), cudaMemcpyDeviceToHost, s));
    MM_CUDA_TRY(cudaStreamSynchronize(s));
    if (reset) {
        MM_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(unsigned int), s));
        MM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return (int)v;
}

extern "C" const char* mm_status_str(int code) {
    switch (code) {
    case MM_OK: return "ok";
    case MM_ERR_ARG: return "invalid argument";
    case MM_ERR_SHAPE: return "invalid shape";
    case MM_ERR_UNSUPPORTED: return "unsupported request";
    case MM_ERR_CUDA: return "CUDA runtime error";
    case MM_ERR_TIMEOUT: return "bounded device wait timed out";
    case MM_ERR_NONFINITE: return "non-finite value produced";
    case MM_ERR_NOMEM: return "device allocation failed";
    case MM_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
    }
}

extern "C" int mm_version(void) { return 100; }
