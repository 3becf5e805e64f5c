// tucker_apply_noalloc: the FP64 Tucker chain with its intermediate tensor in a
// fixed device array compiled into the library, for callers that cannot
// allocate device memory (see include/phisplit.h).
//
// The intermediate lives in g_noalloc_scratch, a file-scope __device__ array of
// MM_NOALLOC_MAX_ELEMS doubles that every GPU loading this library holds until
// the process exits.  Host code cannot use the symbol itself as a device
// address (on the host it names a shadow variable), so the first call on each
// device, with that device current, resolves the real address once with
// cudaGetSymbolAddress and caches it per device.  No call here allocates.
#include <mutex>

#include "common.cuh"

namespace mm {

namespace {

static __device__ __align__(256) double g_noalloc_scratch[MM_NOALLOC_MAX_ELEMS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
int noalloc_scratch(double** out) {
    int dev = -1;
    MM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return MM_ERR_CUDA;
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return MM_OK;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + nb && y < x + na;
}

}  // namespace

}  // namespace mm

using namespace mm;

extern "C" int tucker_apply_noalloc(int d, const int64_t* n, const double* const* M,
                                    const double* V, double* P, double alpha, void* stream) {
    if (!n || !M || !V || !P || d < 1 || d > MM_MAX_D || !isfinite(alpha)) return MM_ERR_ARG;
    int64_t N = 1;
    for (int mu = 0; mu < d; ++mu) {
        if (n[mu] < 1 || n[mu] > 8192) return MM_ERR_SHAPE;
        if (!M[mu]) return MM_ERR_ARG;
        N *= n[mu];
        if (N > MM_NOALLOC_MAX_ELEMS) return MM_ERR_SHAPE;   // beyond the fixed scratch
    }
    const size_t bytes = (size_t)N * sizeof(double);
    if (ranges_overlap(V, bytes, P, bytes)) return MM_ERR_ARG;
    double* T = nullptr;
    if (d >= 2) {
        int rc = noalloc_scratch(&T);
        if (rc) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Mode d writes P, mode d-1 writes T, earlier modes alternate backwards, so the
    // scratch is always fully written before it is read: nothing needs clearing.
    const double* cur = V;
    for (int mu = 1; mu <= d; ++mu) {
        Epi e{};
        e.kind = EPI_STORE;
        e.alpha = (mu == d) ? alpha : 1.0;
        e.C = (mu == d) ? P : (((d - 1 - mu) % 2 == 0) ? T : P);
        Gemm g = mode_gemm(d, n, mu, M[mu - 1], cur);
        int rc = launch_dgemm(g, e, s);
        if (rc) return rc;
        cur = e.C;
    }
    return MM_OK;
}
