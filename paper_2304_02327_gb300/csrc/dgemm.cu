// FP64 contraction kernel of the plain (MM_FP64) form.
//
// On GB300 the FP64 pipe delivers ~1.1 TFLOP/s against ~6.7 TB/s of HBM, so a
// mu-mode product with n >= 48 is bound by DFMA issue, not by memory (n/8
// flop per byte >> 0.16).  The kernel therefore aims at (a) keeping every SM's
// DFMA pipe busy -- one output tile per CTA, tile size picked so that the grid
// covers the 152 SMs several times over and the block scheduler balances the
// tail -- and (b) never re-reading the big tensor more than once per tile
// column.  Tiles stage through shared memory with coalesced loads along the
// contiguous index of each operand, so the strided middle and last modes need
// no transpose pass: the operand whose contiguous index is the output's row
// index is read directly.
#include "common.cuh"
#include "trace.cuh"

namespace mm {

namespace {

// TWO: two-level summation -- each K-tile's FMA chain (BK terms) is added into a
// separate total, so rounding grows with BK + K/BK instead of K (the plan's
// squaring products, whose errors the squarings amplify).
template <int BM, int BN, int BK, int TM, int TN, bool TWO>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
dgemm_kernel(Gemm g, Epi e, int tilesM, int tilesN) {
    constexpr int TX = BM / TM;
    constexpr int TY = BN / TN;
    constexpr int NT = TX * TY;
    __shared__ double As[BK][BM];
    __shared__ double Bs[BK][BN];

    const int64_t tile = blockIdx.x;
    const int bm = (int)(tile % tilesM);
    const int bn = (int)((tile / tilesM) % tilesN);
    const int64_t bb = tile / ((int64_t)tilesM * tilesN);
    const int m0 = bm * BM, n0 = bn * BN;
    const double* A = g.A + bb * g.sA;
    const double* B = g.B + bb * g.sB;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    double acc[TM][TN], tot[TWO ? TM : 1][TWO ? TN : 1];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    if (TWO) {
#pragma unroll
        for (int i = 0; i < (TWO ? TM : 1); ++i)
#pragma unroll
            for (int j = 0; j < (TWO ? TN : 1); ++j) tot[i][j] = 0.0;
    }

    for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int q = 0; q < (BK * BM) / NT; ++q) {
            int el = tid + q * NT;
            int m = el % BM, k = el / BM;
            int gm = m0 + m, gk = k0 + k;
            As[k][m] = (gm < g.M && gk < g.K) ? A[gm + g.lda * (int64_t)gk] : 0.0;
        }
        if (g.b_kcontig) {
#pragma unroll
            for (int q = 0; q < (BK * BN) / NT; ++q) {
                int el = tid + q * NT;
                int k = el % BK, n = el / BK;
                int gn = n0 + n, gk = k0 + k;
                Bs[k][n] = (gn < g.N && gk < g.K) ? B[gk + g.ldb * (int64_t)gn] : 0.0;
            }
        } else {
#pragma unroll
            for (int q = 0; q < (BK * BN) / NT; ++q) {
                int el = tid + q * NT;
                int n = el % BN, k = el / BN;
                int gn = n0 + n, gk = k0 + k;
                Bs[k][n] = (gn < g.N && gk < g.K) ? B[gn + g.ldb * (int64_t)gk] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + i * TX];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + j * TY];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (TWO) {
#pragma unroll
            for (int i = 0; i < (TWO ? TM : 1); ++i)
#pragma unroll
                for (int j = 0; j < (TWO ? TN : 1); ++j) {
                    tot[i][j] += acc[i][j];
                    acc[i][j] = 0.0;
                }
        }
        __syncthreads();
    }
    if (TWO) {
#pragma unroll
        for (int i = 0; i < (TWO ? TM : 1); ++i)
#pragma unroll
            for (int j = 0; j < (TWO ? TN : 1); ++j) acc[i][j] = tot[i][j];
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int m = m0 + tx + i * TX;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int n = n0 + ty + j * TY;
            if (n >= g.N) continue;
            int64_t off = (int64_t)m + g.ldc * (int64_t)n + bb * g.sC;
            apply_epilogue(e, acc[i][j], off, m, n);
        }
    }
}

template <int BM, int BN, int BK, int TM, int TN, bool TWO>
int launch_cfg(const Gemm& g, const Epi& e, cudaStream_t s) {
    int tilesM = (g.M + BM - 1) / BM, tilesN = (g.N + BN - 1) / BN;
    int64_t ntiles = (int64_t)tilesM * tilesN * g.batch;
    if (ntiles <= 0) return MM_OK;
    if (ntiles > 0x7fffffffLL) return MM_ERR_SHAPE;
    TraceScope tr(KC_CONTRACT_FP64, s);
    dgemm_kernel<BM, BN, BK, TM, TN, TWO><<<(unsigned)ntiles, (BM / TM) * (BN / TN), 0, s>>>(g, e, tilesM, tilesN);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int64_t tiles_of(const Gemm& g, int bm, int bn) {
    return (int64_t)((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * g.batch;
}

}  // namespace

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

int launch_dgemm(const Gemm& g, const Epi& e, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return MM_OK;
    const int64_t sms = num_sms();
    // Largest tile whose grid still fills the machine several times; smaller
    // tiles trade operand reuse (irrelevant when DFMA-bound) for balance.
    // 32 x 32 tiles use 64 threads of 4 x 4 outputs: two FMAs per shared-memory
    // load (2 x 2 outputs would give one, and the shared-memory pipe would bind).
    if (g.two_level) {
        if (tiles_of(g, 64, 64) >= 6 * sms) return launch_cfg<64, 64, 16, 4, 4, true>(g, e, s);
        if (tiles_of(g, 32, 32) >= 3 * sms) return launch_cfg<32, 32, 16, 4, 4, true>(g, e, s);
        return launch_cfg<16, 16, 16, 1, 1, true>(g, e, s);
    }
    if (tiles_of(g, 64, 64) >= 6 * sms) return launch_cfg<64, 64, 16, 4, 4, false>(g, e, s);
    if (tiles_of(g, 32, 32) >= 3 * sms) return launch_cfg<32, 32, 16, 4, 4, false>(g, e, s);
    return launch_cfg<16, 16, 16, 1, 1, false>(g, e, s);
}

Gemm mode_gemm(int d, const int64_t* n, int mu, const double* M, const double* V) {
    int64_t L = 1, R = 1;
    for (int v = 0; v < mu - 1; ++v) L *= n[v];
    for (int v = mu; v < d; ++v) R *= n[v];
    const int64_t nm = n[mu - 1];
    Gemm g{};
    if (L == 1) {
        // Mode 1: Y(i, r) = sum_j M(i, j) V(j, r): a plain column-major GEMM.
        g.M = (int)nm; g.N = (int)R; g.K = (int)nm; g.batch = 1;
        g.A = M; g.lda = nm; g.sA = 0;
        g.B = V; g.ldb = nm; g.sB = 0; g.b_kcontig = 1;
        g.ldc = nm; g.sC = 0;
    } else {
        // Mode mu > 1: for each trailing index r, Y_r(l, i) = sum_j V_r(l, j) M(i, j):
        // the tensor is the (l-contiguous) left operand, M^T the right one.
        g.M = (int)L; g.N = (int)nm; g.K = (int)nm; g.batch = (int)R;
        g.A = V; g.lda = L; g.sA = L * nm;
        g.B = M; g.ldb = nm; g.sB = 0; g.b_kcontig = 0;
        g.ldc = L; g.sC = L * nm;
    }
    return g;
}

}  // namespace mm
