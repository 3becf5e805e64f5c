// Split-precision mu-mode contraction on tcgen05 tensor cores (sm_103a), fed by TMA.
//
// Mode rotation.  Mode mu reads its operand with the contraction index i_mu
// fastest -- fibre ("row") q holds its n_mu values contiguously, rows at a pitch
// p_mu >= n_mu -- and writes its output with the new index i_mu' slowest, in the
// layout the next mode reads: output element (q, i) goes to fibre position
// q mod n_{mu+1} of row q div n_{mu+1} + (R_mu / n_{mu+1}) i.  After d modes the
// order is back to natural (i_1 fastest), so no mode ever reads a strided operand
// and there is no transpose pass: every mode is the same K-major GEMM
//
//   M = 128 rows (TMEM lanes) per tile, N = nc output columns i (<= 128 per CTA),
//   K = n_mu in blocks of one 128-byte swizzle row (32 TF32 or 64 BF16 values).
//
// Split precision.  The operand is stored already split into parts by whoever
// wrote it (the prepass, the previous mode's epilogue, the update pass):
//   TF32x3: x = a0 + a1 (TF32, residual 2^-22), Phi = b0 + b1 + b2, 4 MMAs
//           a0 b0 | a1 b0 + a0 b1 + a0 b2
//   BF16x3: x = a0 + a1 + a2 (BF16, residual ~2^-25), Phi in 3 parts, 6 MMAs
//           a0 b0 | a1 b0 + a0 b1 + a2 b0 + a1 b1 + a0 b2
// The tensor cores' FP32 accumulation truncates toward zero, which biases long
// sums (measured: a one-sided relative error growing with K).  So the main
// product of each K-block goes into a fresh TMEM slot (only its four MMAs
// accumulate in hardware) and the epilogue warps add the slots into FP32 registers
// with round-to-nearest; the much smaller corrections accumulate in TMEM over the
// whole tile.  The three-way split of the fixed matrix keeps its rounding, which
// would repeat identically every step, at 2^-33.
//
// Kernel structure: persistent, one CTA per SM over tiles t = blockIdx.x + i grid.
//   warp 0      loader: per K-block, one TMA tensor load per operand part (the
//               3-D map {K, rows, part} zero-fills the ragged K tail and the last
//               rows) and bulk copies of this tile's columns of the plan's Phi image
//   warp 1      MMA issuer (one thread): per K-block the main product into slot
//               (K-block mod 2) of a two-slot ring, corrections into the tile's
//               accumulator (two, alternating between tiles)
//   warps 2-17  epilogue, four warps per TMEM lane quarter, each owning a quarter
//               of the columns: drain each main slot into register accumulators as
//               it completes (all chunk loads issued before one wait), then add the
//               corrections and write the next mode's split operand (or FP32 after
//               the last mode); the two-slot ring lets the MMAs of the next tile's
//               first K-blocks run meanwhile
// TMEM: [main slot 0 | main slot 1 | corr tile-even | corr tile-odd], nc each.
// Every mbarrier wait is bounded (tcgen05.cuh).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "forms.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "stencil.cuh"
#include "tcgen05.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

namespace {

constexpr int kRows = 128;                 // MMA M / rows per tile
constexpr uint32_t kATile = kRows * 128;   // bytes of one operand part tile (128-byte rows)
constexpr int kMaxStages = 4;
constexpr int kBParts = 3;                 // Phi = b0 + b1 + b2 in both forms
constexpr int kNcMax = 128;                // two sets of [main | corr] fit 512 TMEM columns
constexpr int kBars = 2 * kMaxStages + 9;  // full, empty per stage; main full/empty (slot);
                                           // corr full/empty (tile parity); mma_done
constexpr int kSmemLimit = 227 * 1024;
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kQuartCols = kNcMax / 4;     // columns per epilogue thread (upper bound)

template <class F> __device__ __forceinline__ uint32_t idesc_of(int nc);
template <> __device__ __forceinline__ uint32_t idesc_of<FormTF32>(int nc) { return tc::idesc_tf32(128, nc); }
template <> __device__ __forceinline__ uint32_t idesc_of<FormBF16>(int nc) { return tc::idesc_bf16(128, nc); }

template <class F> __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc);
template <> __device__ __forceinline__ void mma<FormTF32>(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_tf32(d, a, b, id, acc);
}
template <> __device__ __forceinline__ void mma<FormBF16>(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_bf16(d, a, b, id, acc);
}

// Byte offset of element k of `row` in a K-major 128-byte-swizzled tile.
template <class F>
__host__ __device__ __forceinline__ uint32_t sw_off(uint32_t row, uint32_t k) {
    constexpr uint32_t per = 16 / F::kElem;     // elements per 16-byte chunk
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((k / per) ^ (row & 7u)) & 7u) << 4) +
           (k % per) * F::kElem;
}

struct TcMode {
    int n, nkb, nc, splits, stages, n_img;
    int64_t rows, row_tiles;
    const uint8_t* bimg;
    // output: next mode's parts (layout above) or FP32 after the last mode
    int last;
    float* yout;
    uint8_t* pout;           // part q at pout + q * out_part_pitch elements
    int64_t out_part_pitch;  // elements per part
    int next_n, next_p;      // next mode's fibre length and row pitch
    int64_t next_rows_per_i; // R_mu / n_{mu+1}
    unsigned int* status;
};

// 3-D TMA load of one part tile: box {K block, 128 rows} at (k0, row0, part).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int k0, int row0, int part,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(map), "r"(k0), "r"(row0), "r"(part), "r"(bar)
        : "memory");
}


template <class F>
__global__ void __launch_bounds__(kThreads, 1) tc_mode_kernel(TcMode a, const __grid_constant__ CUtensorMap amap) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t b_tile = (uint32_t)a.nc * 128u;
    const uint32_t a_bytes = F::kAParts * kATile;
    const uint32_t stage_bytes = a_bytes + kBParts * b_tile;
    uint64_t* bars = (uint64_t*)(smem + a.stages * stage_bytes);
    uint32_t* tmem_slot = (uint32_t*)(bars + kBars);
    auto full = [&](int s) { return tc::smem_u32(bars + s); };
    auto empty = [&](int s) { return tc::smem_u32(bars + kMaxStages + s); };
    // Parity waits are only sound for a waiter that consumes every phase in order:
    // the "full" barriers are waited only by the epilogue (in K-block / tile
    // order), the "empty" ones only by the MMA thread.
    auto mfull = [&](int r) { return tc::smem_u32(bars + 2 * kMaxStages + r); };
    auto mempty = [&](int r) { return tc::smem_u32(bars + 2 * kMaxStages + 2 + r); };
    auto cfull = [&](int b) { return tc::smem_u32(bars + 2 * kMaxStages + 4 + b); };
    auto cempty = [&](int b) { return tc::smem_u32(bars + 2 * kMaxStages + 6 + b); };
    const uint32_t mma_done = tc::smem_u32(bars + 2 * kMaxStages + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stages = a.stages;
    const int64_t ntiles = a.row_tiles * a.splits;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(mfull(b), 1);
            tc::mbar_init(mempty(b), kEpiWarps);
            tc::mbar_init(cfull(b), 1);
            tc::mbar_init(cempty(b), kEpiWarps);
        }
        tc::mbar_init(mma_done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- loader: operand parts by TMA, Phi columns by bulk copy ----
            int64_t issued_last[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) issued_last[s] = -1;
            const size_t kb_bytes = (size_t)kBParts * a.n_img * 128;   // one K-block of the image
            const int64_t total = my_tiles * a.nkb;
            for (int64_t it = 0; it < total; ++it) {
                const int s = (int)(it % stages);
                if (it >= stages && !tc::mbar_wait(empty(s), (uint32_t)((it / stages) - 1) & 1, a.status)) break;
                const int64_t t = blockIdx.x + (it / a.nkb) * gridDim.x;
                const int kb = (int)(it % a.nkb);
                const int row0 = (int)((t / a.splits) * kRows);
                const int col0 = (int)(t % a.splits) * a.nc;
                tc::mbar_arrive_expect_tx(full(s), a_bytes + kBParts * b_tile);
                const uint32_t st = tc::smem_u32(smem + s * stage_bytes);
                for (int q = 0; q < F::kAParts; ++q)
                    tma_load_3d(st + q * kATile, &amap, kb * F::kBK, row0, q, full(s));
                for (int part = 0; part < kBParts; ++part) {  // b0 rows, b1 rows, b2 rows
                    const uint8_t* src = a.bimg + (size_t)kb * kb_bytes +
                                         (size_t)part * a.n_img * 128 + (size_t)col0 * 128;
                    const uint32_t d0 = st + a_bytes + part * b_tile;
                    for (uint32_t off = 0; off < b_tile; off += 16384) {
                        const uint32_t len = min(16384u, b_tile - off);
                        tc::bulk_g2s(d0 + off, src + off, len, full(s));
                    }
                }
                issued_last[s] = it;
            }
            // never leave the CTA with copies in flight
            for (int s = 0; s < stages; ++s)
                if (issued_last[s] >= 0)
                    tc::mbar_wait(full(s), (uint32_t)(issued_last[s] / stages) & 1, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            const uint32_t id = idesc_of<F>(a.nc);
            int64_t it = 0;
            int64_t uses[2] = {0, 0};      // uses of each main slot so far
            bool ok = true;
            for (int64_t i = 0; i < my_tiles && ok; ++i) {
                const int b = (int)(i & 1);
                if (i >= 2 && !tc::mbar_wait(cempty(b), (uint32_t)((i >> 1) - 1) & 1, a.status)) break;
                const uint32_t corr = tmem + (uint32_t)((2 + b) * a.nc);
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = (int)(it % stages);
                    const int r = (int)(it & 1);
                    if (uses[r] >= 1 && !tc::mbar_wait(mempty(r), (uint32_t)(uses[r] - 1) & 1, a.status)) {
                        ok = false;
                        break;
                    }
                    ++uses[r];
                    if (!tc::mbar_wait(full(s), (uint32_t)(it / stages) & 1, a.status)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t mainacc = tmem + (uint32_t)(r * a.nc);
                    const uint32_t abase = tc::smem_u32(smem + s * stage_bytes);
                    const uint32_t bbase = abase + a_bytes;
#pragma unroll 1
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ko = kk * 32;
                        mma<F>(mainacc, tc::desc_k_sw128(abase + ko), tc::desc_k_sw128(bbase + ko), id, kk != 0);
#pragma unroll
                        for (int c = 0; c < F::kCorr; ++c)
                            mma<F>(corr, tc::desc_k_sw128(abase + F::corr_a(c) * kATile + ko),
                                   tc::desc_k_sw128(bbase + F::corr_b(c) * b_tile + ko), id,
                                   (c == 0 && (kb | kk) == 0) ? 0u : 1u);
                    }
                    tc::mma_commit(empty(s));
                    tc::mma_commit(mfull(r));
                }
                if (ok) tc::mma_commit(cfull(b));
            }
            // every issued MMA has completed before TMEM can be released
            tc::mma_commit(mma_done);
            tc::mbar_wait(mma_done, 0, a.status);
        }
    } else {
        // ---- epilogue: lane quarter (warp mod 4), column quarter ((warp - 2) / 4) ----
        const int quarter = warp & 3;
        const int cq = (warp - 2) >> 2;
        const int r = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int nch = a.nc / 16;                        // <= 8 chunks of 16 columns
        const int c0 = 2 * cq, c1 = min(nch, 2 * cq + 2);
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int b = (int)(i & 1);
            float acc[kQuartCols];
#pragma unroll
            for (int u = 0; u < kQuartCols; ++u) acc[u] = 0.f;
            bool ok = true;
            // main product, one K-block slot at a time, summed in FP32 registers
            for (int kb = 0; kb < a.nkb && ok; ++kb) {
                const int64_t it = i * a.nkb + kb;
                const int rs = (int)(it & 1);
                ok = __all_sync(0xffffffffu, tc::mbar_wait(mfull(rs), (uint32_t)(it >> 1) & 1, a.status));
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t slot = tmem + lane_off + (uint32_t)(rs * a.nc);
#pragma unroll
                for (int c = 0; c < kQuartCols / 16; ++c) {
                    if (c0 + c < c1) {          // warp-uniform
                        uint32_t v[16];
                        tc::tmem_ld16(slot + (uint32_t)((c0 + c) * 16), v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int u = 0; u < 16; ++u) acc[c * 16 + u] += __uint_as_float(v[u]);
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(mempty(rs));
            }
            if (!ok) break;
            ok = __all_sync(0xffffffffu, tc::mbar_wait(cfull(b), (uint32_t)(i >> 1) & 1, a.status));
            if (!ok) break;
            tc::tc_fence_after();
            const int64_t t = blockIdx.x + i * gridDim.x;
            const int64_t q = (t / a.splits) * kRows + r;
            const int col0 = (int)(t % a.splits) * a.nc;
            const bool valid = q < a.rows;
            // next-mode layout of output (q, i): position jq + p' (rq + (R / n') i)
            int64_t jq = 0, rq = 0;
            if (!a.last) { jq = q % a.next_n; rq = q / a.next_n; }
            const uint32_t cset = tmem + lane_off + (uint32_t)((2 + b) * a.nc);
#pragma unroll
            for (int c = 0; c < kQuartCols / 16; ++c) {    // y = corrections + main, in FP32
                if (c0 + c < c1) {
                    uint32_t w[16];
                    tc::tmem_ld16(cset + (uint32_t)((c0 + c) * 16), w);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc[c * 16 + u] += __uint_as_float(w[u]);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(cempty(b));      // corrections read: TMEM set free
            if (!valid) continue;
            // output column col of row q: next-mode position jq + p' (rq + (R / n') col)
            // (or q + R col after the last mode); successive columns step by dpos
            const int64_t dpos = a.last ? a.rows : (int64_t)a.next_p * a.next_rows_per_i;
#pragma unroll
            for (int c = 0; c < kQuartCols / 16; ++c) {
                if (c0 + c >= c1) continue;
                const int i0 = col0 + (c0 + c) * 16;
                int64_t pos = a.last ? q + a.rows * (int64_t)i0
                                     : jq + (int64_t)a.next_p * (rq + a.next_rows_per_i * (int64_t)i0);
                const int lim = min(16, a.n - i0);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (u >= lim) break;
                    const float y = acc[c * 16 + u];
                    if (a.last) a.yout[pos] = y;
                    else store_parts<F>(a.pout, a.out_part_pitch, pos, y, 0.f);
                    pos += dpos;
                }
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Phi image of one K-block: rows i < n_img of kBK values j for each of the three
// parts b0, b1, b2 in turn (Phi = b0 + b1 + b2, each rounded to the form's type
// in turn), K-major, 128-byte swizzled, zero outside the n x n matrix.
template <class F>
__global__ void build_phi_image_kernel(const double* __restrict__ phi, int n, int n_img, int nkb,
                                       uint8_t* __restrict__ img) {
    const int64_t total = (int64_t)nkb * n_img * F::kBK;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % F::kBK);
        const int i = (int)((t / F::kBK) % n_img);
        const int kb = (int)(t / ((int64_t)F::kBK * n_img));
        const int j = kb * F::kBK + c;
        const double v = (i < n && j < n) ? phi[i + (int64_t)n * j] : 0.0;
        uint8_t* blk = img + (size_t)kb * kBParts * n_img * 128;
        const uint32_t off = sw_off<F>(i, c);
        double rr = v;
        for (int part = 0; part < kBParts; ++part) {
            uint8_t* dst = blk + (size_t)part * n_img * 128 + off;
            if (F::kElem == 4) {
                const float bq = mx::tf32((float)rr);
                *(float*)dst = bq;
                rr -= (double)bq;
            } else {
                const __nv_bfloat16 bq = __float2bfloat16_rn((float)rr);
                *(__nv_bfloat16*)dst = bq;
                rr -= (double)__bfloat162float(bq);
            }
        }
    }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Geometry {
    int n, n_img, nkb, nc, splits, stages;
    size_t smem;
};

// Columns per CTA (nc <= 128, one MMA), pipeline depth.
template <class F>
int geometry(int n, Geometry* g) {
    const int n16 = round_up(n, 16);
    if (n16 > 512) return MM_ERR_UNSUPPORTED;
    g->n = n;
    g->nkb = (n + F::kBK - 1) / F::kBK;
    g->splits = (n16 + kNcMax - 1) / kNcMax;
    g->nc = round_up((n16 + g->splits - 1) / g->splits, 16);
    g->n_img = g->splits * g->nc;
    const size_t stage = (size_t)F::kAParts * kATile + kBParts * (size_t)g->nc * 128;
    const size_t fixed = 1024 + kBars * 8 + 16;
    int st = (int)((kSmemLimit - fixed) / stage);
    st = std::min(st, kMaxStages);
    if (st < 2) return MM_ERR_UNSUPPORTED;
    g->stages = st;
    g->smem = fixed + st * stage;
    return MM_OK;
}

int geometry_for(int prec, int n, Geometry* g) {
    return prec == MM_BF16X3 ? geometry<FormBF16>(n, g) : geometry<FormTF32>(n, g);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

template <class F>
int launch_form(const TcMode& m, const PartView& in, size_t smem, int64_t ctas, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        MM_CUDA_TRY(cudaFuncSetAttribute(tc_mode_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemLimit));
        configured = true;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) return MM_ERR_CUDA;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)in.n, (cuuint64_t)in.rows, (cuuint64_t)F::kAParts};
    const cuuint64_t strides[2] = {(cuuint64_t)in.p * F::kElem, (cuuint64_t)in.part_pitch * F::kElem};
    const cuuint32_t box[3] = {(cuuint32_t)F::kBK, (cuuint32_t)kRows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = F::kElem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (enc(&map, dt, 3, (void*)in.base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return MM_ERR_CUDA;
    TraceScope tr(KC_CONTRACT_TF32, s);
    tc_mode_kernel<F><<<(unsigned)ctas, kThreads, smem, s>>>(m, map);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

}  // namespace

int form_elem_bytes(int prec) { return prec == MM_BF16X3 ? FormBF16::kElem : FormTF32::kElem; }
int form_parts(int prec) { return prec == MM_BF16X3 ? FormBF16::kAParts : FormTF32::kAParts; }
int form_pitch(int prec, int n) { return round_up(n, 16 / form_elem_bytes(prec)); }

int plan_prepare_tf32(mm_plan_s* p, cudaStream_t s) {
    if (!encode_fn()) return MM_ERR_UNSUPPORTED;
    for (int mu = 0; mu < p->d; ++mu) {
        Geometry g;
        int rc = geometry_for(p->prec, (int)p->n[mu], &g);
        if (rc) return rc;
        if (p->owner[mu] != mu) {
            for (int l = 0; l <= p->ell_max; ++l) p->phi_split[mu][l] = p->phi_split[p->owner[mu]][l];
            p->coef3f[mu] = p->coef3f[p->owner[mu]];
            continue;
        }
        if (!p->alloc((void**)&p->coef3f[mu], 3 * p->n[mu] * sizeof(float))) return MM_ERR_NOMEM;
        rc = build_stencil_coef(p->A[mu], (int)p->n[mu], p->coef3f[mu], s);
        if (rc) return rc;
        const size_t bytes = (size_t)g.nkb * kBParts * g.n_img * 128;
        const int bk = p->prec == MM_BF16X3 ? FormBF16::kBK : FormTF32::kBK;
        for (int l = 0; l <= p->ell_max; ++l) {
            if (!p->alloc((void**)&p->phi_split[mu][l], bytes)) return MM_ERR_NOMEM;
            const int64_t total = (int64_t)g.nkb * g.n_img * bk;
            const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
            uint8_t* img = (uint8_t*)p->phi_split[mu][l];
            if (p->prec == MM_BF16X3)
                build_phi_image_kernel<FormBF16><<<grid, 256, 0, s>>>(p->phi[mu][l], g.n, g.n_img, g.nkb, img);
            else
                build_phi_image_kernel<FormTF32><<<grid, 256, 0, s>>>(p->phi[mu][l], g.n, g.n_img, g.nkb, img);
            MM_LAUNCH_CHECK();
        }
    }
    return MM_OK;
}

PartView mode_input_view(const mm_plan_s* p, int mu, uint8_t* base) {
    PartView v;
    v.base = base;
    v.n = (int)p->n[mu - 1];
    v.p = form_pitch(p->prec, v.n);
    v.rows = p->N / v.n;
    v.part_pitch = v.rows * v.p;
    return v;
}

size_t part_set_bytes(const mm_plan_s* p) {
    size_t mxb = 0;
    for (int mu = 1; mu <= p->d; ++mu) {
        const PartView v = mode_input_view(p, mu, nullptr);
        const size_t b = (size_t)form_parts(p->prec) * (size_t)v.part_pitch * form_elem_bytes(p->prec);
        mxb = std::max(mxb, (b + 255) / 256 * 256);
    }
    return mxb;
}

int tc_mode_product(mm_plan_s* p, int ell, int mu, const PartView& in, uint8_t* out_parts, float* yout,
                    cudaStream_t s) {
    Geometry g;
    int rc = geometry_for(p->prec, (int)p->n[mu - 1], &g);
    if (rc) return rc;
    TcMode m{};
    m.n = g.n; m.nkb = g.nkb; m.nc = g.nc; m.splits = g.splits; m.stages = g.stages; m.n_img = g.n_img;
    m.rows = p->N / g.n;
    m.row_tiles = (m.rows + kRows - 1) / kRows;
    m.bimg = (const uint8_t*)p->phi_split[mu - 1][ell];
    m.status = p->status;
    m.last = mu == p->d;
    if (m.last) {
        m.yout = yout;
    } else {
        const PartView nx = mode_input_view(p, mu + 1, out_parts);
        m.pout = out_parts;
        m.out_part_pitch = nx.part_pitch;
        m.next_n = nx.n;
        m.next_p = nx.p;
        m.next_rows_per_i = m.rows / nx.n;
    }
    if (m.rows > 0x7fffffffLL) return MM_ERR_SHAPE;
    const int64_t tiles = m.row_tiles * g.splits;
    const int64_t ctas = std::min<int64_t>(tiles, num_sms());
    if (p->prec == MM_BF16X3) return launch_form<FormBF16>(m, in, g.smem, ctas, s);
    return launch_form<FormTF32>(m, in, g.smem, ctas, s);
}

int tf32_supported(int prec, int n) {
    Geometry g;
    return geometry_for(prec, n, &g);
}

}  // namespace mm
