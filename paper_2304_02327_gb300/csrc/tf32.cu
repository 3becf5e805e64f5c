// TF32x3 mu-mode contraction on tcgen05 tensor cores (sm_103a).
//
// One mode product Y[l, i, r] = sum_j Phi[i, j] V[l, j, r] is a GEMM whose rows are
// the fibres of V along direction mu: row q = (l, r) with l = q mod L, r = q div L,
// fibre element j at V[l + L j + L n r].  Flattening the rows this way makes every
// mode -- the contiguous first, the strided middle and the last -- the same
// 128-row-tile GEMM with no ragged middle tiles and no transpose pass:
//
//   MMA M = 128 rows (TMEM lanes), MMA N = Nc output columns i (all n of them, or
//   half when n > 256), K = n inputs j in blocks of 32 (one 128-byte swizzle row).
//
// Split precision: the tensor operand is x = x_hi + x_lo with x_hi = rn_tf32(x),
// x_lo = rn_tf32(x - x_hi) (residual <= 2^-22 |x|, a different pattern every
// step); the fixed matrix is split three ways, Phi = b0 + b1 + b2 (residual
// 2^-33), because its rounding error would otherwise repeat identically every
// step and grow linearly over a run.  The products x_hi*b0 go to G accumulators,
// one per contiguous group of K-blocks, and the corrections x_lo*b0 + x_hi*b1 +
// x_hi*b2 to one more; the epilogue adds the G + 1 FP32 partial sums.  Keeping
// the small corrections out of the main sum and restarting it every few K-blocks
// cuts the number of roundings of a full-magnitude FP32 sum per output from
// 4n/8 to about n/(8G), which is what bounds a long FP32 accumulation.
//
// The Phi operand is split once by the plan into the exact shared-memory image
// the MMA reads and streamed per K-block with bulk async copies (the TMA engine).
// The V operand is loaded by four producer warps a K-block ahead into registers
// (coalesced: along rows for strided modes, along the fibre for the contiguous
// one), split, and stored K-major with the 128-byte swizzle.  One thread issues
// the MMAs; all eight warps then drain TMEM and either store FP32 (intermediate
// modes) or run the FP64 integrator epilogue (last mode).
#include <cuda_bf16.h>

#include <algorithm>

#include "mixed.cuh"
#include "plan.cuh"
#include "stencil.cuh"
#include "tcgen05.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

namespace {

constexpr int kRows = 128;                 // MMA M / rows per CTA tile
constexpr uint32_t kATile = kRows * 128;   // bytes of one A tile part (128 B rows)
constexpr int kMaxStages = 4;
constexpr int kMaxGroups = 4;
constexpr int kBParts = 3;                 // Phi = b0 + b1 + b2 in both forms
constexpr int kSmemLimit = 227 * 1024;

// The two split-precision forms.  A K-block is one 128-byte swizzle row of
// operand elements; every MMA consumes 32 bytes of K (8 TF32 or 16 BF16).
//   TF32x3: x = a0 + a1 (TF32, residual 2^-22), Phi 3 parts, products
//           a0 b0 | a1 b0 + a0 b1 + a0 b2                          (4 MMAs)
//   BF16x3: x = a0 + a1 + a2 (BF16, residual ~2^-25), Phi 3 parts, products
//           a0 b0 | a1 b0 + a0 b1 + a2 b0 + a1 b1 + a0 b2          (6 MMAs)
// The main product a0 b0 goes to the K-grouped accumulators, the rest to one
// correction accumulator.
struct FormTF32 {
    static constexpr int kElem = 4, kBK = 32, kAParts = 2, kNcMax = 192;
    static constexpr int kCorr = 3;
    __host__ __device__ static constexpr int corr_a(int c) { return c == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int corr_b(int c) { return c == 0 ? 0 : c; }
};
struct FormBF16 {
    static constexpr int kElem = 2, kBK = 64, kAParts = 3, kNcMax = 160;
    static constexpr int kCorr = 5;
    __host__ __device__ static constexpr int corr_a(int c) { return c == 0 ? 1 : c == 2 ? 2 : c == 3 ? 1 : 0; }
    __host__ __device__ static constexpr int corr_b(int c) { return c == 1 ? 1 : c == 3 ? 1 : c == 4 ? 2 : 0; }
};

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

struct Tf32Mode {
    int n, n_pad, nkb, nc, splits, groups, stages;   // n_pad: image rows per half (splits * nc)
    int64_t L, rows;
    const void* in;
    float* out;
    const uint8_t* bimg;
    uint32_t tmem_cols;
    unsigned int* status;
};

// Split one operand value into the form's parts, as 32-bit patterns (TF32 in an
// FP32 container) or 16-bit patterns (BF16) in the low half.
template <class F> __device__ __forceinline__ void split_parts(float x, float xl, uint32_t (&p)[3]);
template <> __device__ __forceinline__ void split_parts<FormTF32>(float x, float xl, uint32_t (&p)[3]) {
    const float h = mx::tf32(x);
    const float l = mx::tf32((x - h) + xl);
    p[0] = __float_as_uint(h); p[1] = __float_as_uint(l); p[2] = 0;
}
template <> __device__ __forceinline__ void split_parts<FormBF16>(float x, float xl, uint32_t (&p)[3]) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
    const float r1 = (x - __bfloat162float(b0)) + xl;
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    p[0] = __bfloat16_as_ushort(b0); p[1] = __bfloat16_as_ushort(b1); p[2] = __bfloat16_as_ushort(b2);
}
template <class F> __device__ __forceinline__ void split_val(float x, uint32_t (&p)[3]) { split_parts<F>(x, 0.f, p); }
template <class F> __device__ __forceinline__ void split_val(double x, uint32_t (&p)[3]) {
    float a, b;
    mx::d2ff(x, a, b);
    split_parts<F>(a, b, p);
}

__device__ __forceinline__ void flag_nonfinite_bits(const Epi& e, double v) {
    if (!mx::finite_bits(v) && e.status) atomicOr(e.status, MM_STATUS_NONFINITE);
}

// Last-mode epilogue of the mixed form, 16 consecutive output columns of one
// row: the state update in FP64 (one DFMA per element), everything else in FP32.
// The state values are loaded into registers first, so the loads are not
// serialised behind the stores.
__device__ __forceinline__ void mixed_epilogue16(const Epi& e, const float (&y)[16], int64_t base,
                                                 int i0, int n, int64_t L, float alphaf, float t0f,
                                                 float t1f) {
    if (e.kind == EPI_STORE) {
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (i0 + t < n) e.C[base + (int64_t)(i0 + t) * L] = e.alpha * mx::f2d(y[t]);
        return;
    }
    const double* src = (e.kind == EPI_EE || e.kind == EPI_ETD_S1) ? e.U : e.U2;
    double u[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) u[t] = (i0 + t < n) ? __ldg(src + base + (int64_t)(i0 + t) * L) : 0.0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        if (i0 + t >= n) continue;
        const int64_t off = base + (int64_t)(i0 + t) * L;
        switch (e.kind) {
        case EPI_EE:
        case EPI_ETD_S2: {
            const double v = fma(e.alpha, mx::f2d(y[t]), u[t]);
            flag_nonfinite_bits(e, v);
            e.U[off] = v;
            break;
        }
        case EPI_ETD_S1: {
            e.U2[off] = fma(e.alpha, mx::f2d(y[t]), u[t]);
            float uh, ul;
            mx::d2ff(u[t], uh, ul);
            e.W2f[off] = mx::dg32(e.g, uh + ul, alphaf * y[t], t0f, t1f, off);
            break;
        }
        case EPI_LAWSON2: {
            float uh, ul;
            mx::d2ff(u[t], uh, ul);
            const float gv = (float)e.beta * mx::g32(e.g, uh + ul, t1f, off);
            const double v = fma(e.alpha, mx::f2d(y[t]), mx::f2d(gv));
            flag_nonfinite_bits(e, v);
            e.U[off] = v;
            break;
        }
        default: break;
        }
    }
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// The producer's register stage: one K-block slice of the A operand (kBK values
// per row of the 128-row tile).
//   strided modes (L > 1): thread r owns row r, values along j (each load
//     instruction of a warp covers 32 consecutive rows: coalesced);
//   contiguous mode (L == 1): thread t owns runs of 8 consecutive j of several
//     rows, so each load instruction covers whole row segments.
template <class F, typename TIn>
struct AStage {
    static constexpr int kVals = F::kBK;            // values per thread per K-block
    static constexpr int kRun = 8;                   // contiguous-mode run length
    static constexpr int kRunsPerRow = F::kBK / kRun;
    static constexpr int kRowStep = 128 / kRunsPerRow;
    TIn v[kVals];

    __device__ __forceinline__ void load(const Tf32Mode& a, const TIn* __restrict__ in, int64_t q0,
                                         int kb, int tid) {
        const int j0 = kb * F::kBK;
        if (a.L > 1) {
            const int64_t q = q0 + tid;
            const bool valid = q < a.rows;
            const int64_t base = valid ? (q % a.L) + (q / a.L) * a.L * a.n : 0;
#pragma unroll
            for (int t = 0; t < kVals; ++t) {
                const int j = j0 + t;
                v[t] = (valid && j < a.n) ? __ldg(in + base + (int64_t)j * a.L) : (TIn)0;
            }
        } else {
            const int c = tid % kRunsPerRow, rg = tid / kRunsPerRow;
#pragma unroll
            for (int i = 0; i < kVals / kRun; ++i) {
                const int64_t q = q0 + rg + kRowStep * i;
                const int j = j0 + c * kRun;
#pragma unroll
                for (int e = 0; e < kRun; ++e)
                    v[i * kRun + e] = (q < a.rows && j + e < a.n) ? __ldg(in + q * a.n + j + e) : (TIn)0;
            }
        }
    }

    // Split and store: each 16-byte chunk of every part is written at once.
    __device__ __forceinline__ void store(const Tf32Mode& a, uint8_t* const (&parts)[3], int tid) const {
        constexpr int per = 16 / F::kElem;               // elements per 16-byte chunk
        if (a.L > 1) {
#pragma unroll
            for (int c = 0; c < kVals / per; ++c) store_chunk(parts, tid, c * per, &v[c * per]);
        } else {
            const int c = tid % kRunsPerRow, rg = tid / kRunsPerRow;
#pragma unroll
            for (int i = 0; i < kVals / kRun; ++i)
#pragma unroll
                for (int h = 0; h < kRun / per; ++h)
                    store_chunk(parts, rg + kRowStep * i, c * kRun + h * per, &v[i * kRun + h * per]);
        }
    }

    __device__ __forceinline__ static void store_chunk(uint8_t* const (&parts)[3], int row, int k0,
                                                       const TIn* x) {
        constexpr int per = 16 / F::kElem;
        uint32_t w[3][4] = {};
#pragma unroll
        for (int e = 0; e < per; ++e) {
            uint32_t pp[3];
            split_val<F>(x[e], pp);
#pragma unroll
            for (int q = 0; q < F::kAParts; ++q) {
                if (F::kElem == 4) w[q][e] = pp[q];
                else w[q][e >> 1] |= pp[q] << (16 * (e & 1));
            }
        }
        const uint32_t off = sw_off<F>(row, k0);
#pragma unroll
        for (int q = 0; q < F::kAParts; ++q)
            *(uint4*)(parts[q] + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
};

template <class F, typename TIn, bool LAST>
__global__ void __launch_bounds__(256, 1) tc_mode_kernel(Tf32Mode a, Epi e) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t b_tile = (uint32_t)a.nc * 128u;
    const uint32_t a_bytes = F::kAParts * kATile;
    const uint32_t stage_bytes = a_bytes + kBParts * b_tile;
    uint64_t* bars = (uint64_t*)(smem + a.stages * stage_bytes);
    uint32_t* tmem_slot = (uint32_t*)(bars + 3 * kMaxStages + 1);
    auto full = [&](int s) { return tc::smem_u32(bars + s); };
    auto bfull = [&](int s) { return tc::smem_u32(bars + kMaxStages + s); };
    auto empty = [&](int s) { return tc::smem_u32(bars + 2 * kMaxStages + s); };
    const uint32_t accum = tc::smem_u32(bars + 3 * kMaxStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = (int)(blockIdx.x % a.splits);                 // column slice of this CTA
    const int64_t q0 = (int64_t)(blockIdx.x / a.splits) * kRows;
    const int col0 = h * a.nc;                                   // first output column i
    const int stages = a.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            tc::mbar_init(full(s), 128);
            tc::mbar_init(bfull(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        tc::mbar_init(accum, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), a.tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ---- producers: K-block kb+1 is in flight while kb is split and stored ----
        const int tid = threadIdx.x;
        const TIn* __restrict__ in = (const TIn*)a.in;
        AStage<F, TIn> st;
        st.load(a, in, q0, 0, tid);
        for (int kb = 0; kb < a.nkb; ++kb) {
            const int s = kb % stages;
            if (kb >= stages && !tc::mbar_wait(empty(s), ((kb / stages) - 1) & 1, a.status)) break;
            uint8_t* base = smem + s * stage_bytes;
            uint8_t* const parts[3] = {base, base + kATile, base + 2 * kATile};
            st.store(a, parts, tid);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(full(s));
            if (kb + 1 < a.nkb) st.load(a, in, q0, kb + 1, tid);
        }
    } else if (warp == 4) {
        if (lane == 0) {
            // ---- Phi loader: this CTA's rows of the plan's pre-split image ----
            int issued_last[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) issued_last[s] = -1;
            const size_t kb_bytes = (size_t)kBParts * a.n_pad * 128;   // one K-block of the image
            for (int kb = 0; kb < a.nkb; ++kb) {
                const int s = kb % stages;
                if (kb >= stages && !tc::mbar_wait(empty(s), ((kb / stages) - 1) & 1, a.status)) break;
                tc::mbar_arrive_expect_tx(bfull(s), kBParts * b_tile);
                const uint32_t dst = tc::smem_u32(smem + s * stage_bytes + a_bytes);
                for (int part = 0; part < kBParts; ++part) {  // b0 rows, b1 rows, b2 rows
                    const uint8_t* src = a.bimg + (size_t)kb * kb_bytes +
                                         (size_t)part * a.n_pad * 128 + (size_t)col0 * 128;
                    const uint32_t d0 = dst + part * b_tile;
                    for (uint32_t off = 0; off < b_tile; off += 16384) {
                        const uint32_t len = min(16384u, b_tile - off);
                        tc::bulk_g2s(d0 + off, src + off, len, bfull(s));
                    }
                }
                issued_last[s] = kb;
            }
            // never leave the CTA with copies in flight
            for (int s = 0; s < stages; ++s)
                if (issued_last[s] >= 0) tc::mbar_wait(bfull(s), (issued_last[s] / stages) & 1, a.status);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // ---- MMA issuer: a0 b0 into accumulator group g, corrections into the last ----
            bool started[kMaxGroups] = {false, false, false, false};
            const uint32_t corr = tmem + (uint32_t)(a.groups * a.nc);
            const uint32_t id = idesc_of<F>(a.nc);
            for (int kb = 0; kb < a.nkb; ++kb) {
                const int s = kb % stages;
                const uint32_t par = (kb / stages) & 1;
                if (!tc::mbar_wait(full(s), par, a.status) || !tc::mbar_wait(bfull(s), par, a.status)) break;
                tc::tc_fence_after();
                const int g = kb * a.groups / a.nkb;
                const uint32_t mainacc = tmem + (uint32_t)(g * a.nc);
                const uint32_t abase = tc::smem_u32(smem + s * stage_bytes);
                const uint32_t bbase = abase + a_bytes;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t ko = kk * 32;
                    mma<F>(mainacc, tc::desc_k_sw128(abase + ko), tc::desc_k_sw128(bbase + ko), id,
                           started[g] ? 1u : 0u);
                    started[g] = true;
#pragma unroll
                    for (int c = 0; c < F::kCorr; ++c)
                        mma<F>(corr, tc::desc_k_sw128(abase + F::corr_a(c) * kATile + ko),
                               tc::desc_k_sw128(bbase + F::corr_b(c) * b_tile + ko), id,
                               (c == 0 && (kb | kk) == 0) ? 0u : 1u);
                }
                tc::mma_commit(empty(s));
            }
            tc::mma_commit(accum);     // arrives once every issued MMA has completed
        }
    }

    // ---- epilogue: all eight warps drain TMEM, partial sums added in FP32 ----
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(accum, 0, a.status));
    tc::tc_fence_after();
    if (ok) {
        const int quarter = warp & 3, half = warp >> 2;
        const int r = quarter * 32 + lane;
        const int64_t q = q0 + r;
        const bool valid = q < a.rows;
        const int64_t base = valid ? (q % a.L) + (q / a.L) * a.L * a.n : 0;
        const int chunks = a.nc / 16;
        const int c_lo = half ? (chunks + 1) / 2 : 0;
        const int c_hi = half ? chunks : (chunks + 1) / 2;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        float alphaf = 0.f, t0f = 0.f, t1f = 0.f;
        if constexpr (LAST) { alphaf = (float)e.alpha; t0f = (float)e.t0; t1f = (float)e.t1; }
        for (int c = c_lo; c < c_hi; ++c) {
            // y = corrections + main groups, added in FP32 (round to nearest)
            float y[16];
            uint32_t v[16];
            tc::tmem_ld16(tmem + lane_off + (uint32_t)(a.groups * a.nc + c * 16), v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 16; ++t) y[t] = __uint_as_float(v[t]);
            for (int g = 0; g < a.groups; ++g) {
                tc::tmem_ld16(tmem + lane_off + (uint32_t)(g * a.nc + c * 16), v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; ++t) y[t] += __uint_as_float(v[t]);
            }
            if (!valid) continue;
            const int i0 = col0 + c * 16;
            if constexpr (LAST) {
                mixed_epilogue16(e, y, base, i0, a.n, a.L, alphaf, t0f, t1f);
            } else if (a.L == 1 && (a.n & 3) == 0 && i0 + 16 <= a.n) {
                float4* o = (float4*)(a.out + base + i0);
#pragma unroll
                for (int t = 0; t < 4; ++t) o[t] = make_float4(y[4 * t], y[4 * t + 1], y[4 * t + 2], y[4 * t + 3]);
            } else {
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (i0 + t < a.n) a.out[base + (int64_t)(i0 + t) * a.L] = y[t];
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
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
        double r = v;
        for (int part = 0; part < kBParts; ++part) {
            uint8_t* dst = blk + (size_t)part * n_img * 128 + off;
            if (F::kElem == 4) {
                const float b = mx::tf32((float)r);
                *(float*)dst = b;
                r -= (double)b;
            } else {
                const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
                *(__nv_bfloat16*)dst = b;
                r -= (double)__bfloat162float(b);
            }
        }
    }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Geometry {
    int n, n_img, nkb, nc, splits, groups, stages;
    uint32_t tmem_cols;
    size_t smem;
};

// Columns per CTA (nc, one MMA), accumulator groups, pipeline depth.
template <class F>
int geometry(int n, Geometry* g) {
    const int n16 = round_up(n, 16);
    if (n16 > 512) return MM_ERR_UNSUPPORTED;
    g->n = n;
    g->nkb = (n + F::kBK - 1) / F::kBK;
    // columns per CTA: at most kNcMax, so that two pipeline stages of the A parts
    // and the three Phi parts fit in shared memory
    g->splits = (n16 + F::kNcMax - 1) / F::kNcMax;
    g->nc = round_up((n16 + g->splits - 1) / g->splits, 16);
    g->n_img = g->splits * g->nc;
    g->groups = std::min(std::min(g->nkb, kMaxGroups), std::max(1, 512 / g->nc - 1));
    const int cols = (g->groups + 1) * g->nc;
    uint32_t pow2 = 32;
    while (pow2 < (uint32_t)cols) pow2 <<= 1;
    if (pow2 > 512) return MM_ERR_UNSUPPORTED;
    g->tmem_cols = pow2;
    const size_t stage = (size_t)F::kAParts * kATile + kBParts * (size_t)g->nc * 128;
    const size_t fixed = 1024 + (3 * kMaxStages + 1) * 8 + 16;
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

template <class F, typename TIn, bool LAST>
int launch_mode(const Tf32Mode& m, const Epi& e, size_t smem, int64_t ctas, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        MM_CUDA_TRY(cudaFuncSetAttribute(tc_mode_kernel<F, TIn, LAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
        configured = true;
    }
    TraceScope tr(KC_CONTRACT_TF32, s);
    tc_mode_kernel<F, TIn, LAST><<<(unsigned)ctas, 256, smem, s>>>(m, e);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

template <class F>
int launch_form(const Tf32Mode& m, const Epi& e, bool in_fp64, bool last, size_t smem, int64_t ctas,
                cudaStream_t s) {
    if (in_fp64) {
        return last ? launch_mode<F, double, true>(m, e, smem, ctas, s)
                    : launch_mode<F, double, false>(m, e, smem, ctas, s);
    }
    return last ? launch_mode<F, float, true>(m, e, smem, ctas, s)
                : launch_mode<F, float, false>(m, e, smem, ctas, s);
}

}  // namespace

int plan_prepare_tf32(mm_plan_s* p, cudaStream_t s) {
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

int tf32_mode_product(mm_plan_s* p, int ell, int mu, const void* in, bool in_fp64, float* out,
                      const Epi* last, cudaStream_t s) {
    Geometry g;
    int rc = geometry_for(p->prec, (int)p->n[mu - 1], &g);
    if (rc) return rc;
    Tf32Mode m{};
    m.n = g.n; m.n_pad = g.n_img; m.nkb = g.nkb; m.nc = g.nc; m.splits = g.splits;
    m.groups = g.groups; m.stages = g.stages;
    int64_t L = 1;
    for (int v = 0; v < mu - 1; ++v) L *= p->n[v];
    m.L = L;
    m.rows = p->N / g.n;
    m.in = in;
    m.out = out;
    m.bimg = (const uint8_t*)p->phi_split[mu - 1][ell];
    m.tmem_cols = g.tmem_cols;
    m.status = p->status;
    const int64_t ctas = (m.rows + kRows - 1) / kRows * g.splits;
    if (ctas > 0x7fffffffLL) return MM_ERR_SHAPE;
    Epi e{};
    if (last) e = *last;
    if (p->prec == MM_BF16X3) return launch_form<FormBF16>(m, e, in_fp64, last != nullptr, g.smem, ctas, s);
    return launch_form<FormTF32>(m, e, in_fp64, last != nullptr, g.smem, ctas, s);
}

int tf32_supported(int prec, int n) {
    Geometry g;
    return geometry_for(prec, n, &g);
}

}  // namespace mm
