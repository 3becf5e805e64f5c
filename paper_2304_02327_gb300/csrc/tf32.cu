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
// product of every K-block goes into a fresh TMEM slot (only its four MMAs
// accumulate in hardware) and the epilogue warps add the slots into FP32 registers
// with round-to-nearest; the much smaller corrections accumulate in TMEM
// over the whole tile, in an accumulator of their own: added onto the main product,
// their low-order bits would force a truncation at main-product magnitude into sums
// that are otherwise exact (an exactly representable operand, such as the 0/alpha
// matrix B of the LQ Riccati problem, makes every main-product sum exact), and the
// resulting bias accumulated over the steps of that problem to 1.4e-6 in 30 steps
// against 1.5e-7 this way.  The three-way split of the fixed matrix keeps its
// rounding, which would repeat identically every step, at ~2^-25 (BF16) or 2^-33
// (TF32) of its entries.
//
// Kernel structure: persistent, one CTA per SM over tiles t = blockIdx.x + i grid.
//   warp 0      loader: per K-block, one TMA tensor load per part of either
//               operand (the 3-D maps {K, rows, part} zero-fill the ragged K tail
//               and the last rows)
//   warp 1      MMA issuer (one thread): per K-block one asm block of main-product
//               MMAs into the current slot of a kMainSlots-slot ring (a fresh slot
//               every kGroup K-blocks) and one of corrections into the tile's
//               accumulator
//   warps 2-17  epilogue, four warps per TMEM lane quarter, each owning a quarter
//               of the columns: drain each main slot into register accumulators as
//               it completes, then add the corrections and write the next mode's
//               split operand (or FP32 after the last mode); the slot ring lets the
//               MMAs of the next tile's first K-blocks run meanwhile
// TMEM: [main slot 0 | ... | main slot kMainSlots-1 | corrections], nc columns each;
// the next tile's corrections wait until the epilogue has read this tile's.  Every
// mbarrier wait is bounded (tcgen05.cuh).
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
constexpr uint32_t kRowBytes = 128;        // one stage's K slice of a row (128-byte swizzle)
constexpr uint32_t kATile = kRows * kRowBytes;   // bytes of one operand part tile
constexpr int kMaxStages = 4;
// Stages whose main products share a TMEM slot.  Measured on the 100-step 3D ADR run
// at n = 320: with 2, the truncation bias of the slot sums took the TF32x3 form to
// 1.16e-6 (BF16x3 8.8e-7) of the FP64 run; with 1, 5.5e-7 (5.6e-7), for ~7 % of
// contraction time.
constexpr int kGroup = 1;
constexpr int kBParts = 3;                 // Phi = b0 + b1 + b2 in both forms
// TMEM main-product slots in the ring.  [main slots | corrections] share the 512 TMEM
// columns, which caps the tile width: two slots allow tiles of 160 columns.  Measured
// with three slots (tiles of <= 128 columns, so the next tile's MMAs run three K-blocks
// ahead of the epilogue's stores): the n = 320 contraction went from 0.636 to 0.780 ms
// per ETD2RK step (three column splits of 112 instead of two of 160), the batch's from
// 0.910 to 1.033 ms; only the n = 2048 Riccati products gained (0.905 -> 0.893 ms).
constexpr int kMainSlots = 2;
constexpr int kNcMax = 512 / (kMainSlots + 1) / 16 * 16;
constexpr int kBars = 2 * kMaxStages + 2 * kMainSlots + 5;  // full, empty per stage; main full/empty
                                                            // per slot; corr full/empty (tile
                                                            // parity); mma_done
constexpr int kSmemLimit = 227 * 1024;
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kChunks = (kNcMax + 63) / 64;  // 16-column chunks per epilogue warp (4 x kChunks x 16 >= kNcMax)
constexpr int kQuartCols = 16 * kChunks;   // columns per epilogue thread (upper bound)
constexpr int kMaxClasses = MM_TC_MAX_CLASSES;

template <class F> __device__ __forceinline__ uint32_t idesc_of(int nc);
template <> __device__ __forceinline__ uint32_t idesc_of<FormTF32>(int nc) { return tc::idesc_tf32(128, nc); }
template <> __device__ __forceinline__ uint32_t idesc_of<FormBF16>(int nc) { return tc::idesc_bf16(128, nc); }

// ---- the MMAs of one K-block, each group from a single asm block ----------
// One thread issues every MMA of the CTA, so its instruction count per MMA bounds
// the tensor pipe: at ~90 cycles per MMA (per-MMA descriptor arithmetic and
// predicate set-up) it, not the pipe (N / 2 cycles at N = 160), set the tile time.
// Here each descriptor is assembled from its two 32-bit words (tcgen05.cuh): the
// low word on the stage base plus a constant offset, the high word shared.  A part
// tile q starts 16 KB (1024 units) after part 0, B part q at q * bstep units, and
// K slice kk at 2 kk units (32 bytes).
constexpr uint32_t kDescHi = tc::kDescSw128Hi;
__device__ __forceinline__ uint32_t desc_lo(uint32_t addr) { return tc::desc_sw128_lo(addr); }

#define MM_TC_MMA(KIND, D, AOFF, B, BOFF, P)                         \
    "add.u32 la, %1, " AOFF ";\n\t"                                 \
    "add.u32 lb, " B ", " BOFF ";\n\t"                              \
    "mov.b64 da, {la, %3};\n\t"                                     \
    "mov.b64 db, {lb, %3};\n\t"                                     \
    "tcgen05.mma.cta_group::1.kind::" KIND " [" D "], da, db, %4, " P ";\n\t"

// main product a0 b0 over the four K slices; the first one overwrites unless acc
#define MM_TC_MAIN(KIND)                                                                 \
    asm volatile(                                                                        \
        "{\n\t.reg .pred pa, pt;\n\t.reg .b32 la, lb;\n\t.reg .b64 da, db;\n\t"       \
        "setp.ne.b32 pa, %5, 0;\n\t"                                                    \
        "setp.eq.b32 pt, %5, %5;\n\t"                                                   \
        MM_TC_MMA(KIND, "%0", "0", "%2", "0", "pa")                                      \
        MM_TC_MMA(KIND, "%0", "2", "%2", "2", "pt")                                      \
        MM_TC_MMA(KIND, "%0", "4", "%2", "4", "pt")                                      \
        MM_TC_MMA(KIND, "%0", "6", "%2", "6", "pt")                                      \
        "}" ::"r"(d), "r"(alo), "r"(blo), "r"(kDescHi), "r"(idesc), "r"(acc)              \
        : "memory")

template <class F>
__device__ __forceinline__ void mma_main(uint32_t d, uint32_t alo, uint32_t blo, uint32_t idesc, uint32_t acc);
template <>
__device__ __forceinline__ void mma_main<FormTF32>(uint32_t d, uint32_t alo, uint32_t blo, uint32_t idesc,
                                                   uint32_t acc) {
    MM_TC_MAIN("tf32");
}
template <>
__device__ __forceinline__ void mma_main<FormBF16>(uint32_t d, uint32_t alo, uint32_t blo, uint32_t idesc,
                                                   uint32_t acc) {
    MM_TC_MAIN("f16");
}

// corrections of one K block (slice-major, the form's pairs within a slice) into d;
// the first overwrites unless acc.  b1, b2: B parts 1 and 2.
#define MM_TC_CORR_PRE                                                                   \
    "{\n\t.reg .pred pa, pt;\n\t.reg .b32 la, lb, b1, b2;\n\t.reg .b64 da, db;\n\t"   \
    "setp.ne.b32 pa, %5, 0;\n\t"                                                        \
    "setp.eq.b32 pt, %5, %5;\n\t"                                                       \
    "add.u32 b1, %2, %6;\n\t"                                                           \
    "add.u32 b2, b1, %6;\n\t"

template <class F>
__device__ __forceinline__ void mma_corr(uint32_t d, uint32_t alo, uint32_t blo, uint32_t bstep, uint32_t idesc,
                                         uint32_t acc);
// TF32x3: a1 b0, a0 b1, a0 b2 per slice
template <>
__device__ __forceinline__ void mma_corr<FormTF32>(uint32_t d, uint32_t alo, uint32_t blo, uint32_t bstep,
                                                   uint32_t idesc, uint32_t acc) {
    asm volatile(MM_TC_CORR_PRE
                 MM_TC_MMA("tf32", "%0", "1024", "%2", "0", "pa")
                 MM_TC_MMA("tf32", "%0", "0", "b1", "0", "pt")
                 MM_TC_MMA("tf32", "%0", "0", "b2", "0", "pt")
                 MM_TC_MMA("tf32", "%0", "1026", "%2", "2", "pt")
                 MM_TC_MMA("tf32", "%0", "2", "b1", "2", "pt")
                 MM_TC_MMA("tf32", "%0", "2", "b2", "2", "pt")
                 MM_TC_MMA("tf32", "%0", "1028", "%2", "4", "pt")
                 MM_TC_MMA("tf32", "%0", "4", "b1", "4", "pt")
                 MM_TC_MMA("tf32", "%0", "4", "b2", "4", "pt")
                 MM_TC_MMA("tf32", "%0", "1030", "%2", "6", "pt")
                 MM_TC_MMA("tf32", "%0", "6", "b1", "6", "pt")
                 MM_TC_MMA("tf32", "%0", "6", "b2", "6", "pt")
                 "}" ::"r"(d), "r"(alo), "r"(blo), "r"(kDescHi), "r"(idesc), "r"(acc), "r"(bstep)
                 : "memory");
}
// BF16x3: a1 b0, a0 b1, a2 b0, a1 b1, a0 b2 per slice
template <>
__device__ __forceinline__ void mma_corr<FormBF16>(uint32_t d, uint32_t alo, uint32_t blo, uint32_t bstep,
                                                   uint32_t idesc, uint32_t acc) {
    asm volatile(MM_TC_CORR_PRE
                 MM_TC_MMA("f16", "%0", "1024", "%2", "0", "pa")
                 MM_TC_MMA("f16", "%0", "0", "b1", "0", "pt")
                 MM_TC_MMA("f16", "%0", "2048", "%2", "0", "pt")
                 MM_TC_MMA("f16", "%0", "1024", "b1", "0", "pt")
                 MM_TC_MMA("f16", "%0", "0", "b2", "0", "pt")
                 MM_TC_MMA("f16", "%0", "1026", "%2", "2", "pt")
                 MM_TC_MMA("f16", "%0", "2", "b1", "2", "pt")
                 MM_TC_MMA("f16", "%0", "2050", "%2", "2", "pt")
                 MM_TC_MMA("f16", "%0", "1026", "b1", "2", "pt")
                 MM_TC_MMA("f16", "%0", "2", "b2", "2", "pt")
                 MM_TC_MMA("f16", "%0", "1028", "%2", "4", "pt")
                 MM_TC_MMA("f16", "%0", "4", "b1", "4", "pt")
                 MM_TC_MMA("f16", "%0", "2052", "%2", "4", "pt")
                 MM_TC_MMA("f16", "%0", "1028", "b1", "4", "pt")
                 MM_TC_MMA("f16", "%0", "4", "b2", "4", "pt")
                 MM_TC_MMA("f16", "%0", "1030", "%2", "6", "pt")
                 MM_TC_MMA("f16", "%0", "6", "b1", "6", "pt")
                 MM_TC_MMA("f16", "%0", "2054", "%2", "6", "pt")
                 MM_TC_MMA("f16", "%0", "1030", "b1", "6", "pt")
                 MM_TC_MMA("f16", "%0", "6", "b2", "6", "pt")
                 "}" ::"r"(d), "r"(alo), "r"(blo), "r"(kDescHi), "r"(idesc), "r"(acc), "r"(bstep)
                 : "memory");
}
#undef MM_TC_CORR_PRE
#undef MM_TC_MAIN
#undef MM_TC_MMA

// One class of tiles: instances of equal shape whose operands sit packed one after
// the other (instance j's tensor operand rows at j * rows, its matrix operand rows
// at j * ncols).  A single product is one class with one instance.
struct TcClass {
    CUtensorMap xmap;        // tensor operand parts {k, rows x instances, kAParts}
    CUtensorMap mmap;        // matrix operand parts {k, ncols x instances, 3}
    int k, ncols, nkb, nc, splits;
    int rows;                // tensor operand rows (output rows) per instance
    int last, accum;         // FP32 output (stored, or added when accum) / split parts
    float* yout;             // instance j: y[j y_stride + q + ldy col]
    int64_t ldy, y_stride;
    uint8_t* pout;           // instance j: part m element j p_stride + layout position
    int64_t out_part_pitch, p_stride;
    int next_n, next_p;      // fibre length and row pitch of the output layout
    int64_t next_rows_per_i; // rows of the output layout per output column
};

template <int C>
struct TcGroup {
    TcClass cls[C];
    const int4* tiles;       // {class, instance, row tile, column split}; NULL: class 0,
    int64_t ntiles;          //   instance 0, tile t = row tile (t / splits), split (t % splits)
    int stage_nc;            // widest nc of the classes (shared-memory and TMEM slots)
    int stages;
    unsigned int* status;
};

template <int E> struct PartType;
template <> struct PartType<2> { using type = uint16_t; };
template <> struct PartType<4> { using type = uint32_t; };

struct TileId {
    int c, inst, rt, sp;
};

template <int C>
__device__ __forceinline__ TileId tile_of(const TcGroup<C>& g, int64_t t) {
    TileId id;
    if (g.tiles) {
        const int4 v = g.tiles[t];
        id.c = v.x; id.inst = v.y; id.rt = v.z; id.sp = v.w;
    } else {
        id.c = 0; id.inst = 0;
        id.rt = (int)(t / g.cls[0].splits);
        id.sp = (int)(t % g.cls[0].splits);
    }
    return id;
}

template <class F, int C>
__global__ void __launch_bounds__(kThreads, 1) tc_mode_kernel(const __grid_constant__ TcGroup<C> g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);   // 1024-byte aligned
    const uint32_t b_slot = (uint32_t)g.stage_nc * kRowBytes;  // one part of the matrix tile
    const uint32_t a_bytes = F::kAParts * kATile;
    const uint32_t stage_bytes = a_bytes + kBParts * b_slot;
    uint64_t* bars = (uint64_t*)(smem + g.stages * stage_bytes);
    uint32_t* tmem_slot = (uint32_t*)(bars + kBars);
    auto full = [&](int s) { return tc::smem_u32(bars + s); };
    auto empty = [&](int s) { return tc::smem_u32(bars + kMaxStages + s); };
    // Parity waits are only sound for a waiter that consumes every phase in order:
    // the "full" barriers are waited only by the epilogue (in K-block / tile
    // order), the "empty" ones only by the MMA thread.
    auto mfull = [&](int r) { return tc::smem_u32(bars + 2 * kMaxStages + r); };
    auto mempty = [&](int r) { return tc::smem_u32(bars + 2 * kMaxStages + kMainSlots + r); };
    auto cfull = [&](int b) { return tc::smem_u32(bars + 2 * kMaxStages + 2 * kMainSlots + b); };
    auto cempty = [&](int b) { return tc::smem_u32(bars + 2 * kMaxStages + 2 * kMainSlots + 2 + b); };
    const uint32_t mma_done = tc::smem_u32(bars + 2 * kMaxStages + 2 * kMainSlots + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stages = g.stages;
    const int64_t my_tiles = blockIdx.x < g.ntiles ? (g.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            tc::mbar_init(full(s), 1);
            tc::mbar_init(empty(s), 1);
        }
        for (int b = 0; b < kMainSlots; ++b) {
            tc::mbar_init(mfull(b), 1);
            tc::mbar_init(mempty(b), kEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
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
            // ---- loader: both operands' parts by TMA ----
            int64_t issued_last[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) issued_last[s] = -1;
            int64_t it = 0;
            int s = 0;                     // it mod stages
            uint32_t ph = 0;               // (it / stages) mod 2
            bool ok = true;
            for (int64_t i = 0; i < my_tiles && ok; ++i) {
                const TileId id = tile_of(g, blockIdx.x + i * gridDim.x);
                const TcClass& k = g.cls[id.c];
                const int row0 = id.inst * k.rows + id.rt * kRows;
                const int col0 = id.inst * k.ncols + id.sp * k.nc;
                const uint32_t b_tile = (uint32_t)k.nc * kRowBytes;
                for (int kb = 0; kb < k.nkb; ++kb, ++it) {
                    if (it >= stages && !tc::mbar_wait(empty(s), ph ^ 1u, g.status)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(full(s), a_bytes + kBParts * b_tile);
                    const uint32_t st = tc::smem_u32(smem + s * stage_bytes);
                    for (int q = 0; q < F::kAParts; ++q)
                        tc::tma_load_3d(st + q * kATile, &k.xmap, kb * F::kBK, row0, q, full(s));
                    for (int part = 0; part < kBParts; ++part)   // rows col0.. of b0, b1, b2
                        tc::tma_load_3d(st + a_bytes + part * b_slot, &k.mmap, kb * F::kBK, col0, part, full(s));
                    issued_last[s] = it;
                    if (++s == stages) { s = 0; ph ^= 1u; }
                }
            }
            // never leave the CTA with copies in flight
            for (int s = 0; s < stages; ++s)
                if (issued_last[s] >= 0)
                    tc::mbar_wait(full(s), (uint32_t)(issued_last[s] / stages) & 1, g.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            int s = 0;                     // stage of the next K-block
            uint32_t ph = 0;               // its fill phase parity
            int64_t git = 0;               // main-slot groups issued
            int64_t uses[kMainSlots] = {};  // uses of each main slot so far
            bool ok = true;
            const uint32_t corr = tmem + (uint32_t)(kMainSlots * g.stage_nc);   // the tile's corrections
            const uint32_t sbase = tc::smem_u32(smem);
            const uint32_t bstep = b_slot >> 4;                        // one B part, descriptor units
            for (int64_t i = 0; i < my_tiles && ok; ++i) {
                const TileId id = tile_of(g, blockIdx.x + i * gridDim.x);
                const TcClass& k = g.cls[id.c];
                const uint32_t idd = idesc_of<F>(k.nc);
                // main products: one TMEM slot per group of kGroup stages (a fresh slot
                // per group, drained by the epilogue); corrections: one accumulator per
                // tile, free again once the epilogue has read the previous tile's (its
                // wait comes after the first stage's main products are queued)
                int r = 0;
                for (int kb = 0; kb < k.nkb; ++kb) {
                    const bool gfirst = (kb % kGroup) == 0;
                    const bool glast = (kb % kGroup) == kGroup - 1 || kb == k.nkb - 1;
                    if (gfirst) {
                        r = (int)(git % kMainSlots);
                        if (uses[r] >= 1 && !tc::mbar_wait(mempty(r), (uint32_t)(uses[r] - 1) & 1, g.status)) {
                            ok = false;
                            break;
                        }
                        ++uses[r];
                    }
                    if (!tc::mbar_wait(full(s), ph, g.status)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t abase = sbase + (uint32_t)s * stage_bytes;
                    const uint32_t alo = desc_lo(abase), blo = desc_lo(abase + a_bytes);
                    mma_main<F>(tmem + (uint32_t)(r * g.stage_nc), alo, blo, idd, gfirst ? 0u : 1u);
                    if (kb == 0 && i >= 1 && !tc::mbar_wait(cempty(0), (uint32_t)((i - 1) & 1), g.status)) {
                        ok = false;
                        break;
                    }
                    mma_corr<F>(corr, alo, blo, bstep, idd, kb == 0 ? 0u : 1u);
                    tc::mma_commit(empty(s));
                    if (glast) {
                        tc::mma_commit(mfull(r));
                        ++git;
                    }
                    if (++s == stages) { s = 0; ph ^= 1u; }
                }
                if (ok) tc::mma_commit(cfull(0));
            }
            // every issued MMA has completed before TMEM can be released
            tc::mma_commit(mma_done);
            tc::mbar_wait(mma_done, 0, g.status);
        }
    } else {
        // ---- epilogue: lane quarter (warp mod 4), column quarter ((warp - 2) / 4) ----
        const int quarter = warp & 3;
        const int cq = (warp - 2) >> 2;
        const int r = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        int64_t it = 0;                    // main-slot groups drained
        for (int64_t i = 0; i < my_tiles; ++i) {
            const TileId id = tile_of(g, blockIdx.x + i * gridDim.x);
            const TcClass& k = g.cls[id.c];
            const int nch = k.nc / 16;                        // <= 8 chunks of 16 columns
            const int c0 = kChunks * cq, c1 = min(nch, kChunks * cq + kChunks);
            float acc[kQuartCols];
#pragma unroll
            for (int u = 0; u < kQuartCols; ++u) acc[u] = 0.f;
            bool ok = true;
            // main product, one slot (kGroup stages) at a time, summed in FP32 registers
            const int ngroups = (k.nkb + kGroup - 1) / kGroup;
            for (int gi = 0; gi < ngroups && ok; ++gi, ++it) {
                const int rs = (int)(it % kMainSlots);
                ok = __all_sync(0xffffffffu, tc::mbar_wait(mfull(rs), (uint32_t)(it / kMainSlots) & 1, g.status));
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t slot = tmem + lane_off + (uint32_t)(rs * g.stage_nc);
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
            ok = __all_sync(0xffffffffu, tc::mbar_wait(cfull(0), (uint32_t)(i & 1), g.status));
            if (!ok) break;
            tc::tc_fence_after();
            const int64_t q = (int64_t)id.rt * kRows + r;
            const int col0 = id.sp * k.nc;
            const bool valid = q < k.rows;
            // next-mode layout of output (q, i): position jq + p' (rq + (R / n') i)
            int64_t jq = 0, rq = 0;
            if (!k.last) { jq = q % k.next_n; rq = q / k.next_n; }
            const uint32_t cset = tmem + lane_off + (uint32_t)(kMainSlots * g.stage_nc);
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
            if (lane == 0) tc::mbar_arrive(cempty(0));      // corrections read: accumulator free
            if (!valid) continue;
            // output column col of row q: next-mode position jq + p' (rq + (R / n') col)
            // (or q + ldy col for FP32); successive columns step by dpos
            const int64_t dpos = k.last ? k.ldy : (int64_t)k.next_p * k.next_rows_per_i;
            if (k.last) {
                float* const yb = k.yout + (int64_t)id.inst * k.y_stride + q;
                const bool accum = k.accum != 0;
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    if (c0 + c >= c1) continue;
                    const int i0 = col0 + (c0 + c) * 16;
                    float* y = yb + k.ldy * (int64_t)i0;
                    const int lim = min(16, k.ncols - i0);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        if (u >= lim) break;
                        *y = accum ? *y + acc[c * 16 + u] : acc[c * 16 + u];
                        y += dpos;
                    }
                }
            } else {
                // the parts of one element sit part_pitch apart; three pointers walk
                // the columns together
                using T = typename PartType<F::kElem>::type;
                const int64_t pp = k.out_part_pitch;
                T* const ob = (T*)k.pout + (int64_t)id.inst * k.p_stride + jq;
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    if (c0 + c >= c1) continue;
                    const int i0 = col0 + (c0 + c) * 16;
                    T* p0 = ob + (int64_t)k.next_p * (rq + k.next_rows_per_i * (int64_t)i0);
                    T* p1 = p0 + pp;
                    T* p2 = F::kAParts == 3 ? p1 + pp : p1;
                    const int lim = min(16, k.ncols - i0);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        if (lim < 16 && u >= lim) break;
                        uint32_t v[3];
                        split_parts<F>(acc[c * 16 + u], 0.f, v);
                        *p0 = (T)v[0];
                        *p1 = (T)v[1];
                        if (F::kAParts == 3) *p2 = (T)v[2];
                        p0 += dpos; p1 += dpos; p2 += dpos;
                    }
                }
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Matrix operand M (rows x K, M[i][k]) -> its parts at dst[j part_pitch + k + pitch i],
// from the FP64 matrix `src`: src[i + ld k] if colmajor (M itself stored column-major)
// else src[k + ld i] (M^T stored column-major).  zero_band drops |i - k| <= 1 (the
// tridiagonal band, evaluated apart as a stencil).  32 x 32 tiles through shared
// memory, so both the read and the write are coalesced.
template <class F, int NP>
__global__ void __launch_bounds__(256) split_matrix_kernel(const double* __restrict__ src, int64_t ld, int rows,
                                                           int K, int colmajor, int zero_band, uint8_t* dst,
                                                           int pitch, int64_t part_pitch) {
    __shared__ double t[32][33];          // t[k - k0][i - i0]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int y = ty + 8 * r;
        if (colmajor) {                    // lanes along i
            const int i = i0 + tx, k = k0 + y;
            t[y][tx] = (i < rows && k < K) ? __ldg(src + i + ld * k) : 0.0;
        } else {                           // lanes along k
            const int i = i0 + y, k = k0 + tx;
            t[tx][y] = (i < rows && k < K) ? __ldg(src + k + ld * i) : 0.0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 8 * r, k = k0 + tx;
        if (i >= rows || k >= K) continue;
        double v = t[tx][ty + 8 * r];
        if (zero_band && i - k <= 1 && k - i <= 1) v = 0.0;
        float h, l;
        mx::d2ff(v, h, l);
        uint32_t pp[3];
        split_parts3<F>(h, l, pp);
        const int64_t pos = k + (int64_t)pitch * i;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (F::kElem == 4) ((uint32_t*)dst)[j * part_pitch + pos] = pp[j];
            else ((uint16_t*)dst)[j * part_pitch + pos] = (uint16_t)pp[j];
        }
    }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Geometry {
    int nc, splits;
};

// Columns per CTA tile given at most nc_cap (a multiple of 16, <= kNcMax): the
// fewest splits, then the narrowest multiple of 16 that covers the columns.
Geometry split_cols(int ncols, int nc_cap) {
    nc_cap = std::min(nc_cap, kNcMax);
    const int n16 = round_up(ncols, 16);
    Geometry g;
    g.splits = (n16 + nc_cap - 1) / nc_cap;
    g.nc = round_up((n16 + g.splits - 1) / g.splits, 16);
    g.splits = (n16 + g.nc - 1) / g.nc;
    return g;
}

// Relative time of one tile of width nc: a tcgen05.mma of M = 128 takes the same
// time for every N up to 160 (measured), so a tile costs about the same whatever
// its width, plus an epilogue share that grows with nc.
int64_t tile_cost(int nkb, int nc) { return (int64_t)nkb * (256 + nc); }

// One product alone on the GPU: among the column splittings, the one whose tile
// waves over the SMs cost least.
Geometry geometry_single(int ncols, int64_t rows) {
    const int n16 = round_up(ncols, 16);
    const int64_t row_tiles = (rows + kRows - 1) / kRows;
    const int64_t sms = num_sms();
    const int s_min = (n16 + kNcMax - 1) / kNcMax;
    Geometry best{};
    int64_t best_cost = -1;
    for (int sp = s_min; sp <= 2 * s_min && sp <= n16 / 16; ++sp) {
        const Geometry g = split_cols(ncols, round_up((n16 + sp - 1) / sp, 16));
        const int64_t waves = (row_tiles * g.splits + sms - 1) / sms;
        const int64_t cost = waves * tile_cost(1, g.nc);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = g;
        }
    }
    return best;
}

// Pipeline depth and dynamic shared memory for tiles up to stage_nc columns.
template <class F>
int stages_for(int stage_nc, int* stages, size_t* smem) {
    const size_t stage = (size_t)F::kAParts * kATile + kBParts * (size_t)stage_nc * kRowBytes;
    const size_t fixed = 1024 + kBars * 8 + 16;
    int st = (int)((kSmemLimit - fixed) / stage);
    st = std::min(st, kMaxStages);
    if (st < 2) return MM_ERR_UNSUPPORTED;
    *stages = st;
    *smem = fixed + st * stage;
    return MM_OK;
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

// 3-D map {K, rows, parts} of a part array, box {one K-block, box_rows, 1 part},
// 128-byte swizzle; loads past K or the last row read zeros.
template <class F>
int encode_parts(CUtensorMap* map, const PartView& v, int nparts, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return MM_ERR_UNSUPPORTED;
    if (((uintptr_t)v.base & 15) || ((int64_t)v.p * F::kElem) % 16 || (v.part_pitch * F::kElem) % 16)
        return MM_ERR_ARG;
    const cuuint64_t dims[3] = {(cuuint64_t)v.n, (cuuint64_t)v.rows, (cuuint64_t)nparts};
    const cuuint64_t strides[2] = {(cuuint64_t)v.p * F::kElem, (cuuint64_t)v.part_pitch * F::kElem};
    const cuuint32_t box[3] = {(cuuint32_t)F::kBK, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = F::kElem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (enc(map, dt, 3, (void*)v.base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return MM_ERR_CUDA;
    return MM_OK;
}

template <class F>
int fill_class(TcClass& k, const TcClassSpec& c, const Geometry& geo) {
    if (c.X.n != c.M.n || c.count < 1 || c.rows < 1 || c.ncols < 1) return MM_ERR_SHAPE;
    if ((int64_t)c.rows * c.count > 0x7fffffffLL || (int64_t)c.ncols * c.count > 0x7fffffffLL)
        return MM_ERR_SHAPE;
    k.k = c.X.n;
    k.ncols = c.ncols;
    k.nkb = (c.X.n + F::kBK - 1) / F::kBK;
    k.nc = geo.nc;
    k.splits = geo.splits;
    k.rows = c.rows;
    k.last = c.out.last;
    k.accum = c.out.accum;
    k.yout = c.out.y;
    k.ldy = c.out.ldy;
    k.y_stride = c.y_stride;
    k.pout = c.out.parts;
    k.out_part_pitch = c.out.part_pitch;
    k.p_stride = c.p_stride;
    k.next_n = c.out.next_n;
    k.next_p = c.out.next_p;
    k.next_rows_per_i = c.out.next_rows_per_i;
    if (!k.last && (k.next_n < 1 || k.next_p < k.next_n)) return MM_ERR_ARG;
    int rc = encode_parts<F>(&k.xmap, c.X, F::kAParts, kRows);
    if (!rc) rc = encode_parts<F>(&k.mmap, c.M, kBParts, geo.nc);
    return rc;
}

// The kernels' shared-memory attribute, set once per process (outside any stream
// capture: plan creation and batch creation call it first).
template <class F, int C>
int configure_kernel() {
    static bool configured = false;
    if (!configured) {
        MM_CUDA_TRY(cudaFuncSetAttribute(tc_mode_kernel<F, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemLimit));
        configured = true;
    }
    return MM_OK;
}

template <class F, int C>
int launch_group(TcGroup<C>& g, int64_t ctas, cudaStream_t s) {
    int rc0 = configure_kernel<F, C>();
    if (rc0) return rc0;
    int stages;
    size_t smem;
    int rc = stages_for<F>(g.stage_nc, &stages, &smem);
    if (rc) return rc;
    g.stages = stages;
    if (ctas < 1) return MM_OK;
    TraceScope tr(KC_CONTRACT_TF32, s);
    tc_mode_kernel<F, C><<<(unsigned)ctas, kThreads, smem, s>>>(g);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

template <class F>
int launch_single(const PartView& X, const PartView& M, const TcOut& o, unsigned int* status, cudaStream_t s) {
    if (X.n != M.n || X.rows > 0x7fffffffLL || M.rows > 0x7fffffffLL) return MM_ERR_SHAPE;
    TcClassSpec c{};
    c.X = X; c.rows = (int)X.rows; c.M = M; c.ncols = (int)M.rows; c.count = 1; c.out = o;
    const Geometry geo = geometry_single(c.ncols, X.rows);
    TcGroup<1> g{};
    int rc = fill_class<F>(g.cls[0], c, geo);
    if (rc) return rc;
    g.tiles = nullptr;
    g.ntiles = ((X.rows + kRows - 1) / kRows) * geo.splits;
    g.stage_nc = geo.nc;
    g.status = status;
    return launch_group<F, 1>(g, std::min<int64_t>(g.ntiles, num_sms()), s);
}

template <class F>
int launch_grouped(const TcClassSpec* cls, int ncls, const int* nc_cap, const int4* tiles, int64_t ntiles,
                   unsigned int* status, cudaStream_t s) {
    if (ncls < 1 || ncls > kMaxClasses) return MM_ERR_ARG;
    TcGroup<kMaxClasses> g{};            // the kernel parameters (~12 KB)
    int stage_nc = 16;
    for (int c = 0; c < ncls; ++c) {
        const Geometry geo = split_cols(cls[c].ncols, nc_cap[c]);
        int rc = fill_class<F>(g.cls[c], cls[c], geo);
        if (rc) return rc;
        stage_nc = std::max(stage_nc, geo.nc);
    }
    g.tiles = tiles;
    g.ntiles = ntiles;
    g.stage_nc = stage_nc;
    g.status = status;
    return launch_group<F, kMaxClasses>(g, std::min<int64_t>(ntiles, num_sms()), s);
}

}  // namespace

int form_elem_bytes(int prec) { return prec == MM_BF16X3 ? FormBF16::kElem : FormTF32::kElem; }
int form_parts(int prec) { return prec == MM_BF16X3 ? FormBF16::kAParts : FormTF32::kAParts; }
int form_pitch(int prec, int n) { return round_up(n, 16 / form_elem_bytes(prec)); }

PartView matrix_view(int prec, uint8_t* base, int64_t rows, int K) {
    PartView v;
    v.base = base;
    v.n = K;
    v.p = form_pitch(prec, K);
    v.rows = rows;
    v.part_pitch = rows * v.p;
    return v;
}

size_t matrix_parts_bytes(int prec, int64_t rows, int K, int nparts) {
    const size_t b = (size_t)nparts * rows * form_pitch(prec, K) * form_elem_bytes(prec);
    return (b + 255) / 256 * 256;
}

int split_matrix(int prec, const double* src, int64_t ld, int colmajor, int zero_band, const PartView& dst,
                 int nparts, cudaStream_t s) {
    if (nparts < 2 || nparts > 3 || dst.rows > 0x7fffffffLL) return MM_ERR_ARG;
    const dim3 grid((unsigned)((dst.n + 31) / 32), (unsigned)((dst.rows + 31) / 32));
    if (grid.y > 65535) return MM_ERR_SHAPE;
    TraceScope tr(KC_SPLIT, s);
    const int rows = (int)dst.rows;
#define MM_SPLIT_LAUNCH(F, NP)                                                                            \
    split_matrix_kernel<F, NP><<<grid, 256, 0, s>>>(src, ld, rows, dst.n, colmajor, zero_band, dst.base, \
                                                     dst.p, dst.part_pitch)
    if (prec == MM_BF16X3) {
        if (nparts == 3) MM_SPLIT_LAUNCH(FormBF16, 3);
        else MM_SPLIT_LAUNCH(FormBF16, 2);
    } else {
        if (nparts == 3) MM_SPLIT_LAUNCH(FormTF32, 3);
        else MM_SPLIT_LAUNCH(FormTF32, 2);
    }
#undef MM_SPLIT_LAUNCH
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int tc_product(int prec, const PartView& X, const PartView& M, const TcOut& o, unsigned int* status,
               cudaStream_t s) {
    if (prec == MM_BF16X3) return launch_single<FormBF16>(X, M, o, status, s);
    return launch_single<FormTF32>(X, M, o, status, s);
}

int tc_group_tiles(int prec, const TcClassSpec* cls, int ncls, const int* nc_cap, std::vector<int4>& tiles) {
    if (ncls < 1 || ncls > kMaxClasses) return MM_ERR_ARG;
    const int bk = prec == MM_BF16X3 ? FormBF16::kBK : FormTF32::kBK;
    std::vector<std::pair<int64_t, int4>> v;
    for (int c = 0; c < ncls; ++c) {
        const Geometry geo = split_cols(cls[c].ncols, nc_cap[c]);
        const int nkb = (cls[c].X.n + bk - 1) / bk;
        const int rt = (cls[c].rows + kRows - 1) / kRows;
        const int64_t cost = tile_cost(nkb, geo.nc);
        for (int j = 0; j < cls[c].count; ++j)
            for (int r = 0; r < rt; ++r)
                for (int sp = 0; sp < geo.splits; ++sp) v.push_back({cost, make_int4(c, j, r, sp)});
    }
    // decreasing cost; the CTAs take tiles round-robin from the front
    std::stable_sort(v.begin(), v.end(), [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& b) {
        return a.first > b.first;
    });
    tiles.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) tiles[i] = v[i].second;
    return MM_OK;
}

int tc_group_product(int prec, const TcClassSpec* cls, int ncls, const int* nc_cap, const int4* dev_tiles,
                     int64_t ntiles, unsigned int* status, cudaStream_t s) {
    if (prec == MM_BF16X3) return launch_grouped<FormBF16>(cls, ncls, nc_cap, dev_tiles, ntiles, status, s);
    return launch_grouped<FormTF32>(cls, ncls, nc_cap, dev_tiles, ntiles, status, s);
}

int encode_f64_box3(CUtensorMap* map, const double* base, const int64_t* dims, const uint32_t* box) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return MM_ERR_UNSUPPORTED;
    const uint64_t row = (uint64_t)dims[0] * 8, plane = row * (uint64_t)dims[1];
    if (((uintptr_t)base & 15) || row % 16 || plane % 16 || (box[0] * 8) % 16) return MM_ERR_ARG;
    const cuuint64_t d[3] = {(cuuint64_t)dims[0], (cuuint64_t)dims[1], (cuuint64_t)dims[2]};
    const cuuint64_t st[2] = {(cuuint64_t)row, (cuuint64_t)plane};
    const cuuint32_t bx[3] = {box[0], box[1], box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)base, d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return MM_ERR_CUDA;
    return MM_OK;
}

int plan_prepare_tf32(mm_plan_s* p, cudaStream_t s) {
    if (!encode_fn()) return MM_ERR_UNSUPPORTED;
    if (int rcp = configure_prepass_kernels()) return rcp;
    int rc0 = p->prec == MM_BF16X3 ? configure_kernel<FormBF16, 1>() : configure_kernel<FormTF32, 1>();
    if (!rc0) rc0 = p->prec == MM_BF16X3 ? configure_kernel<FormBF16, kMaxClasses>()
                                         : configure_kernel<FormTF32, kMaxClasses>();
    if (rc0) return rc0;
    for (int mu = 0; mu < p->d; ++mu) {
        if (p->owner[mu] != mu) {
            for (int l = 0; l <= p->ell_max; ++l) p->phi_split[mu][l] = p->phi_split[p->owner[mu]][l];
            p->coef3f[mu] = p->coef3f[p->owner[mu]];
            p->rem_split[mu] = p->rem_split[p->owner[mu]];
            continue;
        }
        const int n = (int)p->n[mu];
        if (!p->alloc((void**)&p->coef3f[mu], 3 * p->n[mu] * sizeof(float))) return MM_ERR_NOMEM;
        int rc = build_stencil_coef(p->A[mu], n, p->coef3f[mu], s);
        if (rc) return rc;
        const size_t bytes = matrix_parts_bytes(p->prec, n, n, kBParts);
        for (int l = 0; l <= p->ell_max; ++l) {
            if (!p->alloc((void**)&p->phi_split[mu][l], bytes)) return MM_ERR_NOMEM;
            rc = split_matrix(p->prec, p->phi[mu][l], n, 1, 0,
                              matrix_view(p->prec, (uint8_t*)p->phi_split[mu][l], n, n), kBParts, s);
            if (rc) return rc;
        }
        if (!p->tridiag && p->d == 2) {   // A_mu minus its band: the dense part of K u (d = 2)
            if (!p->alloc((void**)&p->rem_split[mu], bytes)) return MM_ERR_NOMEM;
            rc = split_matrix(p->prec, p->A[mu], n, 1, 1,
                              matrix_view(p->prec, (uint8_t*)p->rem_split[mu], n, n), kBParts, s);
            if (rc) return rc;
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
    const int n = (int)p->n[mu - 1];
    const PartView M = matrix_view(p->prec, (uint8_t*)p->phi_split[mu - 1][ell], n, n);
    TcOut o{};
    o.last = mu == p->d;
    if (o.last) {
        o.y = yout;
        o.ldy = in.rows;
    } else {
        const PartView nx = mode_input_view(p, mu + 1, out_parts);
        o.parts = out_parts;
        o.part_pitch = nx.part_pitch;
        o.next_n = nx.n;
        o.next_p = nx.p;
        o.next_rows_per_i = in.rows / nx.n;
    }
    return tc_product(p->prec, in, M, o, p->status, s);
}

}  // namespace mm
