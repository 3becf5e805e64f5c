// Many independent 2D problems of uneven size advanced together (Section 3.2,
// exponential Euler eq. (19), one PHISPLIT Tucker per step), in the mixed forms.
//
// Instances of equal (n1, n2) form a class.  Each class keeps its operands packed
// instance after instance -- the mode-1 input W = K u + g in parts, the mode-2
// input, the two phi_1 matrices of every instance in parts, the FP32 result -- so
// that one pair of TMA maps per class addresses all of its instances.  A step is
// four launches whatever the number of instances:
//   prepass   W = K u + g(t, u) of every instance (32 x 32 tiles)
//   mode 1    one persistent tensor-core launch over the tiles of all classes
//   mode 2    the same for the second direction, FP32 out
//   update    u += tau y, FP64, every instance
// and within a run the update of one step and the prepass of the next are one
// launch (the state then alternates between the caller's buffers and a second set).
// The tiles of a mode are ordered by decreasing cost and taken round-robin by one
// CTA per SM.  The tile width (nc) is picked at creation by timing the candidate
// tilings on the batch itself (mm_tune.autotune), and expint_batch_run captures
// its steps in a CUDA graph, so a run is one graph launch.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <map>
#include <vector>

#include "forms.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

namespace {

constexpr int kChunk = 8192;           // elements per chunk of the elementwise passes
constexpr int kNcCandidates[] = {160, 128, 96, 64};

// Device table, one 96-byte entry per instance, fields used together side by side
// (the kernels read an entry with a few 16-byte loads).
struct alignas(16) BInst {
    double* U;                         // the caller's state
    double* S;                         // the other state buffer of the fused passes
    float* y;                          // this instance's FP32 Tucker result
    uint8_t* w0;                       // its mode-1 input, part 0 (part q at q w_part_pitch elements)
    const float* coef1;                // [a | c | row sum] of the band of A_1, A_2
    const float* coef2;
    int64_t w_part_pitch;
    double tau;
    int n1, n2, p1, pad;
    float g0, g1, g2, g3;              // g = g0 + g1 u + g2 u^2 + g3 u^3 in FP32 (zeros: g = 0)
};

// W = K u + g(t, u) in parts, the stencil from differences of the double-float
// split of the state (the arithmetic of the single-problem mixed prepass, d = 2).
// Work unit: a 32 x 32 tile of one instance (a host table lists every tile, instance
// after instance, {instance, a_1, a_2}); each block takes one contiguous range of
// tiles.  A tile and its one-element halo are split once into the float2 plane sp,
// so each state value is read and split ~1.13 times instead of five.  Thread
// (lane c, warp w) owns column i_1 = a_1 + c and rows i_2 = a_2 + w + 8 q of the tile
// (q = 0..3): it loads, splits and later evaluates exactly those four values, with
// plain index arithmetic and coalesced rows; threads 0..131 also load one value each
// of the halo ring (the rows above and below, the columns left and right).  The next
// tile's values are loaded into registers while this one's stencil runs.
constexpr int kT = 32;
constexpr int kW = kT + 2;                          // a tile with its halo, per side
constexpr int kRing = 4 * kT + 4;                   // 132 halo values around a tile
constexpr int kRowsPer = kT / 8;                    // rows of the tile per thread

// Halo ring position t = 0..131 -> (row, column) of the tile, both in [-1, 32]:
// the row above (t < 34), the row below, the column left, the column right.
__device__ __forceinline__ void ring_pos(int t, int& r, int& c) {
    if (t < kW) { r = -1; c = t - 1; }
    else if (t < 2 * kW) { r = kT; c = t - kW - 1; }
    else if (t < 2 * kW + kT) { r = t - 2 * kW; c = -1; }
    else { r = t - 2 * kW - kT; c = kT; }
}

// FUSE: the previous step's update comes first: the state that the stencil sees is
// u' = u + tau y (the update pass's FMA, from the state buffer `from` -- 0: U, 1: S --
// and the previous Tucker result y), formed for every value of the tile and its halo,
// and each tile writes its own values of u' to the other buffer (reads and writes
// never touch the same buffer, so neighbouring tiles can run in any order).
template <class F, bool FUSE>
__global__ void __launch_bounds__(256, 4) batch_prepass_kernel(const BInst* __restrict__ tab,
                                                            const int4* __restrict__ tiles, int64_t ntiles,
                                                            int from, unsigned int* status) {
    using PT = typename std::conditional<F::kElem == 4, uint32_t, uint16_t>::type;
    __shared__ float2 sp[kW][kW];
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t T0 = blockIdx.x * per, T1 = min(ntiles, T0 + per);
    if (T0 >= T1) return;
    const int c = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool ring = threadIdx.x < kRing;
    int rr = 0, rc = 0;
    if (ring) ring_pos(threadIdx.x, rr, rc);
    double ui[kRowsPer], ur = 0.0;              // this thread's values of the tile, its ring value
    float yi[FUSE ? kRowsPer : 1], yr = 0.f;
    // global loads of a tile's values, left in flight (positions within an instance
    // fit 32 bits)
    auto fetch = [&](const int4 t) {
        const BInst& bi = tab[t.x];
        const double* U = (FUSE && from) ? bi.S : bi.U;
        const float* y = bi.y;
        const int n1 = bi.n1, n2 = bi.n2;
        const int i1 = t.y + c;
        const int o = i1 + n1 * (t.z + w);
#pragma unroll
        for (int q = 0; q < kRowsPer; ++q) {
            const bool in = i1 < n1 && t.z + w + 8 * q < n2;
            ui[q] = in ? __ldg(U + (o + 8 * q * n1)) : 0.0;
            if (FUSE) yi[FUSE ? q : 0] = in ? __ldg(y + (o + 8 * q * n1)) : 0.f;
        }
        if (ring) {
            const int j1 = t.y + rc, j2 = t.z + rr;
            const bool in = (unsigned)j1 < (unsigned)n1 && (unsigned)j2 < (unsigned)n2;
            ur = in ? __ldg(U + (j1 + n1 * j2)) : 0.0;
            if (FUSE) yr = in ? __ldg(y + (j1 + n1 * j2)) : 0.f;
        }
    };
    int4 cur = __ldg(tiles + T0);
    fetch(cur);
    bool bad = false;
    for (int64_t T = T0; T < T1; ++T) {
        // this tile's instance data (loaded before the stores below, which cannot
        // alias them once in registers)
        const BInst& bi = tab[cur.x];
        const int n1 = bi.n1, n2 = bi.n2, p1 = bi.p1;
        const float* cf1 = bi.coef1;
        const float* cf2 = bi.coef2;
        PT* const wt = (PT*)bi.w0;
        const int64_t wpp = bi.w_part_pitch;
        const float g0 = bi.g0, g1 = bi.g1, g2 = bi.g2, g3 = bi.g3;
        const int a1 = cur.y, a2 = cur.z;
        const int i1 = a1 + c;
        const bool in1 = i1 < n1;
        float2 ctr[kRowsPer];                   // this thread's values, split
#pragma unroll
        for (int q = 0; q < kRowsPer; ++q) {
            const int i2 = a2 + w + 8 * q;
            double v = ui[q];
            if (FUSE && in1 && i2 < n2) {
                v = fma(bi.tau, mx::f2d(yi[FUSE ? q : 0]), v);
                bad |= !mx::finite_bits(v);
                (from ? bi.U : bi.S)[i1 + n1 * i2] = v;
            }
            mx::d2ff(v, ctr[q].x, ctr[q].y);
            sp[w + 8 * q + 1][c + 1] = ctr[q];
        }
        if (ring) {
            double v = ur;
            const int j1 = a1 + rc, j2 = a2 + rr;
            if (FUSE && (unsigned)j1 < (unsigned)n1 && (unsigned)j2 < (unsigned)n2)
                v = fma(bi.tau, mx::f2d(yr), v);
            float2 h;
            mx::d2ff(v, h.x, h.y);
            sp[rr + 1][rc + 1] = h;
        }
        if (T + 1 < T1) {                // the next tile's loads overlap this tile's stencil
            cur = __ldg(tiles + T + 1);
            fetch(cur);
        }
        // coefficients along i_1 are fixed for this thread's column of the tile
        const float c1a = in1 ? __ldg(cf1 + i1) : 0.f, c1c = in1 ? __ldg(cf1 + n1 + i1) : 0.f,
                    c1s = in1 ? __ldg(cf1 + 2 * n1 + i1) : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kRowsPer; ++q) {
            const int r = w + 8 * q;
            const int i2 = a2 + r;
            if (!in1 || i2 >= n2) continue;
            const float uh = ctr[q].x, ul = ctr[q].y;
            const float u = uh + ul;
            // g is autonomous in a batch: 0 or a cubic (zero coefficients for g = 0)
            float acc = fmaf(fmaf(fmaf(g3, u, g2), u, g1), u, g0);
            // the edge coefficients are exactly zero and the halo holds zeros there
            acc = fmaf(c1s, u, acc);
            acc = fmaf(c1a, (sp[r + 1][c].x - uh) + (sp[r + 1][c].y - ul), acc);
            acc = fmaf(c1c, (sp[r + 1][c + 2].x - uh) + (sp[r + 1][c + 2].y - ul), acc);
            acc = fmaf(__ldg(cf2 + 2 * n2 + i2), u, acc);
            acc = fmaf(__ldg(cf2 + i2), (sp[r][c + 1].x - uh) + (sp[r][c + 1].y - ul), acc);
            acc = fmaf(__ldg(cf2 + n2 + i2), (sp[r + 2][c + 1].x - uh) + (sp[r + 2][c + 1].y - ul), acc);
            uint32_t v[3];
            split_parts<F>(acc, 0.f, v);
            PT* wp = wt + (i1 + p1 * i2);
            wp[0] = (PT)v[0];
            wp[wpp] = (PT)v[1];
            if (F::kAParts == 3) wp[2 * wpp] = (PT)v[2];
        }
        __syncthreads();
    }
    if (FUSE && bad) atomicOr(status, MM_STATUS_NONFINITE);
}

// The same pass with two adjacent columns per thread, for batches whose every
// instance has an even n_1 and 16-byte aligned states (then every pair of a row starts
// on a 16-byte boundary): thread (lane, warp) owns columns 2 cp, 2 cp + 1 (cp = lane
// mod 16) of rows r0 = lane / 16 + 2 warp and r0 + 16, loads and stores state pairs with
// 16-byte accesses, reads its neighbours with 16-byte shared loads from a split plane
// whose column c sits at index c + 2, and stores the parts of two outputs per 32-bit
// (BF16) or 64-bit (TF32) store.  Every output's arithmetic and its order are
// batch_prepass_kernel's, so the two kernels agree bit for bit.
template <class F, bool FUSE>
__global__ void __launch_bounds__(256, 4) batch_prepass2_kernel(const BInst* __restrict__ tab,
                                                             const int4* __restrict__ tiles, int64_t ntiles,
                                                             int from, unsigned int* status) {
    constexpr int kPW = kT + 4;                     // split-plane row: halo, 32 columns, halo, pad
    __shared__ __align__(16) float2 sp[kW][kPW];
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t T0 = blockIdx.x * per, T1 = min(ntiles, T0 + per);
    if (T0 >= T1) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cp = lane & 15, r0 = (lane >> 4) + 2 * w, j0 = 2 * cp + 2;
    const bool ring = threadIdx.x < kRing;
    int rr = 0, rc = 0;
    if (ring) ring_pos(threadIdx.x, rr, rc);
    double2 ui[2];
    double ur = 0.0;
    float2 yi[FUSE ? 2 : 1];
    float yr = 0.f;
    auto fetch = [&](const int4 t) {
        const BInst& bi = tab[t.x];
        const double* U = (FUSE && from) ? bi.S : bi.U;
        const float* y = bi.y;
        const int n1 = bi.n1, n2 = bi.n2;
        const int i1 = t.y + 2 * cp;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i2 = t.z + r0 + 16 * q;
            const bool in = i1 < n1 && i2 < n2;
            const int o = i1 + n1 * i2;
            ui[q] = in ? __ldg((const double2*)(U + o)) : make_double2(0.0, 0.0);
            if (FUSE) yi[FUSE ? q : 0] = in ? __ldg((const float2*)(y + o)) : make_float2(0.f, 0.f);
        }
        if (ring) {
            const int j1 = t.y + rc, j2 = t.z + rr;
            const bool in = (unsigned)j1 < (unsigned)n1 && (unsigned)j2 < (unsigned)n2;
            ur = in ? __ldg(U + (j1 + n1 * j2)) : 0.0;
            if (FUSE) yr = in ? __ldg(y + (j1 + n1 * j2)) : 0.f;
        }
    };
    int4 cur = __ldg(tiles + T0);
    fetch(cur);
    bool bad = false;
    for (int64_t T = T0; T < T1; ++T) {
        const BInst& bi = tab[cur.x];
        const int n1 = bi.n1, n2 = bi.n2, p1 = bi.p1;
        const float* cf1 = bi.coef1;
        const float* cf2 = bi.coef2;
        uint8_t* const wt = bi.w0;
        const uint32_t wpp = (uint32_t)bi.w_part_pitch;
        const float g0 = bi.g0, g1 = bi.g1, g2 = bi.g2, g3 = bi.g3;
        const int a1 = cur.y, a2 = cur.z;
        const int i1 = a1 + 2 * cp;
        const bool in1 = i1 < n1;               // n1 even: both columns, or neither
        float4 ctr[2];                          // this thread's values, split: (hi, lo) x 2
        if (FUSE) {
            const double tau = bi.tau;
            double* D = from ? bi.U : bi.S;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i2 = a2 + r0 + 16 * q;
                double2 v = ui[q];
                if (in1 && i2 < n2) {
                    v.x = fma(tau, mx::f2d(yi[FUSE ? q : 0].x), v.x);
                    v.y = fma(tau, mx::f2d(yi[FUSE ? q : 0].y), v.y);
                    bad |= !mx::finite_bits(v.x) || !mx::finite_bits(v.y);
                    *(double2*)(D + (i1 + n1 * i2)) = v;
                }
                mx::d2ff(v.x, ctr[q].x, ctr[q].y);
                mx::d2ff(v.y, ctr[q].z, ctr[q].w);
                *(float4*)&sp[r0 + 16 * q + 1][j0] = ctr[q];
            }
            if (ring) {
                double v = ur;
                const int j1 = a1 + rc, j2 = a2 + rr;
                if ((unsigned)j1 < (unsigned)n1 && (unsigned)j2 < (unsigned)n2) v = fma(tau, mx::f2d(yr), v);
                float2 h;
                mx::d2ff(v, h.x, h.y);
                sp[rr + 1][rc + 2] = h;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                mx::d2ff(ui[q].x, ctr[q].x, ctr[q].y);
                mx::d2ff(ui[q].y, ctr[q].z, ctr[q].w);
                *(float4*)&sp[r0 + 16 * q + 1][j0] = ctr[q];
            }
            if (ring) {
                float2 h;
                mx::d2ff(ur, h.x, h.y);
                sp[rr + 1][rc + 2] = h;
            }
        }
        if (T + 1 < T1) {                // the next tile's loads overlap this tile's stencil
            cur = __ldg(tiles + T + 1);
            fetch(cur);
        }
        float c1a[2], c1c[2], c1s[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            c1a[j] = in1 ? __ldg(cf1 + i1 + j) : 0.f;
            c1c[j] = in1 ? __ldg(cf1 + n1 + i1 + j) : 0.f;
            c1s[j] = in1 ? __ldg(cf1 + 2 * n1 + i1 + j) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = r0 + 16 * q;
            const int i2 = a2 + r;
            if (!in1 || i2 >= n2) continue;
            const float2 lft = sp[r + 1][j0 - 1], rgt = sp[r + 1][j0 + 2];
            const float4 up = *(const float4*)&sp[r][j0];
            const float4 dn = *(const float4*)&sp[r + 2][j0];
            const float2 cc[2] = {make_float2(ctr[q].x, ctr[q].y), make_float2(ctr[q].z, ctr[q].w)};
            const float2 nbl[2] = {lft, cc[0]}, nbr[2] = {cc[1], rgt};
            const float2 nbu[2] = {make_float2(up.x, up.y), make_float2(up.z, up.w)};
            const float2 nbd[2] = {make_float2(dn.x, dn.y), make_float2(dn.z, dn.w)};
            const float c2s = __ldg(cf2 + 2 * n2 + i2), c2a = __ldg(cf2 + i2), c2c = __ldg(cf2 + n2 + i2);
            float out[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float uh = cc[j].x, ul = cc[j].y;
                const float u = uh + ul;
                // g is autonomous in a batch: 0 or a cubic (zero coefficients for g = 0)
                float acc = fmaf(fmaf(fmaf(g3, u, g2), u, g1), u, g0);
                // the edge coefficients are exactly zero and the halo holds zeros there
                acc = fmaf(c1s[j], u, acc);
                acc = fmaf(c1a[j], (nbl[j].x - uh) + (nbl[j].y - ul), acc);
                acc = fmaf(c1c[j], (nbr[j].x - uh) + (nbr[j].y - ul), acc);
                acc = fmaf(c2s, u, acc);
                acc = fmaf(c2a, (nbu[j].x - uh) + (nbu[j].y - ul), acc);
                acc = fmaf(c2c, (nbd[j].x - uh) + (nbd[j].y - ul), acc);
                out[j] = acc;
            }
            uint32_t v0[3], v1[3];
            split_parts<F>(out[0], 0.f, v0);
            split_parts<F>(out[1], 0.f, v1);
            const uint32_t pos = (uint32_t)(i1 + p1 * i2);          // even: n1, p1 even
            if (F::kElem == 2) {
                uint32_t* wp = (uint32_t*)((uint16_t*)wt + pos);
                wp[0] = v0[0] | (v1[0] << 16);
                wp[wpp >> 1] = v0[1] | (v1[1] << 16);
                if (F::kAParts == 3) wp[wpp] = v0[2] | (v1[2] << 16);
            } else {
                uint2* wp = (uint2*)((uint32_t*)wt + pos);
                wp[0] = make_uint2(v0[0], v1[0]);
                wp[wpp >> 1] = make_uint2(v0[1], v1[1]);
                if (F::kAParts == 3) wp[wpp] = make_uint2(v0[2], v1[2]);
            }
        }
        __syncthreads();
    }
    if (FUSE && bad) atomicOr(status, MM_STATUS_NONFINITE);
}

// U = u + tau y (one DFMA per element) from the state buffer `from` (0: U itself,
// 1: S), non-finite results flagged.
__global__ void __launch_bounds__(256) batch_update_kernel(const BInst* __restrict__ tab,
                                                           const int4* __restrict__ chunks, int64_t nchunks,
                                                           int from, unsigned int* status) {
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        double* U = tab[ch.x].U;        // loaded once: the stores to U cannot alias them
        const double* src = from ? tab[ch.x].S : U;
        const float* y = tab[ch.x].y;
        const double tau = tab[ch.x].tau;
        bool bad = false;
        for (int e = threadIdx.x; e < ch.z; e += blockDim.x) {
            const int i = ch.y + e;
            const double v = fma(tau, mx::f2d(__ldg(y + i)), src[i]);
            bad |= !mx::finite_bits(v);
            U[i] = v;
        }
        if (bad) atomicOr(status, MM_STATUS_NONFINITE);
    }
}

}  // namespace

}  // namespace mm

using namespace mm;

struct mm_batch_s {
    int count = 0, prec = 0, scheme = 0;
    int64_t total_dof = 0;
    struct Cls {
        int n1, n2;
        std::vector<int> members;
        uint8_t *W = nullptr, *P = nullptr, *phi1 = nullptr, *phi2 = nullptr;
        float* y = nullptr;
    };
    std::vector<Cls> cls;
    std::vector<TcClassSpec> spec1, spec2;   // per class, mode 1 and mode 2
    std::vector<int> nc_cap;                 // per class (same for both modes)
    float tune_ms_uniform = 0.f;             // autotuner: best uniform width's Tucker time
    float tune_ms_chosen = 0.f;              //   and the time of the widths kept
    int tune_per_class = 0;                  //   1: the per-class widths won
    int tile_order = 0;                      //   0 round-robin, 1 alternate rounds reversed
    struct Launch {                          // groups of <= MM_TC_MAX_CLASSES classes
        int c0, nc;
        int4* tiles1 = nullptr;
        int4* tiles2 = nullptr;
        int64_t n1 = 0, n2 = 0;              // tiles in use
        int64_t cap1 = 0, cap2 = 0;          // tiles the arrays hold
    };
    std::vector<Launch> launches;
    BInst* tab = nullptr;
    int4* chunks = nullptr;                 // update pass: {instance, start, length}
    int64_t nchunks = 0;
    int4* ptiles = nullptr;                 // prepass: {instance, a_1, a_2} of every 32 x 32 tile
    bool paired = false;                    // every n1 even, every state 16-byte aligned
    int64_t ntiles = 0;
    unsigned int* status = nullptr;
    int use_graph = 1;
    cudaStream_t cap = nullptr;            // capture stream of the step graph
    cudaGraphExec_t exec = nullptr;
    int exec_steps = -1;
    std::vector<void*> owned;

    bool alloc(void** p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; return false; }
        owned.push_back(*p);
        return true;
    }
    ~mm_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        for (void* q : owned) cudaFree(q);
    }
};

namespace {

// Tile order of a grouped launch: the list comes sorted by decreasing cost and the
// C = min(tiles, SMs) CTAs take it round-robin (CTA j: tiles j, j + C, ...).  Order 1
// reverses every other round of C tiles, so that the CTA given the dearest tile of one
// round gets the cheapest of the next (the autotuner keeps it if it is faster).
void order_tiles(std::vector<int4>& t, int order) {
    if (order != 1) return;
    const size_t C = (size_t)std::min<int64_t>((int64_t)t.size(), num_sms());
    for (size_t w = C; w < t.size(); w += 2 * C) std::reverse(t.begin() + w, t.begin() + std::min(t.size(), w + C));
}

int build_tiles(mm_batch_s* b, cudaStream_t s) {
    for (auto& L : b->launches) {
        std::vector<int4> t1, t2;
        int rc = tc_group_tiles(b->prec, &b->spec1[L.c0], L.nc, &b->nc_cap[L.c0], t1);
        if (!rc) rc = tc_group_tiles(b->prec, &b->spec2[L.c0], L.nc, &b->nc_cap[L.c0], t2);
        if (rc) return rc;
        order_tiles(t1, b->tile_order);
        order_tiles(t2, b->tile_order);
        if (!L.tiles1 || (int64_t)t1.size() > L.cap1 || (int64_t)t2.size() > L.cap2) return MM_ERR_ARG;
        L.n1 = (int64_t)t1.size();
        L.n2 = (int64_t)t2.size();
        MM_CUDA_TRY(cudaMemcpyAsync(L.tiles1, t1.data(), t1.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        MM_CUDA_TRY(cudaMemcpyAsync(L.tiles2, t2.data(), t2.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        MM_CUDA_TRY(cudaStreamSynchronize(s));   // the host vectors go out of scope
    }
    return MM_OK;
}

int tucker_modes(mm_batch_s* b, cudaStream_t s) {
    for (auto& L : b->launches) {
        int rc = tc_group_product(b->prec, &b->spec1[L.c0], L.nc, &b->nc_cap[L.c0], L.tiles1, L.n1, b->status, s);
        if (rc) return rc;
    }
    for (auto& L : b->launches) {
        int rc = tc_group_product(b->prec, &b->spec2[L.c0], L.nc, &b->nc_cap[L.c0], L.tiles2, L.n2, b->status, s);
        if (rc) return rc;
    }
    return MM_OK;
}

int64_t ew_grid(const mm_batch_s* b) { return std::min<int64_t>(b->nchunks, (int64_t)num_sms() * 8); }

typedef void (*PrepassKernel)(const BInst*, const int4*, int64_t, int, unsigned int*);
PrepassKernel prepass_kernel_of(int prec, bool fuse, bool paired) {
    if (paired)
        return prec == MM_BF16X3
                   ? (fuse ? batch_prepass2_kernel<FormBF16, true> : batch_prepass2_kernel<FormBF16, false>)
                   : (fuse ? batch_prepass2_kernel<FormTF32, true> : batch_prepass2_kernel<FormTF32, false>);
    return prec == MM_BF16X3 ? (fuse ? batch_prepass_kernel<FormBF16, true> : batch_prepass_kernel<FormBF16, false>)
                             : (fuse ? batch_prepass_kernel<FormTF32, true> : batch_prepass_kernel<FormTF32, false>);
}

// W = K u + g(u) of every instance (the batch's nonlinearities are autonomous);
// fused: of u' = u + tau y from state buffer `from`, u' written to the other one.
int prepass(mm_batch_s* b, bool fuse, int from, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(b->ntiles, (int64_t)num_sms() * 8);
    TraceScope tr(KC_PREPASS, s);
    auto k = prepass_kernel_of(b->prec, fuse, b->paired);
    k<<<(unsigned)grid, 256, 0, s>>>(b->tab, b->ptiles, b->ntiles, from, b->status);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int update(mm_batch_s* b, int from, cudaStream_t s) {
    TraceScope tr(KC_SPLIT, s);
    batch_update_kernel<<<(unsigned)ew_grid(b), 256, 0, s>>>(b->tab, b->chunks, b->nchunks, from, b->status);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

// nsteps exponential Euler steps from the caller's states U back into U.  Between two
// steps the update u + tau y is fused into the next step's prepass, which reads one
// state buffer and writes the other (U, S, U, ...); the last step's update writes U
// (in place, or from S).  The arithmetic of every value is that of separate passes.
int run_steps(mm_batch_s* b, int nsteps, cudaStream_t s) {
    int from = 0;                        // the buffer that holds the current state
    int rc = prepass(b, false, 0, s);
    for (int k = 0; k < nsteps && !rc; ++k) {
        rc = tucker_modes(b, s);
        if (rc) break;
        if (k + 1 < nsteps) {
            rc = prepass(b, true, from, s);
            from ^= 1;
        } else {
            rc = update(b, from, s);
        }
    }
    return rc;
}

// Mean time of `reps` runs of fn after one warm-up run, in ms.
template <class Fn>
int time_ms(Fn fn, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms, int reps = 3) {
    int rc = fn();
    if (rc) return rc;
    MM_CUDA_TRY(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && !rc; ++r) rc = fn();
    if (rc) return rc;
    MM_CUDA_TRY(cudaEventRecord(e1, s));
    MM_CUDA_TRY(cudaEventSynchronize(e1));
    MM_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    *ms /= reps;
    return MM_OK;
}

// Both directions of class c alone at width nc: its tiles go into its launch
// group's tile arrays (sized for the narrowest width of every class in the group).
int time_class(mm_batch_s* b, int c, int nc, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    const mm_batch_s::Launch* L = nullptr;
    for (auto& G : b->launches)
        if (c >= G.c0 && c < G.c0 + G.nc) L = &G;
    if (!L) return MM_ERR_ARG;
    std::vector<int4> t1, t2;
    int rc = tc_group_tiles(b->prec, &b->spec1[c], 1, &nc, t1);
    if (!rc) rc = tc_group_tiles(b->prec, &b->spec2[c], 1, &nc, t2);
    if (rc) return rc;
    if ((int64_t)t1.size() > L->cap1 || (int64_t)t2.size() > L->cap2) return MM_ERR_ARG;
    MM_CUDA_TRY(cudaMemcpyAsync(L->tiles1, t1.data(), t1.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    MM_CUDA_TRY(cudaMemcpyAsync(L->tiles2, t2.data(), t2.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    MM_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t n1 = (int64_t)t1.size(), n2 = (int64_t)t2.size();
    return time_ms([&] {
        int r = tc_group_product(b->prec, &b->spec1[c], 1, &nc, L->tiles1, n1, b->status, s);
        return r ? r : tc_group_product(b->prec, &b->spec2[c], 1, &nc, L->tiles2, n2, b->status, s);
    }, s, e0, e1, ms);
}

// The autotuner, on the batch's own Tucker launches (they touch only the
// workspace):
//   1. every candidate width for all classes at once; the fastest is the uniform choice;
//   2. each class alone at every candidate width (a size class's best width depends
//      on its n: how its columns split into tiles and how many tiles it brings);
//   3. the per-class choices together, kept only if faster than the uniform one;
//   4. the chosen widths with every other round of tiles reversed (order_tiles), kept
//      only if faster.
// Tiles within a launch are always ordered by decreasing cost (the CTAs take them
// round-robin).  The times of both schedules are kept for expint_batch_schedule.
int autotune(mm_batch_s* b, cudaStream_t s) {
    cudaEvent_t e0, e1;
    MM_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MM_ERR_CUDA;
    }
    const int ncls = (int)b->cls.size();
    auto all_modes = [&] { return tucker_modes(b, s); };
    int rc = MM_OK, best = -1;
    float best_ms = 0.f;
    for (int cand : kNcCandidates) {
        for (auto& v : b->nc_cap) v = cand;
        float ms = 0.f;
        if ((rc = build_tiles(b, s)) || (rc = time_ms(all_modes, s, e0, e1, &ms))) break;
        if (best < 0 || ms < best_ms) { best = cand; best_ms = ms; }
    }
    std::vector<int> per(ncls, best);
    for (int c = 0; c < ncls && !rc; ++c) {
        float cbest = -1.f;
        for (int cand : kNcCandidates) {
            float ms = 0.f;
            if ((rc = time_class(b, c, cand, s, e0, e1, &ms))) break;
            if (cbest < 0.f || ms < cbest) { cbest = ms; per[c] = cand; }
        }
    }
    float per_ms = 0.f;
    if (!rc) {
        b->nc_cap = per;
        if (!(rc = build_tiles(b, s))) rc = time_ms(all_modes, s, e0, e1, &per_ms);
    }
    if (!rc) {
        b->tune_ms_uniform = best_ms;
        b->tune_per_class = per_ms < best_ms;
        b->tune_ms_chosen = b->tune_per_class ? per_ms : best_ms;
        if (!b->tune_per_class)
            for (auto& v : b->nc_cap) v = best;
        // 4. the tile order of the chosen widths: alternate rounds reversed, kept if faster
        b->tile_order = 1;
        float ord_ms = 0.f;
        if (!(rc = build_tiles(b, s)) && !(rc = time_ms(all_modes, s, e0, e1, &ord_ms))) {
            if (ord_ms < b->tune_ms_chosen) b->tune_ms_chosen = ord_ms;
            else b->tile_order = 0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return build_tiles(b, s);
}

// Class grouping of the sizes (n1, n2), in order of first appearance.
std::vector<std::pair<int, int>> size_classes(int count, const int64_t* n1, const int64_t* n2,
                                              std::vector<int>* cls_of) {
    std::map<std::pair<int, int>, int> idx;
    std::vector<std::pair<int, int>> out;
    cls_of->assign(count, 0);
    for (int j = 0; j < count; ++j) {
        const std::pair<int, int> key((int)n1[j], (int)n2[j]);
        auto it = idx.find(key);
        if (it == idx.end()) {
            it = idx.emplace(key, (int)out.size()).first;
            out.push_back(key);
        }
        (*cls_of)[j] = it->second;
    }
    return out;
}

}  // namespace

extern "C" int mm_batch_tile_plan(int count, const int64_t* n1, const int64_t* n2, int prec, int nc_cap,
                                  int mode, int32_t* tiles, int64_t max_tiles, int64_t* ntiles) {
    if (count < 1 || !n1 || !n2 || !ntiles || (mode != 1 && mode != 2)) return MM_ERR_ARG;
    if ((prec != MM_TF32X3 && prec != MM_BF16X3) || nc_cap < 16 || nc_cap > 160 || nc_cap % 16) return MM_ERR_ARG;
    for (int j = 0; j < count; ++j)
        if (n1[j] < 1 || n1[j] > 8192 || n2[j] < 1 || n2[j] > 8192) return MM_ERR_SHAPE;
    std::vector<int> cls_of;
    const auto sizes = size_classes(count, n1, n2, &cls_of);
    if (sizes.size() > MM_TC_MAX_CLASSES) return MM_ERR_UNSUPPORTED;
    std::vector<TcClassSpec> spec(sizes.size());
    std::vector<int> caps(sizes.size(), nc_cap);
    for (size_t c = 0; c < sizes.size(); ++c) {
        const int a = mode == 1 ? sizes[c].first : sizes[c].second;    // contraction length
        const int r = mode == 1 ? sizes[c].second : sizes[c].first;    // rows per instance
        spec[c].X.n = a; spec[c].M.n = a; spec[c].rows = r; spec[c].ncols = a;
        spec[c].count = (int)std::count(cls_of.begin(), cls_of.end(), (int)c);
    }
    std::vector<int4> t;
    int rc = tc_group_tiles(prec, spec.data(), (int)spec.size(), caps.data(), t);
    if (rc) return rc;
    *ntiles = (int64_t)t.size();
    if (tiles) {
        if (max_tiles < (int64_t)t.size()) return MM_ERR_ARG;
        for (size_t i = 0; i < t.size(); ++i) {
            // instance index within its class -> global instance index
            int k = -1, seen = -1;
            for (int j = 0; j < count && k < 0; ++j)
                if (cls_of[j] == t[i].x && ++seen == t[i].y) k = j;
            tiles[4 * i + 0] = k;
            tiles[4 * i + 1] = t[i].z;
            tiles[4 * i + 2] = t[i].w;
            tiles[4 * i + 3] = t[i].x;
        }
    }
    return MM_OK;
}

extern "C" int expint_batch_create(mm_batch* out, int count, const mm_plan* plans, const mm_nonlin* g,
                                   double* const* U, int scheme, const mm_tune* tune, void* stream) {
    NvtxScope nv("expint_batch_create");
    if (!out) return MM_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !plans || !U) return MM_ERR_ARG;
    if (scheme != MM_EXPEULER) return MM_ERR_UNSUPPORTED;
    const int prec = plans[0] ? plans[0]->prec : -1;
    if (prec != MM_TF32X3 && prec != MM_BF16X3) return MM_ERR_UNSUPPORTED;
    std::vector<int64_t> n1(count), n2(count);
    for (int j = 0; j < count; ++j) {
        const mm_plan p = plans[j];
        if (!p || !U[j]) return MM_ERR_ARG;
        if (p->prec != prec || p->d != 2 || !p->tridiag || p->ell_max < 1) return MM_ERR_UNSUPPORTED;
        if (g && g[j].kind != MM_G_NONE && g[j].kind != MM_G_CUBIC) return MM_ERR_UNSUPPORTED;
        if ((uintptr_t)U[j] & 7) return MM_ERR_ARG;
        n1[j] = p->n[0];
        n2[j] = p->n[1];
        if (p->N >= (int64_t(1) << 31)) return MM_ERR_SHAPE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    mm_batch_s* b = new mm_batch_s();
    b->count = count; b->prec = prec; b->scheme = scheme;
    b->paired = true;
    for (int j = 0; j < count; ++j) b->paired = b->paired && n1[j] % 2 == 0 && !((uintptr_t)U[j] & 15);
    b->use_graph = tune ? tune->graph : 1;
    int rc = MM_OK;
    std::vector<int> cls_of;
    const auto sizes = size_classes(count, n1.data(), n2.data(), &cls_of);
    const int E = form_elem_bytes(prec), AP = form_parts(prec);
    std::vector<BInst> tab(count);
    std::vector<int4> chunks;
    b->cls.resize(sizes.size());
    b->spec1.resize(sizes.size());
    b->spec2.resize(sizes.size());
    b->nc_cap.assign(sizes.size(), 160);
    if (tune && tune->nc_cap) {
        if (tune->nc_cap < 16 || tune->nc_cap > 160 || tune->nc_cap % 16) { delete b; return MM_ERR_ARG; }
        for (auto& v : b->nc_cap) v = tune->nc_cap;
    }
    for (int j = 0; j < count; ++j) b->cls[cls_of[j]].members.push_back(j);
    for (size_t c = 0; c < sizes.size(); ++c) {
        auto& C = b->cls[c];
        C.n1 = sizes[c].first;
        C.n2 = sizes[c].second;
        const int cnt = (int)C.members.size();
        const int p1 = form_pitch(prec, C.n1), p2 = form_pitch(prec, C.n2);
        const int64_t nn = (int64_t)C.n1 * C.n2;
        if ((int64_t)p1 * C.n2 >= (int64_t(1) << 31)) {    // 32-bit positions within an instance
            rc = MM_ERR_SHAPE;
            goto fail;
        }
        if (!b->alloc((void**)&C.W, matrix_parts_bytes(prec, (int64_t)cnt * C.n2, C.n1, AP)) ||
            !b->alloc((void**)&C.P, matrix_parts_bytes(prec, (int64_t)cnt * C.n1, C.n2, AP)) ||
            !b->alloc((void**)&C.phi1, matrix_parts_bytes(prec, (int64_t)cnt * C.n1, C.n1, 3)) ||
            !b->alloc((void**)&C.phi2, matrix_parts_bytes(prec, (int64_t)cnt * C.n2, C.n2, 3)) ||
            !b->alloc((void**)&C.y, (size_t)cnt * nn * sizeof(float))) {
            rc = MM_ERR_NOMEM;
            goto fail;
        }
        // the phi_1 parts of every member, packed (part q of member k at rows k n..)
        for (int k = 0; k < cnt; ++k) {
            const mm_plan p = plans[C.members[k]];
            for (int mu = 0; mu < 2; ++mu) {
                const int n = mu == 0 ? C.n1 : C.n2, pp = mu == 0 ? p1 : p2;
                uint8_t* dst = mu == 0 ? C.phi1 : C.phi2;
                const size_t blk = (size_t)n * pp * E;
                for (int q = 0; q < 3; ++q)
                    if (cudaMemcpyAsync(dst + ((size_t)q * cnt + k) * blk, (const uint8_t*)p->phi_split[mu][1] + q * blk,
                                        blk, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                        rc = MM_ERR_CUDA;
                        goto fail;
                    }
            }
        }
        TcClassSpec& m1 = b->spec1[c];
        m1.X = matrix_view(prec, C.W, (int64_t)cnt * C.n2, C.n1);
        if (m1.X.part_pitch * 3 >= (int64_t(1) << 31)) b->paired = false;   // 32-bit part offsets
        m1.rows = C.n2;
        m1.M = matrix_view(prec, C.phi1, (int64_t)cnt * C.n1, C.n1);
        m1.ncols = C.n1;
        m1.count = cnt;
        m1.out.last = 0;
        m1.out.parts = C.P;
        m1.out.part_pitch = (int64_t)cnt * C.n1 * p2;
        m1.out.next_n = C.n2;
        m1.out.next_p = p2;
        m1.out.next_rows_per_i = 1;
        m1.p_stride = (int64_t)C.n1 * p2;
        TcClassSpec& m2 = b->spec2[c];
        m2.X = matrix_view(prec, C.P, (int64_t)cnt * C.n1, C.n2);
        m2.rows = C.n1;
        m2.M = matrix_view(prec, C.phi2, (int64_t)cnt * C.n2, C.n2);
        m2.ncols = C.n2;
        m2.count = cnt;
        m2.out.last = 1;
        m2.out.y = C.y;
        m2.out.ldy = C.n1;
        m2.y_stride = nn;
        for (int k = 0; k < cnt; ++k) {
            const int j = C.members[k];
            const mm_plan p = plans[j];
            BInst& e = tab[j];
            e.U = U[j];
            e.coef1 = p->coef3f[0];
            e.coef2 = p->coef3f[1];
            e.w0 = C.W + (size_t)k * C.n2 * p1 * E;
            e.w_part_pitch = m1.X.part_pitch;
            e.y = C.y + (int64_t)k * nn;
            e.n1 = C.n1; e.n2 = C.n2; e.p1 = p1; e.pad = 0;
            e.tau = p->tau;
            const PointwiseG pg = pointwise_of(g ? &g[j] : nullptr);
            e.g0 = pg.f0; e.g1 = pg.f1; e.g2 = pg.f2; e.g3 = pg.f3;
            for (int64_t s0 = 0; s0 < nn; s0 += kChunk)
                chunks.push_back(make_int4(j, (int)s0, (int)std::min<int64_t>(kChunk, nn - s0), 0));
            b->total_dof += nn;
        }
    }
    for (int c0 = 0; c0 < (int)sizes.size(); c0 += MM_TC_MAX_CLASSES) {
        mm_batch_s::Launch L;
        L.c0 = c0;
        L.nc = std::min<int>(MM_TC_MAX_CLASSES, (int)sizes.size() - c0);
        // room for the most tiles any candidate width makes (nc = 16 bounds them all)
        int64_t cap1 = 0, cap2 = 0;
        for (int c = c0; c < c0 + L.nc; ++c) {
            const int64_t cnt = b->cls[c].members.size();
            const int64_t a1 = b->cls[c].n1, a2 = b->cls[c].n2;
            cap1 += cnt * ((a2 + 127) / 128) * ((a1 + 15) / 16);
            cap2 += cnt * ((a1 + 127) / 128) * ((a2 + 15) / 16);
        }
        if (!b->alloc((void**)&L.tiles1, cap1 * sizeof(int4)) || !b->alloc((void**)&L.tiles2, cap2 * sizeof(int4))) {
            rc = MM_ERR_NOMEM;
            goto fail;
        }
        L.cap1 = cap1;
        L.cap2 = cap2;
        b->launches.push_back(L);
    }
    b->nchunks = (int64_t)chunks.size();
    {
        // the second state buffer of the fused passes, instance after instance
        double* S = nullptr;
        if (!b->alloc((void**)&S, (size_t)b->total_dof * sizeof(double))) {
            rc = MM_ERR_NOMEM;
            goto fail;
        }
        for (int j = 0; j < count; ++j) {
            tab[j].S = S;
            S += n1[j] * n2[j];
        }
    }
    {
        std::vector<int4> pt;
        for (int j = 0; j < count; ++j)
            for (int a2 = 0; a2 < n2[j]; a2 += kT)
                for (int a1 = 0; a1 < n1[j]; a1 += kT) pt.push_back(make_int4(j, a1, a2, 0));
        b->ntiles = (int64_t)pt.size();
        if (!b->alloc((void**)&b->ptiles, pt.size() * sizeof(int4)) ||
            cudaMemcpyAsync(b->ptiles, pt.data(), pt.size() * sizeof(int4), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = MM_ERR_NOMEM;
            goto fail;
        }
    }
    if (!b->alloc((void**)&b->tab, tab.size() * sizeof(BInst)) ||
        !b->alloc((void**)&b->chunks, chunks.size() * sizeof(int4)) ||
        !b->alloc((void**)&b->status, sizeof(unsigned int))) {
        rc = MM_ERR_NOMEM;
        goto fail;
    }
    if (cudaMemcpyAsync(b->tab, tab.data(), tab.size() * sizeof(BInst), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(b->status, 0, sizeof(unsigned int), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = MM_ERR_CUDA;
        goto fail;
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
    rc = build_tiles(b, s);
    if (rc) goto fail;
    // configure the grouped kernels (launch attributes) outside any later capture
    for (auto& L : b->launches) {
        rc = tc_group_product(prec, &b->spec1[L.c0], L.nc, &b->nc_cap[L.c0], L.tiles1, 0, b->status, s);
        if (rc) goto fail;
    }
    if (tune && tune->autotune && !tune->nc_cap) {
        // W from the initial states so the timed products see real operands
        rc = prepass(b, false, 0, s);
        if (rc) goto fail;
        rc = autotune(b, s);
        if (rc) goto fail;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = MM_ERR_CUDA; goto fail; }
    *out = b;
    return MM_OK;
fail:
    cudaStreamSynchronize(s);
    delete b;
    return rc;
}

// The nonlinearities of a batch are autonomous (g = 0 or a cubic in u), so t0 only
// documents the caller's clock.
extern "C" int expint_batch_run(mm_batch b, double t0, int nsteps, void* stream) {
    NvtxScope nv("expint_batch_run");
    if (!b || nsteps < 0 || !isfinite(t0)) return MM_ERR_ARG;
    if (nsteps == 0) return MM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->use_graph) return run_steps(b, nsteps, s);
    if (!b->exec || b->exec_steps != nsteps) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        MM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int rc = MM_OK;
        rc = run_steps(b, nsteps, b->cap);
        const cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
        if (rc || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc ? rc : MM_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            b->exec = nullptr;
            return MM_ERR_CUDA;
        }
        b->exec_steps = nsteps;
    }
    MM_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    // the launches inside the graph, for the launch counters
    trace_count(KC_PREPASS, nsteps);
    trace_count(KC_CONTRACT_TF32, (long long)nsteps * 2 * (long long)b->launches.size());
    trace_count(KC_SPLIT, 1);
    return MM_OK;
}

extern "C" int expint_batch_status(mm_batch b, int reset, void* stream) {
    if (!b) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int v = 0;
    MM_CUDA_TRY(cudaMemcpyAsync(&v, b->status, sizeof(v), cudaMemcpyDeviceToHost, s));
    MM_CUDA_TRY(cudaStreamSynchronize(s));
    if (reset) {
        MM_CUDA_TRY(cudaMemsetAsync(b->status, 0, sizeof(unsigned int), s));
        MM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return (int)v;
}

extern "C" int expint_batch_info(mm_batch b, int* nclasses, int* nc_cap, int64_t* tiles_mode1,
                                 int64_t* total_dof) {
    if (!b) return MM_ERR_ARG;
    if (nclasses) *nclasses = (int)b->cls.size();
    if (nc_cap) *nc_cap = b->nc_cap.empty() ? 0 : b->nc_cap[0];
    if (tiles_mode1) {
        int64_t t = 0;
        for (auto& L : b->launches) t += L.n1;
        *tiles_mode1 = t;
    }
    if (total_dof) *total_dof = b->total_dof;
    return MM_OK;
}

extern "C" int expint_batch_schedule(mm_batch b, int32_t* nc_per_class, int max_classes, int* nclasses,
                                     float* ms_uniform, float* ms_chosen) {
    if (!b || (nc_per_class && max_classes < (int)b->cls.size())) return MM_ERR_ARG;
    if (nclasses) *nclasses = (int)b->cls.size();
    if (nc_per_class)
        for (size_t c = 0; c < b->cls.size(); ++c) nc_per_class[c] = b->nc_cap[c];
    if (ms_uniform) *ms_uniform = b->tune_ms_uniform;
    if (ms_chosen) *ms_chosen = b->tune_ms_chosen;
    return b->tune_per_class;
}

extern "C" int expint_batch_tile_order(mm_batch b) {
    if (!b) return MM_ERR_ARG;
    return b->tile_order;
}

extern "C" int expint_batch_set_graph(mm_batch b, int on) {
    if (!b) return MM_ERR_ARG;
    b->use_graph = on != 0;
    return MM_OK;
}

extern "C" int expint_batch_destroy(mm_batch b) {
    if (!b) return MM_OK;
    cudaDeviceSynchronize();
    delete b;
    return MM_OK;
}

extern "C" int expint_batched(int count, const mm_plan* plans, const mm_nonlin* g, double* const* U, int scheme,
                              double t0, int nsteps, const mm_tune* tune, void* stream) {
    mm_batch b = nullptr;
    int rc = expint_batch_create(&b, count, plans, g, U, scheme, tune, stream);
    if (rc) return rc;
    rc = expint_batch_run(b, t0, nsteps, stream);
    if (!rc && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = MM_ERR_CUDA;
    expint_batch_destroy(b);
    return rc;
}
