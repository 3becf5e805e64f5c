// Many independent 2D problems of uneven size advanced together (Section 3.2,
// exponential Euler eq. (19), one PHISPLIT Tucker per step), in the mixed forms.
//
// Instances of equal (n1, n2) form a class.  Each class keeps its operands packed
// instance after instance -- the mode-1 input W = K u + g in parts, the mode-2
// input, the two phi_1 matrices of every instance in parts, the FP32 result -- so
// that one pair of TMA maps per class addresses all of its instances.  A step is
// four launches whatever the number of instances:
//   prepass   W = K u + g(t, u) of every instance (chunks of one instance each)
//   mode 1    one persistent tensor-core launch over the tiles of all classes
//   mode 2    the same for the second direction, FP32 out
//   update    u += tau y, FP64, every instance
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

struct BInst {                         // device table, one entry per instance
    double* U;
    const float* coef1;                // [a | c | row sum] of the band of A_1, A_2
    const float* coef2;
    uint8_t* wbase;                    // class buffer of mode-1 inputs
    float* y;                          // this instance's FP32 Tucker result
    int64_t w_part_pitch, w_off;
    int n1, n2, p1;
    double tau;
    PointwiseG g;
};

// W = K u + g(t, u) in parts, the stencil from differences of the double-float
// split of the state (the arithmetic of the single-problem mixed prepass, d = 2).
// A 32 x 32 tile of one instance and its one-element halo are split once into
// shared memory (each state value read and split ~1.1 times instead of five);
// 256 threads, four rows each.  Tiles are numbered instance after instance
// (tile_begin holds each instance's first tile) and each block takes one
// contiguous range, so it locates its instance once and then walks forward.
constexpr int kT = 32;
constexpr int kHalo = (kT + 2) * (kT + 2);          // 1156 values of a tile with its halo
constexpr int kPer = (kHalo + 255) / 256;           // of them per thread

struct TileAt {
    int inst, a1, a2;
};

__device__ __forceinline__ TileAt tile_at(const BInst* __restrict__ tab, const int64_t* __restrict__ tile_begin,
                                          int inst, int64_t T) {
    const int n1 = tab[inst].n1;
    const int tiles1 = (n1 + kT - 1) / kT;
    const int lt = (int)(T - __ldg(tile_begin + inst));
    return TileAt{inst, (lt % tiles1) * kT, (lt / tiles1) * kT};
}

template <class F>
__global__ void __launch_bounds__(256, 4) batch_prepass_kernel(const BInst* __restrict__ tab,
                                                            const int64_t* __restrict__ tile_begin, int count,
                                                            int64_t ntiles) {
    using PT = typename std::conditional<F::kElem == 4, uint32_t, uint16_t>::type;
    __shared__ float2 sp[kT + 2][kT + 2];
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t T0 = blockIdx.x * per, T1 = min(ntiles, T0 + per);
    if (T0 >= T1) return;
    int inst = 0, hi = count;                   // tile_begin[inst] <= T0 < tile_begin[hi]
    while (hi - inst > 1) {
        const int mid = (inst + hi) >> 1;
        if (__ldg(tile_begin + mid) <= T0) inst = mid;
        else hi = mid;
    }
    int64_t next = __ldg(tile_begin + inst + 1);
    double raw[kPer];
    // global loads of a tile's halo region, left in flight
    auto fetch = [&](const TileAt& ta) {
        const double* U = tab[ta.inst].U;
        const int n1 = tab[ta.inst].n1, n2 = tab[ta.inst].n2;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int e = threadIdx.x + 256 * k;
            const int r = e / (kT + 2), c = e % (kT + 2);
            const int i1 = ta.a1 - 1 + c, i2 = ta.a2 - 1 + r;
            raw[k] = (e < kHalo && i1 >= 0 && i1 < n1 && i2 >= 0 && i2 < n2) ? __ldg(U + i1 + (int64_t)n1 * i2)
                                                                             : 0.0;
        }
    };
    TileAt cur = tile_at(tab, tile_begin, inst, T0);
    fetch(cur);
    const int c = threadIdx.x % kT;
    for (int64_t T = T0; T < T1; ++T) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int e = threadIdx.x + 256 * k;
            if (e < kHalo) {
                float2 v;
                mx::d2ff(raw[k], v.x, v.y);
                (&sp[0][0])[e] = v;
            }
        }
        // this tile's instance data (loaded before the stores below, which cannot
        // alias them once in registers)
        const BInst& bi = tab[cur.inst];
        const int n1 = bi.n1, n2 = bi.n2, p1 = bi.p1;
        const float* cf1 = bi.coef1;
        const float* cf2 = bi.coef2;
        uint8_t* wbase = bi.wbase;
        const int64_t wpp = bi.w_part_pitch, woff = bi.w_off;
        const float g0 = bi.g.f0, g1 = bi.g.f1, g2 = bi.g.f2, g3 = bi.g.f3;
        const int a1 = cur.a1, a2 = cur.a2;
        if (T + 1 < T1) {                // the next tile's loads overlap this tile's stencil
            while (T + 1 >= next) next = __ldg(tile_begin + (++inst) + 1);
            cur = tile_at(tab, tile_begin, inst, T + 1);
            fetch(cur);
        }
        // coefficients along i_1 are fixed for this thread's column of the tile
        const int i1 = a1 + c;
        const bool in1 = i1 < n1;
        const float c1a = in1 ? __ldg(cf1 + i1) : 0.f, c1c = in1 ? __ldg(cf1 + n1 + i1) : 0.f,
                    c1s = in1 ? __ldg(cf1 + 2 * n1 + i1) : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kT / 8; ++q) {
            const int r = threadIdx.x / kT + 8 * q;
            const int i2 = a2 + r;
            if (!in1 || i2 >= n2) continue;
            const float uh = sp[r + 1][c + 1].x, ul = sp[r + 1][c + 1].y;
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
            PT* w = (PT*)wbase + woff + i1 + (int64_t)p1 * i2;
            w[0] = (PT)v[0];
            w[wpp] = (PT)v[1];
            if (F::kAParts == 3) w[2 * wpp] = (PT)v[2];
        }
        __syncthreads();
    }
}

// u += tau y (one DFMA per element), non-finite results flagged.
__global__ void __launch_bounds__(256) batch_update_kernel(const BInst* __restrict__ tab,
                                                           const int4* __restrict__ chunks, int64_t nchunks,
                                                           unsigned int* status) {
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        double* U = tab[ch.x].U;        // loaded once: the stores to U cannot alias them
        const float* y = tab[ch.x].y;
        const double tau = tab[ch.x].tau;
        bool bad = false;
        for (int e = threadIdx.x; e < ch.z; e += blockDim.x) {
            const int i = ch.y + e;
            const double v = fma(tau, mx::f2d(__ldg(y + i)), U[i]);
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
    int64_t* tile_begin = nullptr;          // prepass: first 32 x 32 tile of each instance
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

int build_tiles(mm_batch_s* b, cudaStream_t s) {
    for (auto& L : b->launches) {
        std::vector<int4> t1, t2;
        int rc = tc_group_tiles(b->prec, &b->spec1[L.c0], L.nc, &b->nc_cap[L.c0], t1);
        if (!rc) rc = tc_group_tiles(b->prec, &b->spec2[L.c0], L.nc, &b->nc_cap[L.c0], t2);
        if (rc) return rc;
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

int prepass(mm_batch_s* b, double t, cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(b->ntiles, (int64_t)num_sms() * 8);
    TraceScope tr(KC_PREPASS, s);
    (void)t;   // the batch's nonlinearities are autonomous
    if (b->prec == MM_BF16X3)
        batch_prepass_kernel<FormBF16><<<(unsigned)grid, 256, 0, s>>>(b->tab, b->tile_begin, b->count, b->ntiles);
    else
        batch_prepass_kernel<FormTF32><<<(unsigned)grid, 256, 0, s>>>(b->tab, b->tile_begin, b->count, b->ntiles);
    MM_LAUNCH_CHECK();
    return MM_OK;
}

int one_step(mm_batch_s* b, double t, cudaStream_t s) {
    int rc0 = prepass(b, t, s);
    if (rc0) return rc0;
    int rc = tucker_modes(b, s);
    if (rc) return rc;
    TraceScope tr(KC_SPLIT, s);
    batch_update_kernel<<<(unsigned)ew_grid(b), 256, 0, s>>>(b->tab, b->chunks, b->nchunks, b->status);
    MM_LAUNCH_CHECK();
    return MM_OK;
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
//   3. the per-class choices together, kept only if faster than the uniform one.
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
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->tune_ms_uniform = best_ms;
    b->tune_per_class = per_ms < best_ms;
    b->tune_ms_chosen = b->tune_per_class ? per_ms : best_ms;
    if (!b->tune_per_class)
        for (auto& v : b->nc_cap) v = best;
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
            e.wbase = C.W;
            e.w_part_pitch = m1.X.part_pitch;
            e.w_off = (int64_t)k * C.n2 * p1;
            e.y = C.y + (int64_t)k * nn;
            e.n1 = C.n1; e.n2 = C.n2; e.p1 = p1;
            e.tau = p->tau;
            e.g = pointwise_of(g ? &g[j] : nullptr);
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
        std::vector<int64_t> tb(count + 1, 0);
        for (int j = 0; j < count; ++j)
            tb[j + 1] = tb[j] + ((n1[j] + kT - 1) / kT) * ((n2[j] + kT - 1) / kT);
        b->ntiles = tb[count];
        if (!b->alloc((void**)&b->tile_begin, tb.size() * sizeof(int64_t)) ||
            cudaMemcpyAsync(b->tile_begin, tb.data(), tb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
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
        rc = prepass(b, 0.0, s);
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
    if (!b->use_graph) {
        for (int k = 0; k < nsteps; ++k) {
            int rc = one_step(b, t0, s);
            if (rc) return rc;
        }
        return MM_OK;
    }
    if (!b->exec || b->exec_steps != nsteps) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        MM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int rc = MM_OK;
        for (int k = 0; k < nsteps && !rc; ++k) rc = one_step(b, t0, b->cap);
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
    trace_count(KC_SPLIT, nsteps);
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
