// Launch tracing (see trace.cuh and mm_trace_* in include/phisplit.h).
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "trace.cuh"

namespace mm {

namespace {

struct Pair { cudaEvent_t a, b; int cls; };

std::mutex g_mu;
bool g_on = false;
long long g_launches[KC_COUNT] = {};
std::vector<Pair> g_pool;     // events, reused across windows
size_t g_used = 0;

}  // namespace

thread_local bool t_capturing = false;
thread_local long long t_cap[KC_COUNT] = {};

NvtxScope::NvtxScope(const char* name) { nvtxRangePushA(name); }
NvtxScope::~NvtxScope() { nvtxRangePop(); }

void trace_count(int cls, long long n) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches[cls] += n;
}

void trace_capture_begin() {
    t_capturing = true;
    for (int c = 0; c < KC_COUNT; ++c) t_cap[c] = 0;
}

void trace_capture_end(long long* counts) {
    t_capturing = false;
    for (int c = 0; c < KC_COUNT; ++c) counts[c] = t_cap[c];
}

bool trace_timing_on() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

TraceScope::TraceScope(int cls, cudaStream_t s) : cls_(cls), s_(s), slot_(-1) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        if (t_capturing) t_cap[cls]++;
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches[cls]++;
    if (!g_on) return;
    if (g_used == g_pool.size()) {
        Pair p{};
        if (cudaEventCreate(&p.a) != cudaSuccess) return;
        if (cudaEventCreate(&p.b) != cudaSuccess) { cudaEventDestroy(p.a); return; }
        g_pool.push_back(p);
    }
    slot_ = (int)g_used++;
    g_pool[slot_].cls = cls;
    cudaEventRecord(g_pool[slot_].a, s);
}

TraceScope::~TraceScope() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_pool[slot_].b, s_);
}

}  // namespace mm

using namespace mm;

extern "C" int mm_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    g_used = 0;
    for (int c = 0; c < KC_COUNT; ++c) g_launches[c] = 0;
    return MM_OK;
}

extern "C" int mm_trace_read(int cls, long long* launches, double* ms) {
    if (cls < 0 || cls >= KC_COUNT) return MM_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (launches) *launches = g_launches[cls];
    if (ms) {
        double total = 0.0;
        for (size_t i = 0; i < g_used; ++i) {
            if (g_pool[i].cls != cls) continue;
            if (cudaEventSynchronize(g_pool[i].b) != cudaSuccess) return MM_ERR_CUDA;
            float t = 0.f;
            if (cudaEventElapsedTime(&t, g_pool[i].a, g_pool[i].b) != cudaSuccess) return MM_ERR_CUDA;
            total += t;
        }
        *ms = total;
    }
    return MM_OK;
}
