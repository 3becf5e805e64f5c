// Launch tracing: per kernel class, the number of launches and (when enabled)
// their device time from CUDA events recorded on the launching stream.
#pragma once

#include "common.cuh"

namespace mm {

enum KernelClass : int {
    KC_CONTRACT_FP64 = MM_KC_CONTRACT_FP64,
    KC_CONTRACT_TF32 = MM_KC_CONTRACT_TF32,
    KC_PREPASS = MM_KC_PREPASS,
    KC_SPLIT = MM_KC_SPLIT,
    KC_COUNT = MM_KC_COUNT,
};

// RAII: counts one launch of class `cls` and, if tracing is on, brackets it with a
// pair of events; launches into a stream under capture are neither counted nor
// timed (their graph's launches are counted with trace_count).
// Adds n launches of class cls that ran inside a CUDA graph (counted, not timed).
void trace_count(int cls, long long n);
// Launches recorded into a stream capture by this host thread between begin and end
// are tallied per class into counts[MM_KC_COUNT] (so each replay can be counted).
void trace_capture_begin();
void trace_capture_end(long long* counts);
// True while launches are being timed with events (graph replay would hide them).
bool trace_timing_on();

// RAII NVTX range around a library entry point (visible in Nsight timelines; costs
// nothing without a profiler attached).
class NvtxScope {
public:
    explicit NvtxScope(const char* name);
    ~NvtxScope();
};

class TraceScope {
public:
    TraceScope(int cls, cudaStream_t s);
    ~TraceScope();
private:
    int cls_;
    cudaStream_t s_;
    int slot_;
};

}  // namespace mm
