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

// RAII: counts one launch of class `cls` and, if tracing is on and the stream is
// not being captured, brackets it with a pair of events.
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
