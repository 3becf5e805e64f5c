// TF32x3 tensor-core path: placeholder until the tcgen05 kernels land.
#include "tf32.cuh"

namespace mm {

int plan_prepare_tf32(mm_plan_s*, cudaStream_t) { return MM_ERR_UNSUPPORTED; }

int tf32_mode_product(mm_plan_s*, int, int, const double*, const Epi&, cudaStream_t) {
    return MM_ERR_UNSUPPORTED;
}

}  // namespace mm
