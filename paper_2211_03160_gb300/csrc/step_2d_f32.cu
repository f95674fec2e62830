// D2Q9 + D2Q5 fused step, FP32 storage.
#include "dispatch.h"

namespace tlbm {
cudaError_t launch_step_2d_f32(int vec, bool trt, int rows, const void* src, void* dst, const KParams& p, dim3 grid,
                        dim3 block, cudaStream_t s) {
    TLBM_STEP_CASE(2, float, 4, true)
    TLBM_STEP_CASE(2, float, 2, true)
    TLBM_STEP_CASE(2, float, 1, true)
    TLBM_STEP_CASE(2, float, 4, false)
    TLBM_ROWS_CASE(2, float, 4, 2)
    TLBM_ROWS_CASE(2, float, 4, 4)
    TLBM_AA_CASE(2, float, 4, true)
    TLBM_AA_CASE(2, float, 1, true)
    TLBM_AA_CASE(2, float, 4, false)
    return cudaErrorInvalidValue;
}

const void* func_step_2d_f32(int vec, bool trt, int rows) {
    TLBM_STEP_FUNC(2, float, 4, true)
    TLBM_STEP_FUNC(2, float, 2, true)
    TLBM_STEP_FUNC(2, float, 1, true)
    TLBM_STEP_FUNC(2, float, 4, false)
    TLBM_ROWS_FUNC(2, float, 4, 2)
    TLBM_ROWS_FUNC(2, float, 4, 4)
    TLBM_AA_FUNC(2, float, 4, true)
    TLBM_AA_FUNC(2, float, 1, true)
    TLBM_AA_FUNC(2, float, 4, false)
    return nullptr;
}
}  // namespace tlbm
