// D3Q19 + D3Q7 fused step, FP32 storage.
#include "dispatch.h"

namespace tlbm {
cudaError_t launch_step_3d_f32(int vec, bool trt, int rows, const void* src, void* dst, const KParams& p, dim3 grid,
                        dim3 block, cudaStream_t s) {
    TLBM_STEP_CASE(3, float, 4, true)
    TLBM_STEP_CASE(3, float, 2, true)
    TLBM_STEP_CASE(3, float, 1, true)
    TLBM_STEP_CASE(3, float, 2, false)
    TLBM_ROWS_CASE(3, float, 1, 2)
    TLBM_ROWS_CASE(3, float, 1, 4)
    TLBM_AA_CASE(3, float, 1, true)
    TLBM_AA_CASE(3, float, 2, true)
    TLBM_AA_CASE(3, float, 1, false)
    return cudaErrorInvalidValue;
}

const void* func_step_3d_f32(int vec, bool trt, int rows) {
    TLBM_STEP_FUNC(3, float, 4, true)
    TLBM_STEP_FUNC(3, float, 2, true)
    TLBM_STEP_FUNC(3, float, 1, true)
    TLBM_STEP_FUNC(3, float, 2, false)
    TLBM_ROWS_FUNC(3, float, 1, 2)
    TLBM_ROWS_FUNC(3, float, 1, 4)
    TLBM_AA_FUNC(3, float, 1, true)
    TLBM_AA_FUNC(3, float, 2, true)
    TLBM_AA_FUNC(3, float, 1, false)
    return nullptr;
}
}  // namespace tlbm
