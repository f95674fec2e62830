// D2Q9 + D2Q5 fused step, FP16 and BF16 offset storage (FP32 collision).
#include "dispatch.h"

namespace tlbm {
cudaError_t launch_step_2d_f16(int prec, int vec, bool trt, int rows, const void* src, void* dst, const KParams& p,
                        dim3 grid, dim3 block, cudaStream_t s) {
    if (prec == 2) {
        TLBM_STEP_CASE(2, __half, 8, true)
        TLBM_STEP_CASE(2, __half, 4, true)
        TLBM_STEP_CASE(2, __half, 2, true)
        TLBM_STEP_CASE(2, __half, 8, false)
        TLBM_ROWS_CASE(2, __half, 4, 2)
        TLBM_ROWS_CASE(2, __half, 4, 4)
        TLBM_ROWS_CASE(2, __half, 8, 2)
        TLBM_ROWS_CASE(2, __half, 8, 4)
        TLBM_AA_CASE(2, __half, 4, true)
        TLBM_AA_CASE(2, __half, 1, true)
        TLBM_AA_CASE(2, __half, 4, false)
    } else {
        TLBM_STEP_CASE(2, __nv_bfloat16, 8, true)
        TLBM_STEP_CASE(2, __nv_bfloat16, 4, true)
        TLBM_STEP_CASE(2, __nv_bfloat16, 2, true)
        TLBM_STEP_CASE(2, __nv_bfloat16, 8, false)
        TLBM_ROWS_CASE(2, __nv_bfloat16, 4, 2)
        TLBM_ROWS_CASE(2, __nv_bfloat16, 4, 4)
        TLBM_ROWS_CASE(2, __nv_bfloat16, 8, 2)
        TLBM_ROWS_CASE(2, __nv_bfloat16, 8, 4)
        TLBM_AA_CASE(2, __nv_bfloat16, 4, true)
        TLBM_AA_CASE(2, __nv_bfloat16, 1, true)
        TLBM_AA_CASE(2, __nv_bfloat16, 4, false)
    }
    return cudaErrorInvalidValue;
}

const void* func_step_2d_f16(int prec, int vec, bool trt, int rows) {
    if (prec == 2) {
        TLBM_STEP_FUNC(2, __half, 8, true)
        TLBM_STEP_FUNC(2, __half, 4, true)
        TLBM_STEP_FUNC(2, __half, 2, true)
        TLBM_STEP_FUNC(2, __half, 8, false)
        TLBM_ROWS_FUNC(2, __half, 4, 2)
        TLBM_ROWS_FUNC(2, __half, 4, 4)
        TLBM_ROWS_FUNC(2, __half, 8, 2)
        TLBM_ROWS_FUNC(2, __half, 8, 4)
        TLBM_AA_FUNC(2, __half, 4, true)
        TLBM_AA_FUNC(2, __half, 1, true)
        TLBM_AA_FUNC(2, __half, 4, false)
    } else {
        TLBM_STEP_FUNC(2, __nv_bfloat16, 8, true)
        TLBM_STEP_FUNC(2, __nv_bfloat16, 4, true)
        TLBM_STEP_FUNC(2, __nv_bfloat16, 2, true)
        TLBM_STEP_FUNC(2, __nv_bfloat16, 8, false)
        TLBM_ROWS_FUNC(2, __nv_bfloat16, 4, 2)
        TLBM_ROWS_FUNC(2, __nv_bfloat16, 4, 4)
        TLBM_ROWS_FUNC(2, __nv_bfloat16, 8, 2)
        TLBM_ROWS_FUNC(2, __nv_bfloat16, 8, 4)
        TLBM_AA_FUNC(2, __nv_bfloat16, 4, true)
        TLBM_AA_FUNC(2, __nv_bfloat16, 1, true)
        TLBM_AA_FUNC(2, __nv_bfloat16, 4, false)
    }
    return nullptr;
}
}  // namespace tlbm
