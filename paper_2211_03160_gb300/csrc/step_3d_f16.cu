// D3Q19 + D3Q7 fused step, FP16 and BF16 offset storage (FP32 collision).
#include "dispatch.h"

namespace tlbm {
cudaError_t launch_step_3d_f16(int prec, int vec, bool trt, int rows, const void* src, void* dst, const KParams& p,
                        dim3 grid, dim3 block, cudaStream_t s) {
    if (prec == 2) {
        TLBM_STEP_CASE(3, __half, 4, true)
        TLBM_STEP96_CASE(3, __half, 2, true)
        TLBM_STEP_CASE(3, __half, 1, true)
        TLBM_STEP_CASE(3, __half, 4, false)
        TLBM_ROWS_CASE(3, __half, 1, 2)
        TLBM_ROWS_CASE(3, __half, 1, 4)
        TLBM_AA96_CASE(3, __half, 2, true)
        TLBM_AA_CASE(3, __half, 1, true)
        TLBM_AA_CASE(3, __half, 2, false)
    } else {
        TLBM_STEP_CASE(3, __nv_bfloat16, 4, true)
        TLBM_STEP96_CASE(3, __nv_bfloat16, 2, true)
        TLBM_STEP_CASE(3, __nv_bfloat16, 1, true)
        TLBM_STEP_CASE(3, __nv_bfloat16, 4, false)
        TLBM_ROWS_CASE(3, __nv_bfloat16, 1, 2)
        TLBM_ROWS_CASE(3, __nv_bfloat16, 1, 4)
        TLBM_AA96_CASE(3, __nv_bfloat16, 2, true)
        TLBM_AA_CASE(3, __nv_bfloat16, 1, true)
        TLBM_AA_CASE(3, __nv_bfloat16, 2, false)
    }
    return cudaErrorInvalidValue;
}

const void* func_step_3d_f16(int prec, int vec, bool trt, int rows) {
    if (prec == 2) {
        TLBM_STEP_FUNC(3, __half, 4, true)
        TLBM_STEP96_FUNC(3, __half, 2, true)
        TLBM_STEP_FUNC(3, __half, 1, true)
        TLBM_STEP_FUNC(3, __half, 4, false)
        TLBM_ROWS_FUNC(3, __half, 1, 2)
        TLBM_ROWS_FUNC(3, __half, 1, 4)
        TLBM_AA96_FUNC(3, __half, 2, true)
        TLBM_AA_FUNC(3, __half, 1, true)
        TLBM_AA_FUNC(3, __half, 2, false)
    } else {
        TLBM_STEP_FUNC(3, __nv_bfloat16, 4, true)
        TLBM_STEP96_FUNC(3, __nv_bfloat16, 2, true)
        TLBM_STEP_FUNC(3, __nv_bfloat16, 1, true)
        TLBM_STEP_FUNC(3, __nv_bfloat16, 4, false)
        TLBM_ROWS_FUNC(3, __nv_bfloat16, 1, 2)
        TLBM_ROWS_FUNC(3, __nv_bfloat16, 1, 4)
        TLBM_AA96_FUNC(3, __nv_bfloat16, 2, true)
        TLBM_AA_FUNC(3, __nv_bfloat16, 1, true)
        TLBM_AA_FUNC(3, __nv_bfloat16, 2, false)
    }
    return nullptr;
}
}  // namespace tlbm
