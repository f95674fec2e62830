// FP64 fused step (2D and 3D).  Built with --fmad=false so that its rounding
// follows the plain multiply-then-add order.  Also holds the variant table.
#include "dispatch.h"

namespace tlbm {

cudaError_t launch_step_f64(int dim, int vec, bool trt, int rows, const void* src, void* dst, const KParams& p, dim3 grid,
                            dim3 block, cudaStream_t s) {
    if (dim == 2) {
        TLBM_STEP_CASE(2, double, 2, true)
        TLBM_STEP_CASE(2, double, 1, true)
        TLBM_STEP_CASE(2, double, 2, false)
        TLBM_AA_CASE(2, double, 2, true)
        TLBM_AA_CASE(2, double, 2, false)
    } else {
        TLBM_STEP_CASE(3, double, 1, true)
        TLBM_STEP_CASE(3, double, 2, true)
        TLBM_STEP_CASE(3, double, 1, false)
        TLBM_AA_CASE(3, double, 1, true)
        TLBM_AA_CASE(3, double, 1, false)
    }
    return cudaErrorInvalidValue;
}

const void* func_step_f64(int dim, int vec, bool trt, int rows) {
    if (dim == 2) {
        TLBM_STEP_FUNC(2, double, 2, true)
        TLBM_STEP_FUNC(2, double, 1, true)
        TLBM_STEP_FUNC(2, double, 2, false)
        TLBM_AA_FUNC(2, double, 2, true)
        TLBM_AA_FUNC(2, double, 2, false)
    } else {
        TLBM_STEP_FUNC(3, double, 1, true)
        TLBM_STEP_FUNC(3, double, 2, true)
        TLBM_STEP_FUNC(3, double, 1, false)
        TLBM_AA_FUNC(3, double, 1, true)
        TLBM_AA_FUNC(3, double, 1, false)
    }
    return nullptr;
}

const void* step_function(int dim, int prec, int vec, bool trt, int rows) {
    if (prec == 0) return func_step_f64(dim, vec, trt, rows);
    if (dim == 2) return prec == 1 ? func_step_2d_f32(vec, trt, rows) : func_step_2d_f16(prec, vec, trt, rows);
    return prec == 1 ? func_step_3d_f32(vec, trt, rows) : func_step_3d_f16(prec, vec, trt, rows);
}

bool step_variant_available(int dim, int prec, int vec, bool trt, int rows) {
    return step_function(dim, prec, vec, trt, rows) != nullptr;
}

cudaError_t launch_step(int dim, int prec, int vec, bool trt, int rows, const void* src, void* dst,
                        const KParams& p, dim3 grid, dim3 block, cudaStream_t s) {
    if (!step_variant_available(dim, prec, vec, trt, rows)) return cudaErrorInvalidValue;
    if (prec == 0) return launch_step_f64(dim, vec, trt, rows, src, dst, p, grid, block, s);
    if (dim == 2) {
        if (prec == 1) return launch_step_2d_f32(vec, trt, rows, src, dst, p, grid, block, s);
        return launch_step_2d_f16(prec, vec, trt, rows, src, dst, p, grid, block, s);
    }
    if (prec == 1) return launch_step_3d_f32(vec, trt, rows, src, dst, p, grid, block, s);
    return launch_step_3d_f16(prec, vec, trt, rows, src, dst, p, grid, block, s);
}

}  // namespace tlbm
