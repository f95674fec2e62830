// FP64 fused step (2D and 3D).  Built with --fmad=false so that its rounding
// follows the plain multiply-then-add order.  Also holds the variant table.
#include "dispatch.h"

namespace tlbm {

cudaError_t launch_step_f64(int dim, int vec, bool trt, const void* src, void* dst, const KParams& p, dim3 grid,
                            dim3 block, cudaStream_t s) {
    if (dim == 2) {
        TLBM_STEP_CASE(2, double, 2, true)
        TLBM_STEP_CASE(2, double, 1, true)
        TLBM_STEP_CASE(2, double, 2, false)
    } else {
        TLBM_STEP_CASE(3, double, 1, true)
        TLBM_STEP_CASE(3, double, 2, true)
        TLBM_STEP_CASE(3, double, 1, false)
    }
    return cudaErrorInvalidValue;
}

const void* func_step_f64(int dim, int vec, bool trt) {
    if (dim == 2) {
        TLBM_STEP_FUNC(2, double, 2, true)
        TLBM_STEP_FUNC(2, double, 1, true)
        TLBM_STEP_FUNC(2, double, 2, false)
    } else {
        TLBM_STEP_FUNC(3, double, 1, true)
        TLBM_STEP_FUNC(3, double, 2, true)
        TLBM_STEP_FUNC(3, double, 1, false)
    }
    return nullptr;
}

const void* step_function(int dim, int prec, int vec, bool trt) {
    if (prec == 0) return func_step_f64(dim, vec, trt);
    if (dim == 2) return prec == 1 ? func_step_2d_f32(vec, trt) : func_step_2d_f16(prec, vec, trt);
    return prec == 1 ? func_step_3d_f32(vec, trt) : func_step_3d_f16(prec, vec, trt);
}

bool step_variant_available(int dim, int prec, int vec, bool trt) {
    static const int table[][4] = {
        // dim, prec, vec, trt
        {2, 1, 4, 1}, {2, 1, 2, 1}, {2, 1, 1, 1}, {2, 1, 4, 0},
        {2, 2, 8, 1}, {2, 2, 4, 1}, {2, 2, 2, 1}, {2, 2, 8, 0},
        {2, 3, 8, 1}, {2, 3, 4, 1}, {2, 3, 2, 1}, {2, 3, 8, 0},
        {3, 1, 4, 1}, {3, 1, 2, 1}, {3, 1, 1, 1}, {3, 1, 2, 0},
        {3, 2, 4, 1}, {3, 2, 2, 1}, {3, 2, 1, 1}, {3, 2, 4, 0},
        {3, 3, 4, 1}, {3, 3, 2, 1}, {3, 3, 1, 1}, {3, 3, 4, 0},
        {2, 0, 2, 1}, {2, 0, 1, 1}, {2, 0, 2, 0},
        {3, 0, 1, 1}, {3, 0, 2, 1}, {3, 0, 1, 0},
    };
    for (const auto& r : table)
        if (r[0] == dim && r[1] == prec && r[2] == vec && r[3] == (trt ? 1 : 0)) return true;
    return false;
}

cudaError_t launch_step(int dim, int prec, int vec, bool trt, const void* src, void* dst, const KParams& p,
                        dim3 grid, dim3 block, cudaStream_t s) {
    if (!step_variant_available(dim, prec, vec, trt)) return cudaErrorInvalidValue;
    if (prec == 0) return launch_step_f64(dim, vec, trt, src, dst, p, grid, block, s);
    if (dim == 2) {
        if (prec == 1) return launch_step_2d_f32(vec, trt, src, dst, p, grid, block, s);
        return launch_step_2d_f16(prec, vec, trt, src, dst, p, grid, block, s);
    }
    if (prec == 1) return launch_step_3d_f32(vec, trt, src, dst, p, grid, block, s);
    return launch_step_3d_f16(prec, vec, trt, src, dst, p, grid, block, s);
}

}  // namespace tlbm
