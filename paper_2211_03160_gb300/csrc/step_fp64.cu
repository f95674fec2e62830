// FP64 fused step (2D and 3D).  Built with --fmad=false so that its rounding
// follows the plain multiply-then-add order.
#include "dispatch.h"

namespace tlbm {

int step_vec(int dim, int prec) {
    if (dim == 2) return prec == 0 ? 2 : (prec == 1 ? 4 : 8);
    return prec == 0 ? 1 : (prec == 1 ? 2 : 4);
}

cudaError_t launch_step_fp64(int dim, const void* src, void* dst, const KParams& p, dim3 grid, dim3 block,
                             cudaStream_t s) {
    if (dim == 2)
        step_kernel<2, double, 2><<<grid, block, 0, s>>>((const double*)src, (double*)dst, p);
    else
        step_kernel<3, double, 1><<<grid, block, 0, s>>>((const double*)src, (double*)dst, p);
    return cudaGetLastError();
}

}  // namespace tlbm
