// D2Q9 + D2Q5 fused step, FP32 and FP16/BF16-offset storage.
#include "dispatch.h"

namespace tlbm {

cudaError_t launch_step_2d(int prec, const void* src, void* dst, const KParams& p, dim3 grid, dim3 block,
                           cudaStream_t s) {
    switch (prec) {
    case 1:
        step_kernel<2, float, 4><<<grid, block, 0, s>>>((const float*)src, (float*)dst, p);
        break;
    case 2:
        step_kernel<2, __half, 8><<<grid, block, 0, s>>>((const __half*)src, (__half*)dst, p);
        break;
    case 3:
        step_kernel<2, __nv_bfloat16, 8>
            <<<grid, block, 0, s>>>((const __nv_bfloat16*)src, (__nv_bfloat16*)dst, p);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tlbm
