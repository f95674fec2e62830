// Shared-memory staged (TMA bulk copy) variants of the fused step, TRT form,
// with 4 or 8 consumer warps in 2D (tiles of up to 256 or 512 nodes) and 4 or 7
// in 3D (256 or 448).
#include "dispatch.h"
#include "staged.cuh"

namespace tlbm {

#define TLBM_STAGED_CASE(DIM, S, PREC, NC)                                                           \
    if (dim == DIM && prec == PREC && nc == NC) {                                                   \
        fn = (const void*)&step_staged_kernel<DIM, S, NC>;                                          \
        if (launch)                                                                                 \
            step_staged_kernel<DIM, S, NC><<<grid, 32 * (NC + 1), smem, s>>>((const S*)src, (S*)dst, p, si); \
    }

static cudaError_t staged_dispatch(int dim, int prec, int nc, bool launch, const void*& fn, const void* src,
                                   void* dst, const KParams& p, const StagedInfo& si, int grid, size_t smem,
                                   cudaStream_t s) {
    fn = nullptr;
    TLBM_STAGED_CASE(2, float, 1, 4)
    TLBM_STAGED_CASE(2, float, 1, 8)
    TLBM_STAGED_CASE(2, __half, 2, 4)
    TLBM_STAGED_CASE(2, __half, 2, 8)
    TLBM_STAGED_CASE(2, __nv_bfloat16, 3, 4)
    TLBM_STAGED_CASE(2, __nv_bfloat16, 3, 8)
    TLBM_STAGED_CASE(3, float, 1, 4)
    TLBM_STAGED_CASE(3, float, 1, 7)
    TLBM_STAGED_CASE(3, __half, 2, 4)
    TLBM_STAGED_CASE(3, __half, 2, 7)
    TLBM_STAGED_CASE(3, __nv_bfloat16, 3, 4)
    TLBM_STAGED_CASE(3, __nv_bfloat16, 3, 7)
    if (!fn) return cudaErrorInvalidValue;
    return launch ? cudaGetLastError() : cudaSuccess;
}

const void* staged_function(int dim, int prec, int nc) {
    const void* fn = nullptr;
    KParams p{};
    StagedInfo si{};
    staged_dispatch(dim, prec, nc, false, fn, nullptr, nullptr, p, si, 0, 0, nullptr);
    return fn;
}

cudaError_t launch_staged(int dim, int prec, int nc, const void* src, void* dst, const KParams& p,
                          const StagedInfo& si, int grid, size_t smem, cudaStream_t s) {
    const void* fn = nullptr;
    return staged_dispatch(dim, prec, nc, true, fn, src, dst, p, si, grid, smem, s);
}

}  // namespace tlbm
