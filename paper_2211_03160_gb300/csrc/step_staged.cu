// Shared-memory staged (TMA bulk copy) variants of the fused step, TRT form.
#include "dispatch.h"
#include "staged.cuh"

namespace tlbm {

#define TLBM_STAGED_CASE(DIM, S, PREC)                                                              \
    if (dim == DIM && prec == PREC) {                                                              \
        fn = (const void*)&step_staged_kernel<DIM, S, true>;                                       \
        if (launch) step_staged_kernel<DIM, S, true><<<grid, STAGED_THREADS, smem, s>>>((const S*)src, (S*)dst, p, si); \
    }

static cudaError_t staged_dispatch(int dim, int prec, bool launch, const void*& fn, const void* src, void* dst,
                                   const KParams& p, const StagedInfo& si, int grid, size_t smem, cudaStream_t s) {
    fn = nullptr;
    TLBM_STAGED_CASE(2, float, 1)
    TLBM_STAGED_CASE(2, __half, 2)
    TLBM_STAGED_CASE(2, __nv_bfloat16, 3)
    TLBM_STAGED_CASE(3, float, 1)
    TLBM_STAGED_CASE(3, __half, 2)
    TLBM_STAGED_CASE(3, __nv_bfloat16, 3)
    if (!fn) return cudaErrorInvalidValue;
    return launch ? cudaGetLastError() : cudaSuccess;
}

const void* staged_function(int dim, int prec) {
    const void* fn = nullptr;
    KParams p{};
    StagedInfo si{};
    staged_dispatch(dim, prec, false, fn, nullptr, nullptr, p, si, 0, 0, nullptr);
    return fn;
}

cudaError_t launch_staged(int dim, int prec, const void* src, void* dst, const KParams& p, const StagedInfo& si,
                          int grid, size_t smem, cudaStream_t s) {
    const void* fn = nullptr;
    return staged_dispatch(dim, prec, true, fn, src, dst, p, si, grid, smem, s);
}

}  // namespace tlbm
