// Host-side launch entry points of the step kernels.  Each translation unit
// instantiates the variants of one (dimension, storage) family; the FP64 unit
// is built without FMA contraction.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "staged.cuh"

namespace tlbm {

// prec: 0 FP64, 1 FP32, 2 FP16-offset, 3 BF16-offset (enum tlbm_prec).
// vec: nodes per thread.  trt: two-relaxation-time form of the collision.
// Returns cudaErrorInvalidValue if the variant is not compiled.
// rows: consecutive rows per thread (1, or 2 / 4 for the software-pipelined kernel);
// -AA_EVEN / -AA_ODD select the two halves of an in-place step pair, which read
// and write `dst` only.
cudaError_t launch_step(int dim, int prec, int vec, bool trt, int rows, const void* src, void* dst,
                        const KParams& p, dim3 grid, dim3 block, cudaStream_t s);
bool step_variant_available(int dim, int prec, int vec, bool trt, int rows);
// device function of a compiled variant (for cudaFuncGetAttributes), or nullptr
const void* step_function(int dim, int prec, int vec, bool trt, int rows);

// shared-memory staged (TMA bulk copy) step, TRT form, FP32/FP16/BF16 storage,
// nc = 4 or 8 consumer warps
const void* staged_function(int dim, int prec, int nc);
cudaError_t launch_staged(int dim, int prec, int nc, const void* src, void* dst, const KParams& p,
                          const StagedInfo& si, int grid, size_t smem, cudaStream_t s);

// per-unit entry points
cudaError_t launch_step_2d_f32(int vec, bool trt, int rows, const void*, void*, const KParams&, dim3, dim3,
                               cudaStream_t);
cudaError_t launch_step_2d_f16(int prec, int vec, bool trt, int rows, const void*, void*, const KParams&, dim3, dim3,
                               cudaStream_t);
cudaError_t launch_step_3d_f32(int vec, bool trt, int rows, const void*, void*, const KParams&, dim3, dim3,
                               cudaStream_t);
cudaError_t launch_step_3d_f16(int prec, int vec, bool trt, int rows, const void*, void*, const KParams&, dim3, dim3,
                               cudaStream_t);
cudaError_t launch_step_f64(int dim, int vec, bool trt, int rows, const void*, void*, const KParams&, dim3, dim3,
                            cudaStream_t);
const void* func_step_2d_f32(int vec, bool trt, int rows);
const void* func_step_2d_f16(int prec, int vec, bool trt, int rows);
const void* func_step_3d_f32(int vec, bool trt, int rows);
const void* func_step_3d_f16(int prec, int vec, bool trt, int rows);
const void* func_step_f64(int dim, int vec, bool trt, int rows);

}  // namespace tlbm

// Instantiate-and-launch helper: one case of a (vec, trt) switch.
#define TLBM_STEP_CASE(DIM, S, VEC, TRT)                                                            \
    if (vec == VEC && trt == TRT && rows == 1) {                                                    \
        tlbm::step_kernel<DIM, S, VEC, TRT><<<grid, block, 0, s>>>((const S*)src, (S*)dst, p);      \
        return cudaGetLastError();                                                                  \
    }

#define TLBM_STEP_FUNC(DIM, S, VEC, TRT) \
    if (vec == VEC && trt == TRT && rows == 1) return (const void*)&tlbm::step_kernel<DIM, S, VEC, TRT>;

// software-pipelined multi-row variants (two-relaxation-time form)
#define TLBM_ROWS_CASE(DIM, S, VEC, ROWS)                                                             \
    if (vec == VEC && trt && rows == ROWS) {                                                        \
        tlbm::step_kernel_rows<DIM, S, VEC, true, ROWS><<<grid, block, 0, s>>>((const S*)src, (S*)dst, p); \
        return cudaGetLastError();                                                                  \
    }
#define TLBM_ROWS_FUNC(DIM, S, VEC, ROWS) \
    if (vec == VEC && trt && rows == ROWS) return (const void*)&tlbm::step_kernel_rows<DIM, S, VEC, true, ROWS>;

// variants held to 96 registers (step_kernel_r96, step_kernel_aa_r96)
#define TLBM_STEP96_CASE(DIM, S, VEC, TRT)                                                          \
    if (vec == VEC && trt == TRT && rows == 1) {                                                    \
        tlbm::step_kernel_r96<DIM, S, VEC, TRT><<<grid, block, 0, s>>>((const S*)src, (S*)dst, p);  \
        return cudaGetLastError();                                                                  \
    }
#define TLBM_STEP96_FUNC(DIM, S, VEC, TRT) \
    if (vec == VEC && trt == TRT && rows == 1) return (const void*)&tlbm::step_kernel_r96<DIM, S, VEC, TRT>;
#define TLBM_AA96_CASE(DIM, S, VEC, TRT)                                                                     \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_EVEN) {                                               \
        tlbm::step_kernel_aa_r96<DIM, S, VEC, TRT, tlbm::AA_EVEN><<<grid, block, 0, s>>>((S*)dst, p);       \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_ODD) {                                                \
        tlbm::step_kernel_aa_r96<DIM, S, VEC, TRT, tlbm::AA_ODD><<<grid, block, 0, s>>>((S*)dst, p);        \
        return cudaGetLastError();                                                                          \
    }
#define TLBM_AA96_FUNC(DIM, S, VEC, TRT)                                                                     \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_EVEN)                                                 \
        return (const void*)&tlbm::step_kernel_aa_r96<DIM, S, VEC, TRT, tlbm::AA_EVEN>;                     \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_ODD)                                                  \
        return (const void*)&tlbm::step_kernel_aa_r96<DIM, S, VEC, TRT, tlbm::AA_ODD>;

// in-place (AA) halves
#define TLBM_AA_CASE(DIM, S, VEC, TRT)                                                                       \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_EVEN) {                                               \
        tlbm::step_kernel_aa<DIM, S, VEC, TRT, tlbm::AA_EVEN><<<grid, block, 0, s>>>((S*)dst, p);           \
        return cudaGetLastError();                                                                          \
    }                                                                                                       \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_ODD) {                                                \
        tlbm::step_kernel_aa<DIM, S, VEC, TRT, tlbm::AA_ODD><<<grid, block, 0, s>>>((S*)dst, p);            \
        return cudaGetLastError();                                                                          \
    }
#define TLBM_AA_FUNC(DIM, S, VEC, TRT)                                                                       \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_EVEN)                                                 \
        return (const void*)&tlbm::step_kernel_aa<DIM, S, VEC, TRT, tlbm::AA_EVEN>;                         \
    if (vec == VEC && trt == TRT && rows == -tlbm::AA_ODD)                                                  \
        return (const void*)&tlbm::step_kernel_aa<DIM, S, VEC, TRT, tlbm::AA_ODD>;
