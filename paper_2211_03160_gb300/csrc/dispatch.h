// Host-side launch entry points of the step kernels (one translation unit per
// lattice dimension, FP64 in its own unit built without FMA contraction).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace tlbm {

// prec: 0 FP64, 1 FP32, 2 FP16-offset, 3 BF16-offset (matches enum tlbm_prec)
// Returns the vector width (nodes per thread) the step kernel uses.
int step_vec(int dim, int prec);

cudaError_t launch_step_2d(int prec, const void* src, void* dst, const KParams& p, dim3 grid, dim3 block,
                           cudaStream_t s);
cudaError_t launch_step_3d(int prec, const void* src, void* dst, const KParams& p, dim3 grid, dim3 block,
                           cudaStream_t s);
cudaError_t launch_step_fp64(int dim, const void* src, void* dst, const KParams& p, dim3 grid, dim3 block,
                             cudaStream_t s);

}  // namespace tlbm
