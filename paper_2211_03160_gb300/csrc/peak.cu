// tlbm_fp64_fma_rate: the FP64 arithmetic roof of this device, measured.
//
// The FP64 storage path of the step is bound by the FP64 pipes of GB300 (far
// fewer per SM than the FP32 ones), not by HBM: its roofline is the rate of
// dependent-free FP64 fused multiply-adds the SMs sustain.  This file measures
// that rate with a plain kernel: every thread runs NCHAIN independent chains of
// x <- fma(x, a, b), enough warps per SM to hide the pipe latency, timed with
// CUDA events on the caller's stream.  Nothing is allocated: the chains' sum is
// kept in a static device word only if it takes an impossible value, which keeps
// the compiler from removing the chains.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "../../include/tlbm.h"

namespace {

constexpr int NCHAIN = 8;
constexpr int THREADS = 256;
__device__ double g_fp64_sink;

__global__ void __launch_bounds__(THREADS) fp64_fma_chains(int iters, double a, double b) {
    double x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    if (s == -1.0) g_fp64_sink = s;  // never true for these inputs
}

}  // namespace

extern "C" int tlbm_fp64_fma_rate(void* stream, double* flops_per_second) {
    if (!flops_per_second) return TLBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    const int blocks = sms * 8;  // 64 warps per SM
    const double a = 0.999999999, b = 1e-9;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return TLBM_ERR_CUDA;
    }
    int rc = TLBM_OK;
    double best = 0.0;
    int iters = 1 << 12;
    for (int rep = 0; rep < 6 && rc == TLBM_OK; ++rep) {
        fp64_fma_chains<<<blocks, THREADS, 0, s>>>(iters, a, b);  // warm-up / sizing
        cudaEventRecord(e0, s);
        fp64_fma_chains<<<blocks, THREADS, 0, s>>>(iters, a, b);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = TLBM_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * NCHAIN * (double)iters * blocks * THREADS;
        if (ms > 0.f) best = std::max(best, flops / (ms * 1e-3));
        // grow the launch towards ~20 ms so that launch overhead does not count
        if (ms < 20.f && iters < (1 << 24)) iters *= 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == TLBM_OK) *flops_per_second = best;
    return rc;
}
