// Host-side state of a tlbm handle (private to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tlbm.h"
#include "kernels.cuh"

struct tlbm_s {
    int nx, ny, nz, dim, lattice, prec;
    int qf, qg;
    double Ra, Pr, Ma;
    tlbm_params prm;
    double U, H, nu, alpha, gbeta, a_T, omega;
    double S[tlbm::MAXQ], Q[7];
    tlbm::KParams kp;
    int vec, trt, bx, by;      // step kernel variant and block shape
    int rows;                  // consecutive rows per thread (software-pipelined when > 1)
    int aa;                    // 1: in-place (AA) streaming in one population buffer
    int nbuf;                  // population buffers: 2, or 1 in place
    int graph_steps;           // steps per CUDA graph replay in tlbm_step (0: plain launches)
    cudaGraphExec_t graph;     // captured block of graph_steps steps starting from buffer 0
    cudaStream_t capture_stream;
    int staged;                // 1: shared-memory staged (TMA bulk copy) kernel
    int variant_chosen;        // set by tlbm_set_variant / tlbm_set_staged: keep the caller's choice
    int staged_tw, staged_nc, staged_stages, staged_grid;
    unsigned long long wait_ns;  // staged kernel: give up on a copy after this long
    size_t staged_smem;
    size_t elem;               // bytes per stored value
    size_t popset_bytes;       // one population buffer (f planes then g planes)
    size_t red_off, res_off, stage_off, total_bytes;
    size_t status_off;         // device status word of the staged kernel
    char* mem;                 // bound device block
    size_t mem_bytes;
    void* buf[2];
    int cur;                   // buffer holding the current state (in place: 0 natural, 1 swapped order)
    int64_t t;
    cudaStream_t stream;
    int64_t launches;
    char err[256];
};
