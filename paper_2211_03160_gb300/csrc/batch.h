// Device-side tables of a batched ensemble, shared by the flattened, persistent
// and staged batch kernels.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace tlbm {

struct BatchInst {
    const void* buf[2];  // population buffers of the instance
    long long block0;    // first flattened block of the instance
    int gx, gy;          // blocks along x and y of the instance (z: nz)
    long long stile0;    // first tile of the instance in the staged form
    int stw, stpr;       // staged form: tile length (elements of a plane's interior rows) and tiles per z-plane
};

// Staged form: the tiles of all instances, stage count and status word.
struct BatchStagedInfo {
    long long tiles;             // sum over instances of nz stpr
    int stages;                  // tiles in flight per CTA, 2 <= stages <= TILE_MAX_STAGES
    int* status;                 // set to 1 by a block that gave up waiting
    unsigned long long wait_ns;  // wait limit for a copy or a free stage
};

// The staged batch kernel for (dim, storage, consumer warps), or nullptr if not built.
const void* batch_staged_function(int dim, int prec, int nc);
cudaError_t launch_batch_staged(int dim, int prec, int nc, const KParams* kps, const BatchInst* inst, int n,
                                int parity, const BatchStagedInfo& si, int grid, size_t smem, cudaStream_t s);

}  // namespace tlbm
