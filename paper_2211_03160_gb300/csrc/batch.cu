// Batched ensemble of independent cells (same lattice and storage, own sizes,
// Rayleigh and Prandtl numbers and seeds): one flattened launch steps every
// instance, captured into a CUDA graph of `graph_steps` steps so that a block
// of steps costs one graph launch.  Each instance is an ordinary handle bound to
// its own slice of the batch's device block, so every single-cell call
// (macros, populations, reductions) works on it unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tlbm.h"
#include "batch.h"
#include "dispatch.h"
#include "handle.h"

using namespace tlbm;

namespace {

// Tile b of the flattened grid belongs to the instance i with
// block0[i] <= b < block0[i+1]; its parameters are staged in shared memory.
// Called by all threads of a block together.  CG: the loads bypass L1 (the
// persistent kernel reads what other blocks wrote in the previous step).  ROWS
// > 1: the software-pipelined body (ROWS rows per thread; flattened form only).
// batch_stage: find the instance of tile b and stage its parameters in sp, si.
__device__ __forceinline__ void batch_stage(const KParams* __restrict__ kps, const BatchInst* __restrict__ inst, int n,
                                            long long b, KParams& sp, int& si) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    if (n <= 128) {
        // warp 0: the instances with block0 <= b, counted by ballot (block0 rises
        // with the instance index), all lanes' loads in flight at once
        if (tid < 32) {
            int count = 0;
#pragma unroll
            for (int base = 0; base < 128; base += 32) {
                const int k = base + tid;
                const bool le = k < n && inst[k].block0 <= b;
                count += __popc(__ballot_sync(0xffffffffu, le));
            }
            if (tid == 0) si = count - 1;
        }
    } else if (tid == 0) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (inst[mid].block0 <= b) lo = mid;
            else hi = mid - 1;
        }
        si = lo;
    }
    __syncthreads();
    const int i = si;
    {
        static_assert(sizeof(KParams) % sizeof(long long) == 0, "KParams copied in 8-byte words");
        const long long* src = reinterpret_cast<const long long*>(kps + i);
        long long* dst = reinterpret_cast<long long*>(&sp);
        for (int w = tid; w < (int)(sizeof(KParams) / sizeof(long long)); w += nt) dst[w] = src[w];
    }
    __syncthreads();
}

// batch_run: step tile b of the staged instance si.
template <int DIM, class S, int VEC, bool TRT, bool CG = false, int ROWS = 1>
__device__ __forceinline__ void batch_run(const BatchInst* __restrict__ inst, int parity, long long b,
                                          const KParams& sp, int si) {
    const BatchInst in = inst[si];
    const long long local = b - in.block0;
    const int bx = (int)(local % in.gx);
    const long long r = local / in.gx;
    const int by = (int)(r % in.gy);
    const int bz = (int)(r / in.gy);
    if constexpr (ROWS > 1) {
        static_assert(!CG, "the pipelined body reads through L1");
        step_rows_block<DIM, S, VEC, TRT, ROWS>((const S*)in.buf[parity], (S*)in.buf[parity ^ 1], sp, bx, by, bz);
    } else {
        step_block<DIM, S, VEC, TRT, CG>((const S*)in.buf[parity], (S*)in.buf[parity ^ 1], sp, bx, by, bz);
    }
}

template <int DIM, class S, int VEC, bool TRT, bool CG = false, int ROWS = 1>
__device__ __forceinline__ void batch_tile(const KParams* __restrict__ kps, const BatchInst* __restrict__ inst, int n,
                                           int parity, long long b, KParams& sp, int& si) {
    batch_stage(kps, inst, n, b, sp, si);
    batch_run<DIM, S, VEC, TRT, CG, ROWS>(inst, parity, b, sp, si);
}

// Flattened form: block k steps the tiles [k tpb, (k + 1) tpb) in order.  The
// tiles of an instance are consecutive, so a block stages an instance's
// parameters only when its run of tiles enters that instance (one tile per
// block staged them for every tile, a lookup and a 1.2 KB copy in front of
// every 1024 nodes).
template <int DIM, class S, int VEC, bool TRT, int ROWS = 1>
__global__ void batch_step_kernel(const KParams* __restrict__ kps, const BatchInst* __restrict__ inst, int n,
                                  int parity, long long tiles, int tpb) {
    __shared__ KParams sp;
    __shared__ int si;
    const long long b0 = (long long)blockIdx.x * tpb;
    const long long b1 = b0 + tpb < tiles ? b0 + tpb : tiles;
    long long next = -1;  // first tile past the staged instance
    for (long long b = b0; b < b1; ++b) {
        if (b >= next) {
            if (next >= 0) __syncthreads();  // every thread is done with sp
            batch_stage(kps, inst, n, b, sp, si);
            next = si + 1 < n ? inst[si + 1].block0 : tiles;
        }
        batch_run<DIM, S, VEC, TRT, false, ROWS>(inst, parity, b, sp, si);
    }
}

// ------------------------------------------------------------------ persistent form

// Grid barrier of the persistent kernel: arrivals are counted, the last block
// of a round opens the next generation.  Waits are bounded in time.
struct GridSync {
    unsigned count;
    unsigned gen;
    int status;         // 1: a block gave up waiting (TLBM_ERR_TIMEOUT)
    int staged_status;  // 1: a block of the staged form gave up waiting for its copies
};
constexpr unsigned long long GRID_WAIT_NS = 500000000;  // default: 0.5 s

__device__ __forceinline__ unsigned long long batch_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks of the (co-resident, cooperatively launched) grid meet; returns
// false in every block that gave up (after wait_ns; 0: at once unless the
// barrier is already open) or found that another block gave up.
__device__ __forceinline__ bool grid_sync(GridSync* gs, int& ok, unsigned long long wait_ns) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* vgen = &gs->gen;
        volatile int* vstat = &gs->status;
        const unsigned g = *vgen;
        __threadfence();  // this block's stores before its arrival
        const unsigned prev = atomicAdd(&gs->count, 1u);
        int good = 1;
        if (prev == gridDim.x - 1) {
            gs->count = 0;
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            const unsigned long long t0 = batch_ns();
            while (*vgen == g) {
                if (*vstat || batch_ns() - t0 > wait_ns || wait_ns == 0) {
                    atomicExch(&gs->status, 1);
                    good = 0;
                    break;
                }
            }
        }
        __threadfence();  // the other blocks' stores before this block reads them
        ok = good && !*vstat;
    }
    __syncthreads();
    return ok != 0;
}

// `steps` steps in one launch: the blocks work through the tiles of all
// instances in a fixed order (block k takes tiles k, k + G, k + 2G, ...) and meet
// at a grid barrier between steps.
template <int DIM, class S, int VEC, bool TRT>
__global__ void batch_persistent_kernel(const KParams* __restrict__ kps, const BatchInst* __restrict__ inst, int n,
                                        long long tiles, int parity0, int steps, GridSync* gs,
                                        unsigned long long wait_ns) {
    __shared__ KParams sp;
    __shared__ int si;
    __shared__ int ok;
    for (int st = 0; st < steps; ++st) {
        const int parity = (parity0 + st) & 1;
        for (long long b = blockIdx.x; b < tiles; b += gridDim.x) {
            batch_tile<DIM, S, VEC, TRT, true>(kps, inst, n, parity, b, sp, si);
            __syncthreads();  // sp and si are reused by the next tile
        }
        if (st + 1 < steps && !grid_sync(gs, ok, wait_ns)) return;
    }
}

// Persistent launch parameters (steps > 0 selects the persistent kernel: grid
// = the co-resident block count, cooperative launch).
struct Persist {
    int steps;
    GridSync* gs;
    unsigned long long wait_ns;
    long long tiles;
    int* per_sm_out;  // when not launching: co-resident blocks per SM of the variant
};

#define TLBM_BATCH_CASE(DIM, S, PREC, VEC, TRT)                                                      \
    if (dim == DIM && prec == PREC && vec == VEC && trt == TRT && rows == 1) {                      \
        if (pp && pp->per_sm_out)                                                                   \
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                   \
                pp->per_sm_out, batch_persistent_kernel<DIM, S, VEC, TRT>, block.x * block.y, 0);    \
        if (launch && pp && pp->steps > 0) {                                                        \
            const KParams* a0 = kps;                                                                \
            const BatchInst* a1 = inst;                                                             \
            int a2 = n;                                                                             \
            long long a3 = pp->tiles;                                                               \
            int a4 = parity, a5 = pp->steps;                                                        \
            GridSync* a6 = pp->gs;                                                                  \
            unsigned long long a7 = pp->wait_ns;                                                    \
            void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7};                                \
            return cudaLaunchCooperativeKernel((const void*)batch_persistent_kernel<DIM, S, VEC, TRT>, \
                                               dim3((unsigned)grid), block, args, 0, s);            \
        }                                                                                           \
        if (launch)                                                                                 \
            batch_step_kernel<DIM, S, VEC, TRT>                                                     \
                <<<(grid + tpb - 1) / tpb, block, 0, s>>>(kps, inst, n, parity, grid, tpb);         \
        return launch ? cudaGetLastError() : cudaSuccess;                                           \
    }

// pipelined rows (flattened form, two-relaxation-time collision)
#define TLBM_BATCH_ROWS_CASE(DIM, S, PREC, VEC, ROWS)                                                  \
    if (dim == DIM && prec == PREC && vec == VEC && trt && rows == ROWS) {                           \
        if (pp) return cudaErrorInvalidValue;                                                         \
        if (launch)                                                                                   \
            batch_step_kernel<DIM, S, VEC, true, ROWS>                                                \
                <<<(grid + tpb - 1) / tpb, block, 0, s>>>(kps, inst, n, parity, grid, tpb);           \
        return launch ? cudaGetLastError() : cudaSuccess;                                             \
    }

cudaError_t batch_dispatch(bool launch, int dim, int prec, int vec, bool trt, const KParams* kps,
                           const BatchInst* inst, int n, int parity, long long grid, dim3 block, cudaStream_t s,
                           const Persist* pp = nullptr, int rows = 1, int tpb = 1) {
    TLBM_BATCH_ROWS_CASE(2, float, 1, 4, 2)
    TLBM_BATCH_ROWS_CASE(2, __half, 2, 4, 2)
    TLBM_BATCH_ROWS_CASE(2, __half, 2, 8, 2)
    TLBM_BATCH_ROWS_CASE(2, __nv_bfloat16, 3, 4, 2)
    TLBM_BATCH_ROWS_CASE(2, __nv_bfloat16, 3, 8, 2)
    TLBM_BATCH_ROWS_CASE(3, float, 1, 1, 2)
    TLBM_BATCH_ROWS_CASE(3, __half, 2, 1, 2)
    TLBM_BATCH_ROWS_CASE(3, __nv_bfloat16, 3, 1, 2)
    TLBM_BATCH_CASE(2, float, 1, 4, true)
    TLBM_BATCH_CASE(2, float, 1, 2, true)
    TLBM_BATCH_CASE(2, float, 1, 4, false)
    TLBM_BATCH_CASE(2, __half, 2, 2, true)
    TLBM_BATCH_CASE(2, __nv_bfloat16, 3, 2, true)
    TLBM_BATCH_ROWS_CASE(2, __half, 2, 2, 2)
    TLBM_BATCH_ROWS_CASE(2, __nv_bfloat16, 3, 2, 2)
    TLBM_BATCH_CASE(2, __half, 2, 4, true)
    TLBM_BATCH_CASE(2, __half, 2, 8, true)
    TLBM_BATCH_CASE(2, __half, 2, 8, false)
    TLBM_BATCH_CASE(2, __nv_bfloat16, 3, 4, true)
    TLBM_BATCH_CASE(2, __nv_bfloat16, 3, 8, true)
    TLBM_BATCH_CASE(2, __nv_bfloat16, 3, 8, false)
    TLBM_BATCH_CASE(2, double, 0, 2, true)
    TLBM_BATCH_CASE(2, double, 0, 2, false)
    TLBM_BATCH_CASE(3, float, 1, 2, true)
    TLBM_BATCH_CASE(3, float, 1, 1, true)
    TLBM_BATCH_CASE(3, float, 1, 2, false)
    TLBM_BATCH_CASE(3, __half, 2, 1, true)
    TLBM_BATCH_CASE(3, __half, 2, 4, false)
    TLBM_BATCH_CASE(3, __nv_bfloat16, 3, 1, true)
    TLBM_BATCH_CASE(3, __nv_bfloat16, 3, 4, false)
    TLBM_BATCH_CASE(3, double, 0, 1, true)
    TLBM_BATCH_CASE(3, double, 0, 1, false)
    return cudaErrorInvalidValue;
}

thread_local char g_batch_create_error[256] = "";

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct tlbm_batch_s {
    int n, dim, lattice, prec;
    std::vector<tlbm_t> inst;
    std::vector<size_t> off;      // byte offset of each instance's slice
    std::vector<uint64_t> seeds;  // per-instance initial-state seeds
    size_t tables_off, total_bytes;
    char* mem;
    size_t mem_bytes;
    KParams* d_kp;
    BatchInst* d_inst;
    GridSync* d_sync;
    int vec, trt, bx, by;
    int rows;           // rows per thread of the flattened launch (1 or 2)
    int tpb;            // tiles per block of the flattened launch
    int graph_steps;
    int persist_steps;  // > 0: persistent kernel, this many steps per launch
    int staged_nc;      // > 0: shared-memory staged form with this many consumer warps
    int staged_stages;
    long long staged_cap;  // co-resident blocks of the staged kernel (blocks per SM x SMs)
    size_t staged_smem;
    long long staged_tiles;
    unsigned long long wait_ns;  // grid-barrier wait limit of the persistent kernel
    long long total_blocks;
    int parity;
    int64_t t;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    cudaGraphExec_t graph;
    int64_t launches;
    char err[256];
};

static int bfail(tlbm_batch_t b, int code, const char* fmt, ...) {
    char* dst = b ? b->err : g_batch_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

static void drop_graph(tlbm_batch_t b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// default variant: the tuned single-cell one (see api.cu), restricted to the
// batch's compiled set
static void batch_default_variant(tlbm_batch_t b) {
    int v = 0, form = 0, bx = 0, by = 0;
    tlbm_get_variant(b->inst[0], &v, &form, &bx, &by, nullptr);
    b->vec = v;
    b->trt = 1;
    for (tlbm_t h : b->inst) b->trt = b->trt && h->kp.trt;
    b->bx = bx;
    b->by = by;
    if (batch_dispatch(false, b->dim, b->prec, b->vec, b->trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr) !=
        cudaSuccess) {
        // fall back to the batch's first compiled vector width for this storage
        const int cand[] = {4, 8, 2, 1};
        for (int c : cand)
            if (batch_dispatch(false, b->dim, b->prec, c, b->trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr) ==
                cudaSuccess) {
                b->vec = c;
                break;
            }
    }
}

// rows per thread of the tables and launches: the persistent form runs one
static int eff_rows(tlbm_batch_t b) { return b->persist_steps > 0 ? 1 : b->rows; }

// per-instance tables for the flattened launch (host side)
static void build_tables(tlbm_batch_t b, std::vector<KParams>& kps, std::vector<BatchInst>& ins) {
    kps.resize(b->n);
    ins.resize(b->n);
    long long block0 = 0, stile0 = 0;
    for (int i = 0; i < b->n; ++i) {
        tlbm_t h = b->inst[i];
        kps[i] = h->kp;
        kps[i].xmax_load = h->kp.L.P - b->vec;
        const int tx = (h->nx + b->vec - 1) / b->vec;
        const int gx = (tx + b->bx - 1) / b->bx;
        const int rows = eff_rows(b);
        const int gy = (h->ny + b->by * rows - 1) / (b->by * rows);
        ins[i].buf[0] = h->buf[0];
        ins[i].buf[1] = h->buf[1];
        ins[i].block0 = block0;
        ins[i].gx = gx;
        ins[i].gy = gy;
        block0 += (long long)gx * gy * h->nz;
        // staged form: stretches of 64 NC elements of each z-plane's interior
        // rows (ny P elements, contiguous; a multiple of the 16-byte copy granule)
        ins[i].stile0 = stile0;
        ins[i].stw = ins[i].stpr = 0;
        if (b->staged_nc > 0) {
            const long long run = (long long)h->ny * h->kp.L.P;
            const int tw = (int)std::min<long long>(64 * b->staged_nc, run);
            ins[i].stw = tw;
            ins[i].stpr = (int)((run + tw - 1) / tw);
            stile0 += (long long)h->nz * ins[i].stpr;
        }
    }
    b->total_blocks = block0;
    b->staged_tiles = stile0;
}

static int upload_tables(tlbm_batch_t b) {
    std::vector<KParams> kps;
    std::vector<BatchInst> ins;
    build_tables(b, kps, ins);
    cudaError_t e = cudaMemcpyAsync(b->d_kp, kps.data(), sizeof(KParams) * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_inst, ins.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    drop_graph(b);
    return TLBM_OK;
}

static cudaError_t launch_batch(tlbm_batch_t b, int parity, cudaStream_t s) {
    if (b->staged_nc > 0) {
        BatchStagedInfo si{b->staged_tiles, b->staged_stages, &b->d_sync->staged_status, b->wait_ns};
        const int grid = (int)std::min<long long>(b->staged_tiles, b->staged_cap);
        return launch_batch_staged(b->dim, b->prec, b->staged_nc, b->d_kp, b->d_inst, b->n, parity, si, grid,
                                   b->staged_smem, s);
    }
    return batch_dispatch(true, b->dim, b->prec, b->vec, b->trt != 0, b->d_kp, b->d_inst, b->n, parity,
                          b->total_blocks, dim3(b->bx, b->by, 1), s, nullptr, eff_rows(b), b->tpb);
}

extern "C" int tlbm_batch_create(tlbm_batch_t* out, int n, const tlbm_instance* instances, int lattice,
                                 int precision, const tlbm_params* p) {
    g_batch_create_error[0] = 0;
    if (!out) return bfail(nullptr, TLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 65536 || !instances) return bfail(nullptr, TLBM_ERR_ARG, "need 1..65536 instances");
    if (p && p->streaming != TLBM_STREAM_PULL)
        return bfail(nullptr, TLBM_ERR_UNSUPPORTED, "batched ensembles use two-buffer streaming");
    tlbm_batch_s* b = new (std::nothrow) tlbm_batch_s();
    if (!b) return bfail(nullptr, TLBM_ERR_OOM, "host allocation failed");
    b->n = n;
    b->lattice = lattice;
    b->prec = precision;
    b->dim = lattice == TLBM_D3Q19_D3Q7 ? 3 : 2;
    b->graph_steps = 16;
    b->rows = 1;
    b->tpb = 8;
    b->wait_ns = GRID_WAIT_NS;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        tlbm_t h = nullptr;
        const tlbm_instance& in = instances[i];
        int rc = tlbm_create(&h, in.nx, in.ny, in.nz, lattice, in.Ra, in.Pr, in.Ma, precision, p);
        if (rc != TLBM_OK) {
            bfail(nullptr, rc, "instance %d: %s", i, tlbm_last_error(nullptr));
            for (tlbm_t q : b->inst) tlbm_destroy(q);
            delete b;
            return rc;
        }
        b->inst.push_back(h);
        b->off.push_back(off);
        b->seeds.push_back(in.seed);
        size_t need = 0;
        tlbm_required_bytes(h, &need);
        off += align_up(need, 256);
    }
    b->tables_off = off;
    b->total_bytes = off + align_up(sizeof(KParams) * n, 256) + align_up(sizeof(BatchInst) * n, 256) +
                     align_up(sizeof(GridSync), 256);
    batch_default_variant(b);
    *out = b;
    return TLBM_OK;
}

extern "C" int tlbm_batch_required_bytes(tlbm_batch_t b, size_t* bytes) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!bytes) return bfail(b, TLBM_ERR_ARG, "bytes is NULL");
    *bytes = b->total_bytes;
    return TLBM_OK;
}

extern "C" int tlbm_batch_bind_memory(tlbm_batch_t b, void* dev_ptr, size_t bytes) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!dev_ptr || ((uintptr_t)dev_ptr) % 256) return bfail(b, TLBM_ERR_ARG, "dev_ptr must be 256-byte aligned");
    if (bytes < b->total_bytes) return bfail(b, TLBM_ERR_OOM, "%zu bytes bound, %zu needed", bytes, b->total_bytes);
    for (int i = 0; i < b->n; ++i) {
        size_t need = 0;
        tlbm_required_bytes(b->inst[i], &need);
        int rc = tlbm_bind_memory(b->inst[i], (char*)dev_ptr + b->off[i], need);
        if (rc != TLBM_OK) return bfail(b, rc, "instance %d: %s", i, tlbm_last_error(b->inst[i]));
    }
    b->mem = (char*)dev_ptr;
    b->mem_bytes = bytes;
    b->d_kp = (KParams*)(b->mem + b->tables_off);
    b->d_inst = (BatchInst*)(b->mem + b->tables_off + align_up(sizeof(KParams) * b->n, 256));
    b->d_sync = (GridSync*)(b->mem + b->tables_off + align_up(sizeof(KParams) * b->n, 256) +
                            align_up(sizeof(BatchInst) * b->n, 256));
    cudaError_t e = cudaMemset(b->d_sync, 0, sizeof(GridSync));
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
    b->parity = 0;
    return upload_tables(b);
}

extern "C" int tlbm_batch_set_stream(tlbm_batch_t b, void* s) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    b->stream = (cudaStream_t)s;
    for (tlbm_t h : b->inst) tlbm_set_stream(h, s);
    drop_graph(b);
    return TLBM_OK;
}

extern "C" int tlbm_batch_init(tlbm_batch_t b, double noise_amp) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!b->mem) return bfail(b, TLBM_ERR_UNBOUND, "device memory not bound");
    for (int i = 0; i < b->n; ++i) {
        int rc = tlbm_init(b->inst[i], b->seeds[i], noise_amp);
        if (rc != TLBM_OK) return bfail(b, rc, "instance %d: %s", i, tlbm_last_error(b->inst[i]));
    }
    b->parity = 0;
    b->t = 0;
    cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(GridSync), b->stream);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return TLBM_OK;
}

static void advance(tlbm_batch_t b, int64_t k) {
    for (tlbm_t h : b->inst) {
        h->cur = (int)((h->cur + k) & 1);
        h->t += k;
    }
    b->parity = (int)((b->parity + k) & 1);
    b->t += k;
}

static int build_graph(tlbm_batch_t b) {
    drop_graph(b);
    cudaError_t e = cudaSuccess;
    if (!b->capture_stream) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < b->graph_steps && le == cudaSuccess; ++k) le = launch_batch(b, k & 1, b->capture_stream);
    e = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, TLBM_ERR_CUDA, "capture: %s", cudaGetErrorString(le != cudaSuccess ? le : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bfail(b, TLBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return TLBM_OK;
}

// One cooperative launch of the persistent kernel for k steps.
static int launch_persistent(tlbm_batch_t b, int k) {
    int per_sm = 0, dev = 0, sms = 0;
    Persist q{0, nullptr, 0, 0, &per_sm};
    cudaError_t e = batch_dispatch(false, b->dim, b->prec, b->vec, b->trt != 0, nullptr, nullptr, 0, 0, 0,
                                   dim3(b->bx, b->by, 1), nullptr, &q);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || per_sm < 1)
        return bfail(b, TLBM_ERR_CUDA, "persistent kernel occupancy: %s", cudaGetErrorString(e));
    const long long grid = std::min<long long>(b->total_blocks, (long long)per_sm * sms);
    Persist pp{k, b->d_sync, b->wait_ns, b->total_blocks, nullptr};
    // reset the barrier's counters; the status word stays set until the state
    // is initialised again, so that a timeout is not lost to a later launch
    e = cudaMemsetAsync(b->d_sync, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess)
        e = batch_dispatch(true, b->dim, b->prec, b->vec, b->trt != 0, b->d_kp, b->d_inst, b->n, b->parity, grid,
                           dim3(b->bx, b->by, 1), b->stream, &pp);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "persistent batch step: %s", cudaGetErrorString(e));
    return TLBM_OK;
}

extern "C" int tlbm_batch_step(tlbm_batch_t b, int64_t n) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!b->mem) return bfail(b, TLBM_ERR_UNBOUND, "device memory not bound");
    if (n < 0) return bfail(b, TLBM_ERR_ARG, "n must be >= 0");
    while (n > 0 && b->persist_steps > 0) {
        const int k = (int)std::min<int64_t>(n, b->persist_steps);
        const int rc = launch_persistent(b, k);
        if (rc != TLBM_OK) return rc;
        advance(b, k);
        b->launches += 1;
        n -= k;
    }
    while (n > 0) {
        if (b->graph_steps >= 2 && b->parity == 0 && n >= b->graph_steps) {
            if (!b->graph) {
                int rc = build_graph(b);
                if (rc != TLBM_OK) return rc;
            }
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
            advance(b, b->graph_steps);
            b->launches += b->graph_steps;
            n -= b->graph_steps;
        } else {
            cudaError_t e = launch_batch(b, b->parity, b->stream);
            if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "batch step: %s", cudaGetErrorString(e));
            advance(b, 1);
            b->launches += 1;
            n -= 1;
        }
    }
    return TLBM_OK;
}

extern "C" int tlbm_batch_set_variant(tlbm_batch_t b, int vec, int form, int block_x, int block_y,
                                      int graph_steps) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    int all_trt = 1;
    for (tlbm_t h : b->inst) all_trt = all_trt && h->kp.trt;
    if (form == 2 && !all_trt) return bfail(b, TLBM_ERR_ARG, "not every instance has two-relaxation-time rates");
    const int trt = form == 1 ? 0 : all_trt;
    const int v = vec > 0 ? vec : b->vec;
    const int bx = block_x > 0 ? block_x : b->bx, by = block_y > 0 ? block_y : b->by;
    if (bx % 32 || bx * by > 1024) return bfail(b, TLBM_ERR_ARG, "block_x must be a multiple of 32, bx*by <= 1024");
    if (graph_steps < 0 || graph_steps % 2) return bfail(b, TLBM_ERR_ARG, "graph_steps must be even (0 = no graph)");
    if (batch_dispatch(false, b->dim, b->prec, v, trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr) != cudaSuccess)
        return bfail(b, TLBM_ERR_UNSUPPORTED, "batch variant (vec %d, %s) not built", v, trt ? "TRT" : "MRT");
    b->vec = v;
    b->trt = trt;
    b->bx = bx;
    b->by = by;
    b->graph_steps = graph_steps;
    b->staged_nc = 0;  // an explicit register-kernel shape
    if (batch_dispatch(false, b->dim, b->prec, v, trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr, nullptr, b->rows) !=
        cudaSuccess)
        b->rows = 1;  // no pipelined-row variant for this one
    if (b->mem) return upload_tables(b);
    return TLBM_OK;
}

extern "C" int tlbm_batch_set_persistent(tlbm_batch_t b, int steps_per_launch) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (steps_per_launch < 0 || steps_per_launch > 1 << 20)
        return bfail(b, TLBM_ERR_ARG, "steps_per_launch must be in [0, 2^20]");
    int coop = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (steps_per_launch > 0 && (e != cudaSuccess || !coop))
        return bfail(b, TLBM_ERR_UNSUPPORTED, "the device has no cooperative launch");
    b->persist_steps = steps_per_launch;
    if (b->mem) return upload_tables(b);  // the persistent form runs one row per thread
    return TLBM_OK;
}

extern "C" int tlbm_batch_set_rows(tlbm_batch_t b, int rows) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (rows != 1 && rows != 2) return bfail(b, TLBM_ERR_ARG, "rows must be 1 or 2");
    if (batch_dispatch(false, b->dim, b->prec, b->vec, b->trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr, nullptr, rows) !=
        cudaSuccess)
        return bfail(b, TLBM_ERR_UNSUPPORTED, "batch variant (vec %d, %d rows) not built", b->vec, rows);
    b->rows = rows;
    if (b->mem) return upload_tables(b);
    return TLBM_OK;
}

extern "C" int tlbm_batch_get_rows(tlbm_batch_t b, int* rows) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!rows) return bfail(b, TLBM_ERR_ARG, "rows is NULL");
    *rows = b->rows;
    return TLBM_OK;
}

// The staged form needs 16-bit or FP32 storage and two-relaxation-time rates
// in every instance (and is not the persistent form).
static bool staged_possible(tlbm_batch_t b) {
    if (b->prec == TLBM_FP64 || b->persist_steps > 0) return false;
    for (tlbm_t h : b->inst)
        if (!h->kp.trt) return false;
    return true;
}

// Staged form with nc consumer warps (0: off) and `stages` tiles in flight per
// block (0: the most tiles in flight per SM up to six, more blocks first, as
// for a single cell).
static int batch_set_staged(tlbm_batch_t b, int nc, int stages) {
    if (nc == 0) {
        b->staged_nc = 0;
        return b->mem ? upload_tables(b) : TLBM_OK;
    }
    if (b->prec == TLBM_FP64) return bfail(b, TLBM_ERR_UNSUPPORTED, "the staged form has no FP64 variant");
    for (tlbm_t h : b->inst)
        if (!h->kp.trt) return bfail(b, TLBM_ERR_UNSUPPORTED, "the staged form needs two-relaxation-time rates");
    const int big = b->dim == 3 ? 7 : 8;
    if (nc != 4 && nc != big) return bfail(b, TLBM_ERR_ARG, "consumer warps must be 4 or %d", big);
    if (stages != 0 && (stages < 2 || stages > TILE_MAX_STAGES))
        return bfail(b, TLBM_ERR_ARG, "stages must be 0 or in [2, %d]", TILE_MAX_STAGES);
    const void* fn = batch_staged_function(b->dim, b->prec, nc);
    if (!fn) return bfail(b, TLBM_ERR_UNSUPPORTED, "staged batch kernel not built for this storage");
    const tlbm_t h0 = b->inst[0];
    const int A = 16 / (int)h0->elem;
    const size_t stage_bytes = (size_t)(h0->qf + h0->qg) * (64 * nc + 2 * A) * h0->elem;
    int dev = 0, optin = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "staged form setup: %s", cudaGetErrorString(e));
    const int threads = 32 * (nc + 1);
    int ns = stages;
    if (ns == 0) {
        int first = 0, best_in = 0, best_b = 0;
        for (int k = 2; k <= TILE_MAX_STAGES; ++k) {
            int blocks = 0;
            const size_t sm = 512 + (size_t)k * stage_bytes;
            if (sm > (size_t)optin) break;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, sm);
            if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
            if (blocks < 1) break;
            if (!first) first = k;
            const int in = blocks * k;
            if (in <= 6 && (in > best_in || (in == best_in && blocks > best_b))) {
                ns = k;
                best_in = in;
                best_b = blocks;
            }
        }
        if (ns == 0) ns = first;
        if (ns == 0) return bfail(b, TLBM_ERR_ARG, "two stages of %zu bytes do not fit in shared memory", stage_bytes);
    }
    const size_t smem = 512 + (size_t)ns * stage_bytes;
    if (smem > (size_t)optin) return bfail(b, TLBM_ERR_ARG, "%zu bytes of shared memory per block exceed %d", smem, optin);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return bfail(b, TLBM_ERR_ARG, "%zu bytes of shared memory per block do not fit", smem);
    b->staged_nc = nc;
    b->staged_stages = ns;
    b->staged_smem = smem;
    b->staged_cap = (long long)per_sm * sms;
    if (b->mem) return upload_tables(b);
    return TLBM_OK;
}

extern "C" int tlbm_batch_set_staged(tlbm_batch_t b, int consumer_warps, int stages) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (consumer_warps != 0 && b->persist_steps > 0)
        return bfail(b, TLBM_ERR_UNSUPPORTED, "the persistent form has no staged variant");
    if (consumer_warps < 0) return bfail(b, TLBM_ERR_ARG, "consumer_warps must be >= 0");
    return batch_set_staged(b, consumer_warps, stages);
}

extern "C" int tlbm_batch_get_staged(tlbm_batch_t b, int* consumer_warps, int* stages, long long* tiles) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (consumer_warps) *consumer_warps = b->staged_nc;
    if (stages) *stages = b->staged_nc ? b->staged_stages : 0;
    if (tiles) *tiles = b->staged_nc ? b->staged_tiles : 0;
    return TLBM_OK;
}

extern "C" int tlbm_batch_get_variant(tlbm_batch_t b, int* vec, int* form, int* block_x, int* block_y,
                                      int* graph_steps) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (vec) *vec = b->vec;
    if (form) *form = b->trt ? 2 : 1;
    if (block_x) *block_x = b->bx;
    if (block_y) *block_y = b->by;
    if (graph_steps) *graph_steps = b->graph_steps;
    return TLBM_OK;
}

// Tuned launch shapes of this process, per (lattice, storage, collision form,
// size class = floor(log2(total nodes))).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::array<int, 7>> g_tune_cache;

static std::tuple<int, int, int, int> tune_key(tlbm_batch_t b) {
    long long nodes = 0;
    for (tlbm_t h : b->inst) nodes += (long long)h->nx * h->ny * h->nz;
    int cls = 0;
    while ((2LL << cls) <= nodes) ++cls;
    return std::make_tuple(b->lattice, b->prec, b->trt, cls);
}

// Time each candidate launch shape on the bound state without changing it
// (every trial step reads the current buffers and writes the other ones, and
// the current buffers stay current), keep the fastest.  trials < 0 reuses the
// choice cached for the batch's (lattice, storage, form, size class) when there
// is one.
extern "C" int tlbm_batch_autotune(tlbm_batch_t b, int trials) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!b->mem) return bfail(b, TLBM_ERR_UNBOUND, "device memory not bound");
    if (trials < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(b));
        if (it != g_tune_cache.end()) {
            b->vec = it->second[0];
            b->bx = it->second[1];
            b->by = it->second[2];
            b->rows = it->second[3];
            b->tpb = it->second[4];
            if (it->second[5] > 0 && staged_possible(b)) return batch_set_staged(b, it->second[5], it->second[6]);
            b->staged_nc = 0;
            return upload_tables(b);
        }
    }
    const int reps = trials > 0 ? trials : 5;
    const int vecs[] = {8, 4, 2, 1};
    const int shapes[][2] = {{32, 1}, {32, 2}, {32, 4}, {64, 1}, {64, 2}, {128, 1}};
    const int keep_vec = b->vec, keep_bx = b->bx, keep_by = b->by, keep_rows = b->rows;
    b->staged_nc = 0;  // the register-kernel shapes first
    float best = 1e30f;
    int bv = keep_vec, bbx = keep_bx, bby = keep_by, brows = keep_rows;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, TLBM_ERR_CUDA, "cudaEventCreate");
    int rc = TLBM_OK;
    // rows per thread: the persistent form runs one
    const int max_rows = b->persist_steps > 0 ? 1 : 2;
    for (int v : vecs)
    for (int nr = 1; nr <= max_rows; ++nr) {
        if (batch_dispatch(false, b->dim, b->prec, v, b->trt != 0, nullptr, nullptr, 0, 0, 0, dim3(), nullptr, nullptr, nr) !=
            cudaSuccess)
            continue;
        for (const auto& sh : shapes) {
            b->vec = v;
            b->rows = nr;
            b->bx = sh[0];
            b->by = sh[1];
            if ((rc = upload_tables(b)) != TLBM_OK) break;
            cudaError_t e = launch_batch(b, b->parity, b->stream);  // warm
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_batch(b, b->parity, b->stream);
            cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                // a shape the kernel cannot launch (resources): skip it
                cudaGetLastError();
                continue;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            b->launches += reps + 1;
            if (ms < best) {
                best = ms;
                bv = v;
                brows = nr;
                bbx = sh[0];
                bby = sh[1];
            }
        }
        if (rc != TLBM_OK) break;
    }
    b->vec = bv;
    b->rows = brows;
    b->bx = bbx;
    b->by = bby;
    // tiles per block of the flattened launch, for the chosen shape
    int btpb = b->tpb;
    if (rc == TLBM_OK && b->persist_steps <= 0 && (rc = upload_tables(b)) == TLBM_OK) {
        best = 1e30f;
        const int tpbs[] = {1, 2, 4, 8, 16, 32};
        for (int tp : tpbs) {
            b->tpb = tp;
            cudaError_t e = launch_batch(b, b->parity, b->stream);  // warm
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_batch(b, b->parity, b->stream);
            cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            b->launches += reps + 1;
            if (ms < best) {
                best = ms;
                btpb = tp;
            }
        }
        b->tpb = btpb;
    }
    // the staged form (4 or the most consumer warps, 2 to 4 stages), against the
    // best register shape
    int bnc = 0, bns = 0;
    if (rc == TLBM_OK && staged_possible(b) && (rc = upload_tables(b)) == TLBM_OK) {
        const int ncs[] = {4, b->dim == 3 ? 7 : 8};
        const int nss[] = {2, 3, 4};
        for (int nc : ncs)
        for (int ns : nss) {
            if (batch_set_staged(b, nc, ns) != TLBM_OK) {
                b->err[0] = 0;
                continue;
            }
            cudaError_t e = launch_batch(b, b->parity, b->stream);  // warm
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_batch(b, b->parity, b->stream);
            cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            b->launches += reps + 1;
            if (ms < best) {
                best = ms;
                bnc = nc;
                bns = ns;
            }
        }
        b->staged_nc = 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == TLBM_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(b)] = {bv, bbx, bby, brows, btpb, bnc, bns};
    }
    int rc2 = bnc > 0 ? batch_set_staged(b, bnc, bns) : upload_tables(b);
    return rc != TLBM_OK ? rc : rc2;
}

extern "C" int tlbm_batch_instance(tlbm_batch_t b, int idx, tlbm_t* out) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (idx < 0 || idx >= b->n || !out) return bfail(b, TLBM_ERR_ARG, "bad instance index");
    *out = b->inst[idx];
    return TLBM_OK;
}

extern "C" int tlbm_batch_nusselt(tlbm_batch_t b, double* nu) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!nu) return bfail(b, TLBM_ERR_ARG, "nu is NULL");
    int first_diverged = -1;
    for (int i = 0; i < b->n; ++i) {
        int rc = tlbm_nusselt(b->inst[i], &nu[i]);
        if (rc == TLBM_ERR_DIVERGED) {
            if (first_diverged < 0) first_diverged = i;
        } else if (rc != TLBM_OK) {
            return bfail(b, rc, "instance %d: %s", i, tlbm_last_error(b->inst[i]));
        }
    }
    if (first_diverged >= 0)
        return bfail(b, TLBM_ERR_DIVERGED, "instance %d (and maybe others) has diverged; every value is written",
                      first_diverged);
    return TLBM_OK;
}

extern "C" int tlbm_batch_set_wait_limit(tlbm_batch_t b, double seconds) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!(seconds >= 0.0 && seconds <= 10.0)) return bfail(b, TLBM_ERR_ARG, "seconds must be in [0, 10]");
    b->wait_ns = (unsigned long long)(seconds * 1e9);
    return TLBM_OK;
}

extern "C" int tlbm_batch_status(tlbm_batch_t b, int* diverged) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (!diverged) return bfail(b, TLBM_ERR_ARG, "diverged is NULL");
    if (b->mem) {
        GridSync gs{};
        cudaError_t e = cudaMemcpyAsync(&gs, b->d_sync, sizeof(gs), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
        if (gs.status) return bfail(b, TLBM_ERR_TIMEOUT, "a persistent launch gave up waiting at a grid barrier");
        if (gs.staged_status) return bfail(b, TLBM_ERR_TIMEOUT, "a staged step gave up waiting for its copies");
    }
    for (int i = 0; i < b->n; ++i) {
        int rc = tlbm_status(b->inst[i], &diverged[i], nullptr);
        if (rc != TLBM_OK) return bfail(b, rc, "instance %d: %s", i, tlbm_last_error(b->inst[i]));
    }
    return TLBM_OK;
}

extern "C" int tlbm_batch_macros(tlbm_batch_t b, int idx, void* rho, void* ux, void* uy, void* uz, void* T,
                                 int out_dtype) {
    if (!b) return bfail(nullptr, TLBM_ERR_ARG, "NULL batch");
    if (idx < 0 || idx >= b->n) return bfail(b, TLBM_ERR_ARG, "bad instance index");
    int rc = tlbm_macros(b->inst[idx], rho, ux, uy, uz, T, out_dtype);
    if (rc != TLBM_OK) return bfail(b, rc, "instance %d: %s", idx, tlbm_last_error(b->inst[idx]));
    return TLBM_OK;
}

extern "C" int tlbm_batch_launch_count(tlbm_batch_t b, int64_t* count) {
    if (!b || !count) return bfail(b, TLBM_ERR_ARG, "NULL argument");
    *count = b->launches;
    return TLBM_OK;
}

extern "C" const char* tlbm_batch_last_error(tlbm_batch_t b) { return b ? b->err : g_batch_create_error; }

extern "C" void tlbm_batch_destroy(tlbm_batch_t b) {
    if (!b) return;
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (tlbm_t h : b->inst) tlbm_destroy(h);
    delete b;
}
