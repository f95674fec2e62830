// tlbm_reduce_noalloc: the FP64 diagnostic reduction (the sums behind
// tlbm_nusselt, tlbm_energy and tlbm_status) for callers that cannot allocate
// device memory.
//
// The handle-based reductions keep their block partials in the scratch part of
// the block the caller bound with tlbm_bind_memory.  Some callers hold a
// population state but cannot allocate any device memory to go with it: for
// example a monitoring process that maps a running simulation's state through
// CUDA IPC on a GPU whose memory that simulation has taken, or an application
// whose device memory is all held by its own pool allocator.
// This entry point needs nothing from them but the state and a host array: its
// partial sums live in a fixed array compiled into this file, and nothing here
// calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/tlbm.h"
#include "handle.h"
#include "kernels.cuh"

using namespace tlbm;

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 16384;  // consecutive nodes summed by one block
constexpr int NA_SLOTS = 8192;         // partial-sum slots held by the static array
constexpr int NA_FIELDS = 6;
constexpr int NA_FINAL_THREADS = 1024;
constexpr int NA_MAX_DEVICES = 64;

// Static scratch: NA_SLOTS partial rows of NA_FIELDS doubles, then one result
// row (8 doubles).  384 KiB + 64 B on every device that loads the library, held
// until the process exits.  Every call overwrites each slot it later reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU (two
// streams, two handles, two threads) share this array and race.
__device__ __align__(256) double g_noalloc_scratch[NA_SLOTS * NA_FIELDS + 8];

// Pass 1: block b sums nodes [b*NA_CHUNK, min(N, (b+1)*NA_CHUNK)); thread t takes
// every NA_THREADS-th node of the chunk in order; fixed shuffle tree; fixed
// cross-warp order.  Fields: sum u_h T, sum 1/2 rho u^2, sum rho, max u^2,
// non-finite flag, sum T.
template <int DIM, class S>
__global__ void __launch_bounds__(NA_THREADS) noalloc_partials(const S* __restrict__ buf, const KParams p,
                                                               double* __restrict__ scratch) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const Layout& L = p.L;
    const long long N = (long long)L.nx * L.ny * L.nz;
    const long long n0 = (long long)blockIdx.x * NA_CHUNK;
    const long long n1 = n0 + NA_CHUNK < N ? n0 + NA_CHUNK : N;
    double acc[NA_FIELDS] = {0, 0, 0, 0, 0, 0};
    for (long long n = n0 + threadIdx.x; n < n1; n += NA_THREADS) {
        const int x = (int)(n % L.nx);
        const long long r = n / L.nx;
        const int y = (int)(r % L.ny);
        const int z = (int)(r / L.ny);
        double t[5];
        node_terms<DIM, S>(buf, p, x, y, z, t);
        acc[0] += t[0];
        acc[1] += t[1];
        acc[2] += t[2];
        acc[3] = fmax(acc[3], t[3]);
        if (!isfinite(t[2]) || !isfinite(t[4]) || !isfinite(t[3])) acc[4] = 1.0;
        acc[5] += t[4];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < NA_FIELDS; ++k) {
            const double o = __shfl_down_sync(0xffffffffu, acc[k], off);
            acc[k] = (k == 3 || k == 4) ? fmax(acc[k], o) : acc[k] + o;
        }
    }
    __shared__ double sm[NA_THREADS / 32][NA_FIELDS];
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < NA_FIELDS; ++k) sm[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < NA_THREADS / 32; ++j)
            for (int k = 0; k < NA_FIELDS; ++k)
                sm[0][k] = (k == 3 || k == 4) ? fmax(sm[0][k], sm[j][k]) : sm[0][k] + sm[j][k];
        for (int k = 0; k < NA_FIELDS; ++k) scratch[(long long)blockIdx.x * NA_FIELDS + k] = sm[0][k];
    }
}

// Pass 2: one block; thread t combines slots t, t + 1024, ... in order, then a
// fixed tree.  Reads only the `slots` rows written by pass 1 of this call.
__global__ void __launch_bounds__(NA_FINAL_THREADS) noalloc_final(double* __restrict__ scratch, int slots) {
    __shared__ double sm[NA_FINAL_THREADS];
    double* out = scratch + (long long)NA_SLOTS * NA_FIELDS;
    for (int k = 0; k < NA_FIELDS; ++k) {
        const bool is_max = (k == 3 || k == 4);
        double a = 0.0;
        for (int s = threadIdx.x; s < slots; s += NA_FINAL_THREADS) {
            const double v = scratch[(long long)s * NA_FIELDS + k];
            a = is_max ? fmax(a, v) : a + v;
        }
        sm[threadIdx.x] = a;
        __syncthreads();
        for (int s = NA_FINAL_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s)
                sm[threadIdx.x] = is_max ? fmax(sm[threadIdx.x], sm[threadIdx.x + s]) : sm[threadIdx.x] + sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sm[0];
        __syncthreads();
    }
}

template <int DIM, class S>
cudaError_t launch_partials(const void* buf, const KParams& p, double* scratch, int slots, cudaStream_t s) {
    noalloc_partials<DIM, S><<<slots, NA_THREADS, 0, s>>>((const S*)buf, p, scratch);
    return cudaGetLastError();
}

cudaError_t launch_partials_any(int dim, int prec, const void* buf, const KParams& p, double* scratch, int slots,
                                cudaStream_t s) {
    if (dim == 2) {
        switch (prec) {
        case TLBM_FP64: return launch_partials<2, double>(buf, p, scratch, slots, s);
        case TLBM_FP32: return launch_partials<2, float>(buf, p, scratch, slots, s);
        case TLBM_FP16_OFFSET: return launch_partials<2, __half>(buf, p, scratch, slots, s);
        default: return launch_partials<2, __nv_bfloat16>(buf, p, scratch, slots, s);
        }
    }
    switch (prec) {
    case TLBM_FP64: return launch_partials<3, double>(buf, p, scratch, slots, s);
    case TLBM_FP32: return launch_partials<3, float>(buf, p, scratch, slots, s);
    case TLBM_FP16_OFFSET: return launch_partials<3, __half>(buf, p, scratch, slots, s);
    default: return launch_partials<3, __nv_bfloat16>(buf, p, scratch, slots, s);
    }
}

int na_fail(tlbm_t h, int code, const char* msg, const char* detail = nullptr) {
    if (detail) snprintf(h->err, sizeof(h->err), "%s: %s", msg, detail);
    else snprintf(h->err, sizeof(h->err), "%s", msg);
    return code;
}

// Device address of g_noalloc_scratch for each device, looked up once per
// device (with that device current) the first time this entry point runs there.
std::mutex g_setup_mutex;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int tlbm_reduce_noalloc(tlbm_t h, const void* state, double* out) {
    if (!h) return TLBM_ERR_ARG;
    h->err[0] = 0;
    if (!out) return na_fail(h, TLBM_ERR_ARG, "out is NULL");
    const long long N = (long long)h->nx * h->ny * h->nz;
    const long long slots = (N + NA_CHUNK - 1) / NA_CHUNK;
    if (slots > NA_SLOTS) {
        char d[160];
        snprintf(d, sizeof(d), "%lld nodes need %lld partial slots; the static scratch holds %d (at most %lld nodes)",
                 N, slots, NA_SLOTS, (long long)NA_SLOTS * NA_CHUNK);
        return na_fail(h, TLBM_ERR_ARG, "cell too large for tlbm_reduce_noalloc", d);
    }
    const void* buf = state;
    if (!buf) {
        if (!h->mem) return na_fail(h, TLBM_ERR_UNBOUND, "state is NULL and no device memory is bound");
        buf = h->buf[h->cur];
    } else {
        cudaPointerAttributes a;
        cudaError_t e = cudaPointerGetAttributes(&a, buf);
        if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "cudaPointerGetAttributes", cudaGetErrorString(e));
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return na_fail(h, TLBM_ERR_ARG, "state is not device memory");
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "cudaGetSymbolAddress", cudaGetErrorString(e));
    KParams kp = h->kp;
#ifdef TLBM_DEBUG_BOUNDS
    // the checks cover the state actually read; with no bound block its
    // violations land in the static scratch and go unreported
    kp.dbg_lo = (const char*)buf;
    kp.dbg_hi = (const char*)buf + h->popset_bytes;
    if (!h->mem) kp.dbg_count = reinterpret_cast<unsigned long long*>(scratch + (long long)NA_SLOTS * NA_FIELDS + 7);
#endif
    e = launch_partials_any(h->dim, h->prec, buf, kp, scratch, (int)slots, h->stream);
    if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "partial-sum kernel", cudaGetErrorString(e));
    noalloc_final<<<1, NA_FINAL_THREADS, 0, h->stream>>>(scratch, (int)slots);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "final-sum kernel", cudaGetErrorString(e));
    h->launches += 2;
    e = cudaMemcpyAsync(out, scratch + (long long)NA_SLOTS * NA_FIELDS, NA_FIELDS * sizeof(double),
                        cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "cudaMemcpyAsync", cudaGetErrorString(e));
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return na_fail(h, TLBM_ERR_CUDA, "cudaStreamSynchronize", cudaGetErrorString(e));
    return TLBM_OK;
}
