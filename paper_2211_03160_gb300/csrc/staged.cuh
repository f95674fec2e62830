// Shared-memory staged variant of the fused step (same arithmetic as
// step_kernel, different data movement).
//
// A persistent CTA walks a list of tiles; a tile is one row segment
// x in [x0, x0 + tw) of row (y, z).  For every population j the source row
// segment (shifted by -e_y, -e_z; the x-shift is a shared-memory offset) is
// copied global -> shared with one cp.async.bulk (TMA bulk copy) that signals an
// mbarrier with its byte count.  STAGES tiles are in flight per CTA, so the
// bytes in flight do not depend on the register budget, and the compute reads
// each node's neighbours from shared memory without shuffles.
//
// Waits are bounded: if a stage does not complete within the iteration budget
// the CTA records TLBM_ERR_TIMEOUT in a status word and returns.
#pragma once
#include "kernels.cuh"

namespace tlbm {

constexpr int STAGED_THREADS = 256;
constexpr int STAGED_MIN_BLOCKS = 4;  // 64 registers per thread, 32 warps per SM
constexpr int STAGED_MAX_STAGES = 8;
constexpr unsigned STAGED_WAIT_LIMIT = 1u << 22;   // try_wait iterations before giving up
constexpr unsigned STAGED_DRAIN_LIMIT = 1u << 16;  // second, shorter wait after a timeout

struct StagedInfo {
    int tw;           // tile width (nodes), a multiple of the 16-byte element count
    int tiles_per_row;
    long long tiles;  // rows * tiles_per_row
    int lw;           // shared row length per population (elements) = tw + 2*A
    int stages;       // tiles in flight per CTA (<= STAGED_MAX_STAGES)
    int* status;      // device status word (0 ok, 1 timeout)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// global -> shared bulk copy; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Issue the copies of tile t into one stage (called by warp 0 only).
template <int DIM, class S>
__device__ __forceinline__ void staged_issue(const S* __restrict__ src, const KParams& p, const StagedInfo& si,
                                             long long t, S* stage, uint64_t* bar) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    constexpr int Q = LF::Q + LG::Q;
    constexpr int A = 16 / (int)sizeof(S);
    const Layout& L = p.L;
    const int lane = threadIdx.x & 31;
    const long long r = t / si.tiles_per_row;
    const int x0 = (int)(t - r * si.tiles_per_row) * si.tw;
    const int y = (int)(r % L.ny);
    const int z = (int)(r / L.ny);
    const int tw_eff = min(si.tw, L.nx - x0);
    // window [x0 - A, end) with end >= x0 + tw_eff + 1, a multiple of A
    const int end = ((x0 + tw_eff + 1 + A - 1) / A) * A;
    const uint32_t bytes = (uint32_t)((end - (x0 - A)) * (int)sizeof(S));
    if (lane == 0) mbar_arrive_expect_tx(bar, bytes * Q);
    __syncwarp();
    if (lane < Q) {
        const S* g = src + L.row(y, z) + p.loff[lane] + (x0 - A);
        bulk_copy_g2s(stage + (long long)lane * si.lw, g, bytes, bar);
    }
}

template <int DIM, class S, bool TRT>
__global__ void __launch_bounds__(STAGED_THREADS, STAGED_MIN_BLOCKS) step_staged_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                                     const KParams p, const StagedInfo si) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    constexpr int QF = LF::Q, QG = LG::Q, Q = QF + QG;
    constexpr int A = 16 / (int)sizeof(S);
    const Layout& L = p.L;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    S* stages = reinterpret_cast<S*>(smem_raw + 128);
    const long long stage_elems = (long long)Q * si.lw;
    const int NS = si.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const long long G = gridDim.x;
    // prologue: fill the pipeline
    if (threadIdx.x < 32) {
        for (int s = 0; s < NS; ++s) {
            const long long t = blockIdx.x + s * G;
            if (t < si.tiles) staged_issue<DIM, S>(src, p, si, t, stages + s * stage_elems, &bars[s]);
        }
    }

    const C scale = ScaleOf<C>::s(p);
    const C inv_scale = ScaleOf<C>::inv(p);
    long long i = 0;
    for (long long t = blockIdx.x; t < si.tiles; t += G, ++i) {
        const int s = (int)(i % NS);
        const uint32_t parity = (uint32_t)((i / NS) & 1);
        unsigned spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&bars[s], parity)) {
            if (++spins > STAGED_WAIT_LIMIT) {
                ok = false;
                break;
            }
        }
        if (__syncthreads_or(!ok)) {
            // A stage never completed: record it, give the copies still in
            // flight a short bounded chance to land, and leave as a whole CTA.
            if (threadIdx.x == 0) {
                atomicExch(si.status, 1);
                for (int k = 0; k < NS; ++k) {
                    const long long tk = t + (long long)k * G;
                    if (tk >= si.tiles) break;
                    const int sk = (int)((i + k) % NS);
                    const uint32_t pk = (uint32_t)(((i + k) / NS) & 1);
                    unsigned d = 0;
                    while (!mbar_try_wait(&bars[sk], pk) && ++d < STAGED_DRAIN_LIMIT) {
                    }
                }
            }
            __syncthreads();
            return;
        }
        const S* st = stages + s * stage_elems;
        const long long r = t / si.tiles_per_row;
        const int x0 = (int)(t - r * si.tiles_per_row) * si.tw;
        const int y = (int)(r % L.ny);
        const int z = (int)(r / L.ny);
        const int tw_eff = min(si.tw, L.nx - x0);
        const long long rowo = L.row(y, z) + x0;
        const bool edge_row = (y == 0) || (y == L.ny - 1) || (DIM == 3 && (z == 0 || z == L.nz - 1));
        for (int xr = threadIdx.x; xr < tw_eff; xr += STAGED_THREADS) {
            C f[QF], g[QG];
            static_for<QF>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                const C raw = to_c<C>(st[q * si.lw + A + xr - LF::e(q, 0)]);
                f[q] = raw_to_dev<LF, S, C>(raw, q, inv_scale);
            });
            static_for<QG>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                const C raw = to_c<C>(st[(QF + q) * si.lw + A + xr - LG::e(q, 0)]);
                g[q] = raw_to_g<S, C>(raw, inv_scale);
            });
            collide<DIM, TRT, C>(f, g, p);
            S* own = dst + rowo + xr;
            static_for<QF>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                own[p.soff[q]] = enc_f<LF, S, C>(f[q], q, scale);
            });
            static_for<QG>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                own[p.soff[QF + q]] = enc_g<S, C>(g[q], scale);
            });
            const int x = x0 + xr;
            if (edge_row || x == 0 || x == L.nx - 1) {
                C post[Q];
#pragma unroll
                for (int q = 0; q < QF; ++q) post[q] = f[q];
#pragma unroll
                for (int q = 0; q < QG; ++q) post[QF + q] = g[q];
                edge_writes<DIM, S, 1, C>(dst, p, x, y, z, post);
            }
        }
        __syncthreads();  // every thread is done with stage s
        const long long tn = t + (long long)NS * G;
        if (threadIdx.x < 32 && tn < si.tiles)
            staged_issue<DIM, S>(src, p, si, tn, stages + s * stage_elems, &bars[s]);
    }
}

}  // namespace tlbm
