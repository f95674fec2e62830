// Shared-memory staged variant of the fused step: the same arithmetic as the
// register kernels (two-relaxation-time form, two nodes per thread on the FP32
// pair instructions), with the loads done by TMA bulk copies instead of
// per-thread loads.
//
// A persistent CTA walks a list of tiles; a tile is one row segment
// x in [x0, x0 + tw) of row (y, z).  Warp 0 is the producer: for every
// population j it copies the source row segment (the row shifted by -e_y, -e_z,
// widened by A elements on both sides so that the x-shift becomes a
// shared-memory offset) global -> shared with one cp.async.bulk, completing on
// the stage's "full" mbarrier; up to `stages` tiles are in flight.  The other NC
// warps are consumers: each thread pulls the populations of two adjacent nodes
// from shared memory (compile-time offsets), hands the stage back through its
// "empty" mbarrier (one arrival per warp), collides the two nodes and stores
// them with one 2-element store per population (a warp writes 64 consecutive
// nodes of each plane).
//
// Every wait is bounded in time: a block whose copies do not arrive records
// TLBM_ERR_TIMEOUT in a status word and returns; the producer warp, and so the
// block, stays until the copies it issued have landed (again bounded).
#pragma once
#include "kernels.cuh"

namespace tlbm {

constexpr int TILE_MAX_STAGES = 8;
constexpr unsigned long long TILE_WAIT_NS = 200000000;  // default: give up on a wait after 0.2 s
constexpr unsigned long long TILE_DRAIN_NS = 10000000;  // and on the drain after 10 ms

struct StagedInfo {
    int tw;             // tile width (nodes): a multiple of A, <= 64 NC
    int tiles_per_row;  // x segments per row
    int tiles;          // ny * nz * tiles_per_row (< 2^31)
    int stages;         // tiles in flight per CTA, 2 <= stages <= TILE_MAX_STAGES
    int* status;        // device status word (0 ok, 1 timeout)
    unsigned long long wait_ns;  // give up on a copy or a free stage after this long (0: at once)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
// Non-blocking test of the same (try_wait may suspend the thread for a while).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// The same with a suspend-time hint: a thread whose phase has not completed is
// parked until it completes or hint_ns have passed.  Without the hint a waiting
// warp returned to the loop below, re-reading the clock, about 20 times per
// tile (profile of the 3D FP16 staged kernel at 257^3).
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}
// Wait for the phase of `parity` to complete; false after `limit_ns` (0: false
// unless it has completed when first tested).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    if (limit_ns == 0) return mbar_test_wait(bar, parity);
    constexpr uint32_t HINT_NS = 1000000;  // park for at most 1 ms per try
    if (mbar_try_wait_hint(bar, parity, HINT_NS)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait_hint(bar, parity, HINT_NS))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// global -> shared bulk copy; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// the value enc_f_k / enc_g_k round to the storage type
template <class LF, class S, bool KS>
__device__ __forceinline__ float enc_val_f(float d, int i, float scale) {
    if constexpr (Storage<S>::offset) return KS ? d : d * scale;
    else return weight<LF, float>(i) + d;
}
template <class S, bool KS>
__device__ __forceinline__ float enc_val_g(float g, float scale) {
    if constexpr (Storage<S>::offset) return KS ? g : g * scale;
    else return g;
}

template <class S> struct Pair;
template <> struct Pair<float> {
    using T = float2;
    __device__ static float2 unpack(T v) { return v; }
    __device__ static T pack(float a, float b, uint32_t) { return make_float2(a, b); }
};
// pack(a, b): a at the lower address; 16-bit storage rounds stochastically
// (the time-step rounding of kernels.cuh, bitwise the scalar stores' result)
template <> struct Pair<__half> {
    using T = __half2;
    __device__ static float2 unpack(T v) { return __half22float2(v); }
    __device__ static T pack(float a, float b, uint32_t salt) {
        const uint32_t d = cvt_rs2<__half>(b, a, salt);
        T v;
        memcpy(&v, &d, 4);
        return v;
    }
};
template <> struct Pair<__nv_bfloat16> {
    using T = __nv_bfloat162;
    __device__ static float2 unpack(T v) { return __bfloat1622float2(v); }
    __device__ static T pack(float a, float b, uint32_t salt) {
        const uint32_t d = cvt_rs2<__nv_bfloat16>(b, a, salt);
        T v;
        memcpy(&v, &d, 4);
        return v;
    }
};

// Stage geometry of a kernel with NC consumer warps: tiles of up to 64 NC nodes,
// each population row padded by A elements on both sides.
template <class S, int NC>
struct TileGeo {
    static constexpr int A = 16 / (int)sizeof(S);
    static constexpr int TWMAX = 64 * NC;
    static constexpr int LW = TWMAX + 2 * A;
};

// Register caps.  An SM sub-partition holds 16384 registers, so a cap of R
// registers leaves room for floor(16384 / (32 R)) warps on each of the four,
// and a block of 1 + NC warps fits as often as those warps allow.  The 2D
// instance with 8 consumer warps fits in 72 registers: three blocks per SM (27
// warps); with two stages each that measured 114.8 GLUPS at 8193^2 FP16 (round
// to nearest) against 113.1 for two blocks of 96 registers with three stages,
// and with stochastic rounding (20 bytes spilled) 102.9 against 93.7 for 7
// consumer warps at 80.  The 3D instance runs 7 consumer warps (tiles up to 448
// nodes, one 385-node row) at 128 registers: two 8-warp blocks per SM without
// spilling, 46.5 GLUPS at 385^3 FP16 against 37.2 for 8 consumer warps held to
// 96 (156 bytes spilled; 48.1 there before stochastic rounding).  GB300, same
// box each.
template <int DIM, class S, int NC>
__global__ void __maxnreg__(DIM == 2 && NC == 8 ? 72 : (NC == 7 ? 128 : 168))
    step_staged_kernel(const S* __restrict__ src, S* __restrict__ dst, const KParams p, const StagedInfo si) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using P2 = Pair<S>;
    using S2 = typename P2::T;
    constexpr int QF = LF::Q, QG = LG::Q, Q = QF + QG;
    constexpr int A = TileGeo<S, NC>::A;
    constexpr int LW = TileGeo<S, NC>::LW;
    constexpr int STAGE = Q * LW;
    constexpr bool KS = Storage<S>::offset;  // offset storage: collide the stored, scaled values
    const Layout& L = p.L;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + TILE_MAX_STAGES;
    int4* head = reinterpret_cast<int4*>(empty + TILE_MAX_STAGES);  // per stage: x0, y, z, width
    S* stages = reinterpret_cast<S*>(smem_raw + 512);
    const int NS = si.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);  // one arrival per consumer warp
        }
        mbar_fence_init();
    }
    __syncthreads();

    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // step counter of 16-bit storage (stochastic rounding salt)
    const uint32_t tcount = step_count<S>(src, 0);
    advance_count<S>(dst, 0, tcount, blockIdx.x == 0 && threadIdx.x == 0);
    if (warp == 0) {
        // producer: tile t = (row r, segment k), row r = (y, z); the tile's
        // coordinates go to the stage header for the consumers; lane j < Q
        // copies population j (x-component ex of its velocity)
        int ex = 0;
        static_for<Q>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            if (lane == j) ex = j < QF ? LF::e(j < QF ? j : 0, 0) : LG::e(j < QF ? 0 : j - QF, 0);
        });
        int i = 0;
        int s = 0, ph = 0;  // stage and the parity of its current use
        for (int t = blockIdx.x; t < si.tiles; t += G, ++i) {
            if (i >= NS && !mbar_wait(&empty[s], (uint32_t)(ph ^ 1), si.wait_ns)) {
                if (lane == 0) atomicExch(si.status, 1);
                break;
            }
            const unsigned r = (unsigned)t / (unsigned)si.tiles_per_row;
            const int x0 = (t - (int)r * si.tiles_per_row) * si.tw;
            const unsigned z = r / (unsigned)L.ny;
            const int y = (int)(r - z * (unsigned)L.ny);
            const int tw = min(si.tw, L.nx - x0);
            // population `lane` needs x0 - 1 only if e_x = +1 and x0 + tw only
            // if e_x = -1; its copy starts and ends on 16-byte boundaries
            const int lo = ex == 1 ? x0 - A : x0;
            const int end = (x0 + tw + (ex == -1 ? 1 : 0) + A - 1) / A * A;
            const uint32_t bytes = lane < Q ? (uint32_t)(end - lo) * (uint32_t)sizeof(S) : 0u;
            const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
            if (lane == 0) {
                head[s] = make_int4(x0, y, (int)z, tw);
                mbar_arrive_expect_tx(&full[s], total);
            }
            __syncwarp();
            if (lane < Q)
                bulk_copy_g2s(stages + s * STAGE + lane * LW + (lo - (x0 - A)),
                              TLBM_DBG(p, (src + L.row(y, (int)z) + p.loff[lane] + lo), 0, (int)(bytes / sizeof(S))), bytes,
                              &full[s]);
            if (++s == NS) {
                s = 0;
                ph ^= 1;
            }
        }
        // the block stays until every copy this warp issued has landed (the
        // consumers have normally seen them all already)
        const int issued = i;
        for (int k = issued > NS ? issued - NS : 0; k < issued; ++k)
            if (!mbar_wait(&full[k % NS], (uint32_t)((k / NS) & 1), TILE_DRAIN_NS) && lane == 0)
                atomicExch(si.status, 1);
        return;
    }

    // consumers: thread c updates nodes x0 + 2c and x0 + 2c + 1 of each tile
    const int c = threadIdx.x - 32;
    const int xr = 2 * c;
    const uint32_t salt = step_salt(tcount);
    const float scale = ScaleOf<float>::s(p);
    const float inv_scale = ScaleOf<float>::inv(p);
    int s = 0, ph = 0;
    for (int t = blockIdx.x; t < si.tiles; t += G) {
        if (!mbar_wait(&full[s], (uint32_t)ph, si.wait_ns)) {
            atomicExch(si.status, 1);
            return;
        }
        const int4 hd = head[s];
        const int x0 = hd.x, y = hd.y, z = hd.z, tw = hd.w;
        const bool active = xr < tw;
        const S* st = stages + s * STAGE;
        float2 fd[QF], gd[QG];
        if (active) {
            static_for<QF>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                constexpr int ex = LF::e(q, 0);
                const S* rp = st + q * LW + A + xr - ex;
                float2 v;
                if constexpr (ex == 0) v = P2::unpack(*reinterpret_cast<const S2*>(rp));
                else v = make_float2(to_c<float>(rp[0]), to_c<float>(rp[1]));
                fd[q] = make_float2(raw_to_dev_k<LF, S, float, KS>(v.x, q, inv_scale),
                                    raw_to_dev_k<LF, S, float, KS>(v.y, q, inv_scale));
            });
            static_for<QG>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                constexpr int ex = LG::e(q, 0);
                const S* rp = st + (QF + q) * LW + A + xr - ex;
                float2 v;
                if constexpr (ex == 0) v = P2::unpack(*reinterpret_cast<const S2*>(rp));
                else v = make_float2(to_c<float>(rp[0]), to_c<float>(rp[1]));
                gd[q] = make_float2(raw_to_g_k<S, float, KS>(v.x, inv_scale), raw_to_g_k<S, float, KS>(v.y, inv_scale));
            });
        }
        // this warp is done with stage s
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == NS) {
            s = 0;
            ph ^= 1;
        }
        if (!active) continue;
        collide_trt_v<DIM, float2, collide_scaled<S, true>, true>(fd, gd, p);
        S* own = dst + L.row(y, z) + x0 + xr;
        if (xr + 1 < tw) {
            static_for<QF>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                *reinterpret_cast<S2*>(TLBM_DBG(p, (own + p.soff[q]), 0, 2)) =
                    P2::pack(enc_val_f<LF, S, KS>(fd[q].x, q, scale), enc_val_f<LF, S, KS>(fd[q].y, q, scale), salt);
            });
            static_for<QG>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                *reinterpret_cast<S2*>(TLBM_DBG(p, (own + p.soff[QF + q]), 0, 2)) =
                    P2::pack(enc_val_g<S, KS>(gd[q].x, scale), enc_val_g<S, KS>(gd[q].y, scale), salt);
            });
        } else {
            static_for<QF>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                *TLBM_DBG(p, (own + p.soff[q]), 0, 1) = enc_f_k<LF, S, float, KS>(fd[q].x, q, scale, salt);
            });
            static_for<QG>([&](auto ii) {
                constexpr int q = decltype(ii)::value;
                *TLBM_DBG(p, (own + p.soff[QF + q]), 0, 1) = enc_g_k<S, float, KS>(gd[q].x, scale, salt);
            });
        }
        float f2[QF][2], g2[QG][2];
#pragma unroll
        for (int q = 0; q < QF; ++q) { f2[q][0] = fd[q].x; f2[q][1] = fd[q].y; }
#pragma unroll
        for (int q = 0; q < QG; ++q) { g2[q][0] = gd[q].x; g2[q][1] = gd[q].y; }
        wall_writes<DIM, S, 2, float, KS>(dst, p, x0 + xr, y, z, f2, g2, salt);
    }
}

}  // namespace tlbm
