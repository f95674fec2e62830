// Shared-memory staged form of the batched ensemble step: the producer /
// consumer pipeline of the single-cell staged kernel (staged.cuh: warp 0 copies
// each tile's source row segments global -> shared with cp.async.bulk on an
// mbarrier ring, NC consumer warps collide two nodes per thread) walking the
// tiles of every instance.  Tiles are numbered instance by instance: instance i
// owns tiles [stile0_i, stile0_{i+1}), stpr_i per z-plane.  A tile is a stretch
// of stw_i elements of a z-plane's interior rows, which lie contiguously at the
// row pitch P (each row's ghost columns sit in its padding): tiles run over row
// ends, so that every tile but a plane's last is full whatever the width of
// the cell; the lanes that fall on padding idle.  The producer puts each tile's instance and that instance's step count
// (the stochastic-rounding salt of 16-bit storage) into the stage header next to
// the tile's coordinates; the consumers read the instance's parameters from the
// global table (read-only, the same block of ~1.2 KB for every tile of an
// instance) rather than from the kernel's parameter space.  The arithmetic per
// node is the single-cell staged kernel's.
#include "batch.h"
#include "staged.cuh"

namespace tlbm {

// Register caps (16384 registers per SM sub-partition): 2D with 8 consumer
// warps three blocks per SM, 3D with 7 two, as for the single-cell staged
// kernel; the 2D 16-bit body with 4 consumer warps at 96 registers, four
// 5-warp blocks per SM without spilling (the 64-cell FP16 ensemble: 78.3 GLUPS
// against 74.4 at its natural 112 registers, three blocks; FP32 stays
// uncapped, 1 % slower at 96).
template <int DIM, class S, int NC>
__global__ void __maxnreg__(DIM == 2 && NC == 8 ? 72
                                                : (NC == 7 ? 128 : (DIM == 2 && sizeof(S) == 2 ? 96 : 168)))
    batch_staged_kernel(const KParams* __restrict__ kps, const BatchInst* __restrict__ inst, int n, int parity,
                        const BatchStagedInfo si) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using P2 = Pair<S>;
    using S2 = typename P2::T;
    constexpr int QF = LF::Q, QG = LG::Q, Q = QF + QG;
    constexpr int A = TileGeo<S, NC>::A;
    constexpr int LW = TileGeo<S, NC>::LW;
    constexpr int STAGE = Q * LW;
    constexpr bool KS = Storage<S>::offset;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + TILE_MAX_STAGES;
    int4* head = reinterpret_cast<int4*>(empty + TILE_MAX_STAGES);  // per stage: x, y of e0, z, length
    int2* hinst = reinterpret_cast<int2*>(head + TILE_MAX_STAGES);  // per stage: instance, step count
    S* stages = reinterpret_cast<S*>(smem_raw + 512);
    const int NS = si.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);
        }
        mbar_fence_init();
    }
    __syncthreads();

    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        int ex = 0;
        static_for<Q>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            if (lane == j) ex = j < QF ? LF::e(j < QF ? j : 0, 0) : LG::e(j < QF ? 0 : j - QF, 0);
        });
        int i = 0;  // instance of tile t (tiles rise with the instance index)
        int k = 0, s = 0, ph = 0;
        for (long long t = blockIdx.x; t < si.tiles; t += G, ++k) {
            while (i + 1 < n && inst[i + 1].stile0 <= t) ++i;
            if (k >= NS && !mbar_wait(&empty[s], (uint32_t)(ph ^ 1), si.wait_ns)) {
                if (lane == 0) atomicExch(si.status, 1);
                break;
            }
            const KParams& p = kps[i];
            const long long local = t - inst[i].stile0;
            const int tpp = inst[i].stpr, tws = inst[i].stw;
            const int z = (int)(local / tpp);
            const int e0 = (int)(local - (long long)z * tpp) * tws;
            const int P = p.L.P;
            const int tw = min(tws, p.L.ny * P - e0);
            const S* src = static_cast<const S*>(inst[i].buf[parity]);
            // population `lane` needs e0 - 1 only if e_x = +1 and e0 + tw only
            // if e_x = -1; its copy starts and ends on 16-byte boundaries
            const int lo = ex == 1 ? e0 - A : e0;
            const int end = (e0 + tw + (ex == -1 ? 1 : 0) + A - 1) / A * A;
            const uint32_t bytes = lane < Q ? (uint32_t)(end - lo) * (uint32_t)sizeof(S) : 0u;
            const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
            if (lane == 0) {
                // the instance's step count; its first tile's producer advances it
                const uint32_t tc = step_count<S>(src, 0);
                advance_count<S>(static_cast<S*>(const_cast<void*>(inst[i].buf[parity ^ 1])), 0, tc, local == 0);
                const int y0 = e0 / P;  // the tile's first element: row y0, column e0 - y0 P
                head[s] = make_int4(e0 - y0 * P, y0, z, tw);
                hinst[s] = make_int2(i, (int)tc);
                mbar_arrive_expect_tx(&full[s], total);
            }
            __syncwarp();
            if (lane < Q)
                bulk_copy_g2s(stages + s * STAGE + lane * LW + (lo - (e0 - A)),
                              TLBM_DBG(p, (src + p.L.row(0, z) + p.loff[lane] + lo), 0, (int)(bytes / sizeof(S))),
                              bytes, &full[s]);
            if (++s == NS) {
                s = 0;
                ph ^= 1;
            }
        }
        const int issued = k;
        for (int q = issued > NS ? issued - NS : 0; q < issued; ++q)
            if (!mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1), TILE_DRAIN_NS) && lane == 0)
                atomicExch(si.status, 1);
        return;
    }

    const int c = threadIdx.x - 32;
    const int xr = 2 * c;
    int s = 0, ph = 0;
    for (long long t = blockIdx.x; t < si.tiles; t += G) {
        if (!mbar_wait(&full[s], (uint32_t)ph, si.wait_ns)) {
            atomicExch(si.status, 1);
            return;
        }
        const int4 hd = head[s];
        const int2 hi = hinst[s];
        const int z = hd.z, tw = hd.w;
        const KParams& p = kps[hi.x];
        int x = hd.x + xr, y = hd.y;  // this thread's first element, carried over row ends
        while (x >= p.L.P) {
            x -= p.L.P;
            ++y;
        }
        const bool active = xr < tw && x < p.L.nx;
        const bool both = xr + 1 < tw && x + 1 < p.L.nx;
        const S* st = stages + s * STAGE;
        const float inv_scale = ScaleOf<float>::inv(p);
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
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == NS) {
            s = 0;
            ph ^= 1;
        }
        if (!active) continue;
        const uint32_t salt = step_salt((uint32_t)hi.y);
        const float scale = ScaleOf<float>::s(p);
        collide_trt_v<DIM, float2, collide_scaled<S, true>, true>(fd, gd, p);
        S* dst = static_cast<S*>(const_cast<void*>(inst[hi.x].buf[parity ^ 1]));
        S* own = dst + p.L.row(y, z) + x;
        if (both) {
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
        wall_writes<DIM, S, 2, float, KS>(dst, p, x, y, z, f2, g2, salt);
    }
}

#define TLBM_BSTAGED_CASE(DIM, S, PREC, NC)                                                            \
    if (dim == DIM && prec == PREC && nc == NC) {                                                     \
        fn = (const void*)&batch_staged_kernel<DIM, S, NC>;                                           \
        if (launch)                                                                                   \
            batch_staged_kernel<DIM, S, NC><<<grid, 32 * (NC + 1), smem, s>>>(kps, inst, n, parity, si); \
    }

static cudaError_t bstaged_dispatch(int dim, int prec, int nc, bool launch, const void*& fn, const KParams* kps,
                                    const BatchInst* inst, int n, int parity, const BatchStagedInfo& si, int grid,
                                    size_t smem, cudaStream_t s) {
    fn = nullptr;
    TLBM_BSTAGED_CASE(2, float, 1, 4)
    TLBM_BSTAGED_CASE(2, float, 1, 8)
    TLBM_BSTAGED_CASE(2, __half, 2, 4)
    TLBM_BSTAGED_CASE(2, __half, 2, 8)
    TLBM_BSTAGED_CASE(2, __nv_bfloat16, 3, 4)
    TLBM_BSTAGED_CASE(2, __nv_bfloat16, 3, 8)
    TLBM_BSTAGED_CASE(3, float, 1, 4)
    TLBM_BSTAGED_CASE(3, float, 1, 7)
    TLBM_BSTAGED_CASE(3, __half, 2, 4)
    TLBM_BSTAGED_CASE(3, __half, 2, 7)
    TLBM_BSTAGED_CASE(3, __nv_bfloat16, 3, 4)
    TLBM_BSTAGED_CASE(3, __nv_bfloat16, 3, 7)
    if (!fn) return cudaErrorInvalidValue;
    return launch ? cudaGetLastError() : cudaSuccess;
}

const void* batch_staged_function(int dim, int prec, int nc) {
    const void* fn = nullptr;
    BatchStagedInfo si{};
    bstaged_dispatch(dim, prec, nc, false, fn, nullptr, nullptr, 0, 0, si, 0, 0, nullptr);
    return fn;
}

cudaError_t launch_batch_staged(int dim, int prec, int nc, const KParams* kps, const BatchInst* inst, int n,
                                int parity, const BatchStagedInfo& si, int grid, size_t smem, cudaStream_t s) {
    const void* fn = nullptr;
    return bstaged_dispatch(dim, prec, nc, true, fn, kps, inst, n, parity, si, grid, smem, s);
}

}  // namespace tlbm
