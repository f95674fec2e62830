// Learned warm start: the layers of a small 3x3 convolutional network and the
// pieces of its training loop, as CUDA kernels behind the C ABI.
//
// Convolutions are implicit GEMMs on the tensor cores, BF16 operands with FP32
// accumulation:
//   forward   out[b][m][p] = bias[m] + sum_k A[m][k] col(x)[k][b, p]
//             with A[m][9c + 3di + dj] = W[m][c][di][dj] (stored in the
//             kernel's shared-memory tile order, pack_weights_kernel) and
//             col(x) the 3x3 patches, on the 5th-generation tensor cores
//             (tcgen05.mma, accumulator in tensor memory);
//   data grad the same kernel with A = W transposed and flipped, x = dL/dy;
//   weight grad  dW[m][n] = sum_{b,p} dy[b][m][p] col(x)[n][b, p], per-CTA
//             partials over tiles of pixels summed in a fixed order
//             (deterministic), also on tcgen05.
// Layout: NCHW, 3x3 kernel, stride 1, zero padding 1.  Channel counts up to 32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tlbm.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int MAX_ROWS = 32;          // output channels at most (the MMA's N)

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ------------------------------------------------------------------ tcgen05 forward
//
// D[pixel][m] = bias[m] + sum_{c, di, dj} x[c][pixel + (di - 1, dj - 1)] A[m][9c + 3di + dj]
// on the 5th-generation tensor cores: tcgen05.mma, cta_group::1, kind::f16 (BF16
// in, FP32 accumulator in 32 columns of tensor memory), M = 128 pixels, N = 32
// output channels (zero-padded), K = 16 input channels per instruction.
//
// Pixels are walked in a padded "virtual" layout.  The image is cut into
// column strips of Wt = min(W, 126) columns; a strip with one halo column on
// either side is a virtual image of width Wv = Wt + 2, whose position
// v = (i + 1) Wv + (jj + 1) holds row i and strip column jj (image column
// j = s Wt + jj).  There the 3x3 neighbour (di - 1, dj - 1) of position v is
// v + (di - 1) Wv + (dj - 1), a constant shift.  A tile is the 128 positions
// v0 .. v0 + 127 (v0 = Wv + 128 t); the CTA stages positions v0 - Wv - 1 ..
// v0 + 128 + Wv of the input in shared memory channel-contiguous: position r
// of channel group g (channels 8g .. 8g + 7, zero past C) is the 16 bytes at
// sX + g PLANE + 16 r.  Read as a K-major operand whose core matrices are 8
// consecutive positions x 8 channels (row step 16 bytes, step between 8-row
// groups 128 bytes, step between the two K-adjacent channel groups PLANE), the
// patch rows of tap (di, dj) are the same bytes from row di Wv + dj on, so the
// layer is 9 x ceil(C / 16) MMAs per tile with no patch matrix built.  The
// halo columns' outputs (jj = -1 or Wt) are computed and dropped.
//
// Shared-memory operands are unswizzled, in 8-row x 16-byte core matrices.
// Matrix descriptor: start address >> 4 (bits 0-13), the byte step between
// K-adjacent core matrices >> 4 (16-29), the step between 8-row groups >> 4
// (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0).  Instruction
// descriptor: FP32 accumulator (bits 4-5 = 1), BF16 A and B (7-9, 10-12 = 1),
// both K-major (15, 16 = 0), N / 8 (17-22), M / 16 (24-28).  (Layouts checked
// on the GPU against a CPU product of one 128 x 32 x 16 tile before this
// kernel was written.)  The weights for tap t and channel chunk h (16
// channels) are a 32 x 16 K-major tile at sW + 1024 (t CH + h): core matrix
// (rows 8a.., channels 8e..) at 512 e + 128 a.  The packed weight operand in
// global memory is that image byte for byte, so staging it is a plain copy.
//
// The kernel is persistent: a CTA stages the weights once, then loops over
// tiles: stage the input tile, issue the MMAs from one thread, wait for their
// commit on an mbarrier (bounded), read the accumulator back with tcgen05.ld
// (warp w reads tensor-memory lanes 32w .. 32w + 31, i.e. its own 32
// positions) and store.
constexpr int TC_PIX = 128;        // output positions per tile (the MMA's M)
constexpr int TC_N = 32;           // output channels, zero-padded (the MMA's N)
constexpr int TC_WT = TC_PIX - 2;  // widest strip: its virtual row is one tile
constexpr int TC_BATCH = 8;        // input-tile items a thread loads before storing them
constexpr unsigned long long TC_WAIT_NS = 500000000;  // give up on the MMAs' completion after 0.5 s
__device__ unsigned long long g_conv_timeouts;        // CTAs that gave up (tlbm_conv3x3_status)

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t k_step, uint32_t row_step) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((k_step >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((row_step >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

struct TcGeom {
    int Wt, Wv, strips, tps;  // strip width, virtual width, strips per image, tiles per strip
    long long tiles;          // B x strips x tps
};

__host__ __device__ inline int tc_rows(int Wv) { return TC_PIX + 2 * Wv + 2; }
// weights, input tile, the tile's position table (int per row, padded to 16
// bytes), mbarrier + tensor-memory address slot
__host__ __device__ inline size_t tc_smem_bytes(int C, int Wv) {
    const int CH = (C + 15) / 16;
    return (size_t)9 * CH * 1024 + (size_t)2 * CH * tc_rows(Wv) * 16 + (size_t)(tc_rows(Wv) + 3) / 4 * 16 + 16;
}

// Image offset i W + j of virtual position v of strip s, or -1 outside the image.
__device__ __forceinline__ int tc_offset(int v, int s, int Wt, int Wv, int H, int W) {
    if (v < 0) return -1;
    const int i = v / Wv - 1, jj = v - (i + 1) * Wv - 1, j = s * Wt + jj;
    return (i >= 0 && i < H && j >= 0 && j < W) ? i * W + j : -1;
}

// out[b][m][i][j] (FP32) = bias[m] + conv; A: the 9 x CH weight tiles in the
// order they take in shared memory (pack_weights_kernel), M <= 32, C <= 32;
// out_act (optional, BF16) = relu(out) if relu else out.  Dynamic shared
// memory: tc_smem_bytes(C, Wv).
__global__ void __launch_bounds__(TC_PIX) conv3x3_tc_kernel(const bf16* __restrict__ A, int M,
                                                            const bf16* __restrict__ x, int C, int H, int W,
                                                            const float* __restrict__ bias, int relu,
                                                            float* __restrict__ out, bf16* __restrict__ out_act,
                                                            TcGeom geo) {
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    const int CH = (C + 15) / 16, G = 2 * CH;
    const int Wt = geo.Wt, Wv = geo.Wv;
    const int rows = tc_rows(Wv), plane = rows * 16;
    uint8_t* sW = tc_sm;
    uint8_t* sX = tc_sm + 9 * CH * 1024;
    int* xoff = reinterpret_cast<int*>(sX + (size_t)G * plane);  // image offset of each staged position
    uint64_t* bar = reinterpret_cast<uint64_t*>(xoff + (rows + 3) / 4 * 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    // this thread's first input-tile item (g0, r0) and the step between its items
    const int g0 = tid / rows, r0 = tid - g0 * rows, dg = TC_PIX / rows, dr = TC_PIX - dg * rows;
    const bf16 zero = __float2bfloat16_rn(0.f);

    // weights, once: a straight copy of 9 x CH KB (at most 9 pieces of 16
    // bytes per thread, all loads issued before the stores)
    {
        const int nw = 9 * CH * 64;
        uint4 v[9];
        if ((reinterpret_cast<uintptr_t>(A) & 15) == 0) {
            const uint4* A4 = reinterpret_cast<const uint4*>(A);
#pragma unroll
            for (int u = 0; u < 9; ++u)
                if (tid + u * TC_PIX < nw) v[u] = A4[tid + u * TC_PIX];
        } else {
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                const bf16* src = A + 8 * (tid + u * TC_PIX);
                if (tid + u * TC_PIX < nw)
                    v[u] = make_uint4(pack2(src[0], src[1]), pack2(src[2], src[3]), pack2(src[4], src[5]),
                                      pack2(src[6], src[7]));
            }
        }
#pragma unroll
        for (int u = 0; u < 9; ++u)
            if (tid + u * TC_PIX < nw) reinterpret_cast<uint4*>(sW)[tid + u * TC_PIX] = v[u];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tc_smem(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_PIX >> 4) << 24);
    const long long HW = (long long)H * W;

    uint32_t it = 0;
    for (long long tile = blockIdx.x; tile < geo.tiles; tile += gridDim.x, ++it) {
        const long long bs = tile / geo.tps;
        const int k = (int)(tile - bs * geo.tps);
        const int b = (int)(bs / geo.strips), s = (int)(bs - (long long)b * geo.strips);
        const int v0 = Wv + k * TC_PIX, vlo = v0 - Wv - 1;
        const bf16* xb = x + (long long)b * C * HW;
        // position table for this tile (the previous tile's readers are past
        // the barrier that ended their iteration)
        for (int r = tid; r < rows; r += TC_PIX) xoff[r] = tc_offset(vlo + r, s, Wt, Wv, H, W);
        __syncthreads();
        // input tile: item (g, r) = 8 channels of virtual position vlo + r;
        // TC_BATCH items per thread in flight before their stores
        int g = g0, r = r0;
        for (int e0 = 0; e0 < G * rows; e0 += TC_BATCH * TC_PIX) {
            uint32_t w4[TC_BATCH][4];
            int dst[TC_BATCH];
#pragma unroll
            for (int u = 0; u < TC_BATCH; ++u) {
                const bool in = e0 + u * TC_PIX + tid < G * rows;
                dst[u] = in ? g * plane + r * 16 : -1;
                w4[u][0] = w4[u][1] = w4[u][2] = w4[u][3] = 0u;
                const int o = (in && 8 * g < C) ? xoff[r] : -1;
                if (o >= 0) {
                    const bf16* p = xb + (long long)(8 * g) * HW + o;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c0 = 8 * g + 2 * q;
                        w4[u][q] = pack2(c0 < C ? p[(2 * q) * HW] : zero, c0 + 1 < C ? p[(2 * q + 1) * HW] : zero);
                    }
                }
                r += dr;
                g += dg;
                if (r >= rows) {
                    r -= rows;
                    ++g;
                }
            }
#pragma unroll
            for (int u = 0; u < TC_BATCH; ++u)
                if (dst[u] >= 0)
                    *reinterpret_cast<uint4*>(sX + dst[u]) = make_uint4(w4[u][0], w4[u][1], w4[u][2], w4[u][3]);
        }
        // the tile written by this CTA's threads becomes visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t x0 = tc_smem(sX), w0 = tc_smem(sW);
            for (int t = 0; t < 9; ++t) {
                const int shift = (t / 3) * Wv + (t % 3);
                for (int h = 0; h < CH; ++h) {
                    const uint64_t ad = tc_desc(x0 + 2 * h * plane + shift * 16, plane, 128);
                    const uint64_t bd = tc_desc(w0 + (t * CH + h) * 1024, 512, 128);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(t + h > 0))
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(bar))
                         : "memory");
        }
        // bounded wait for this tile's MMAs (phase `it` of the barrier)
        uint32_t done = 0;
        unsigned long long t0, t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (!done) {
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(tc_smem(bar)), "r"(it & 1u)
                : "memory");
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (!done && t1 - t0 > TC_WAIT_NS) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int failed = __syncthreads_or(!done);
        if (!failed) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr + ((uint32_t)(32 * warp) << 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int v = v0 + tid;
            const int i = v / Wv - 1, jj = v - (i + 1) * Wv - 1, j = s * Wt + jj;
            if (i < H && jj >= 0 && jj < Wt && j < W) {
                const long long o0 = (long long)b * M * HW + (long long)i * W + j;
#pragma unroll
                for (int m = 0; m < TC_N; ++m) {
                    if (m < M) {
                        const float y = __uint_as_float(r[m]) + (bias ? bias[m] : 0.f);
                        out[o0 + m * HW] = y;
                        if (out_act) out_act[o0 + m * HW] = __float2bfloat16_rn(relu ? fmaxf(y, 0.f) : y);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) {
            if (tid == 0) atomicAdd(&g_conv_timeouts, 1ull);
            break;
        }
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr) : "memory");
}

// ------------------------------------------------------------------ tcgen05 weight gradient
//
// dW[m][c][di][dj] = sum_{b, pixel} dy[b][m][pixel] x[b][c][pixel + (di - 1, dj - 1)]
// is a GEMM whose contraction runs over pixels: D[(t, c)][m] = sum_pos
// P[(t, c)][pos] dy[m][pos] with P the patch matrix (t = 3 di + dj), M = 9 Cp
// rows (Cp = 16 ceil(C / 16)) in blocks of 128, N = 32, K = the 128 virtual
// positions of a tile (the forward kernel's layout, halo columns and rows past
// the image carrying dy = 0).  A tap is a shift along K here, which no
// descriptor start address can express at element granularity, so each tile
// builds P explicitly in shared memory: the input tile is staged
// position-contiguous per channel (sX[c][r], r = 0 .. XR - 1 from virtual
// position v0 - Wv - 1; XR = 2 mod 4 so that a warp's 32 channels hit 32
// banks), and each 16-byte row piece of P, x[c][r + shift_t .. + 7], is put
// together from five aligned words (a byte permute when the shift is odd).
// P is K-major: core matrix (rows 8g.., positions 8k..) at 128 (k 9Cp/8 + g);
// dy is staged K-major too: core matrix (channels 8a.., positions 8k..) at
// 128 (4k + a).  The three (two for C <= 16) M-blocks accumulate in 32
// tensor-memory columns each across all the tiles a CTA takes; the rows of
// the last block past 9 Cp read whatever follows P in shared memory (the
// staged input) and are never read back.  Each CTA writes its partial
// part[cta][m][9c + t]; wgrad_reduce_kernel sums them in CTA order.  Staging
// the next tile's input and dy overlaps the previous tile's MMAs.
constexpr int WG_THREADS = 256;
constexpr int WG_TILE = 128;   // positions per tile (the K of one tile's MMAs)
constexpr int WG_BATCH = 8;    // input pairs a thread loads before storing them

__host__ __device__ inline int wg_xrows(int Wv) {
    const int r = WG_TILE + 2 * Wv + 4;  // shifts up to 2 Wv + 2, plus one word read ahead
    return r + ((2 - (r & 3)) & 3);
}
// patch matrix, input tile, dy tile, position tables (input rows and the
// tile's outputs, ints), mbarrier + tensor-memory address slot
__host__ __device__ inline size_t wg_smem_bytes(int C, int Wv) {
    const int Cp = 16 * ((C + 15) / 16);
    return (size_t)9 * Cp * WG_TILE * 2 + (size_t)Cp * wg_xrows(Wv) * 2 + (size_t)32 * WG_TILE * 2 +
           (size_t)(wg_xrows(Wv) + 2 + WG_TILE) * 4 + 16;
}

__device__ __forceinline__ bool wg_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done = 0;
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(tc_smem(bar)), "r"(parity)
            : "memory");
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (!done && t1 - t0 > TC_WAIT_NS) return false;
    }
    return true;
}

__global__ void __launch_bounds__(WG_THREADS) conv3x3_wgrad_tc_kernel(const bf16* __restrict__ dy, int M,
                                                                      const bf16* __restrict__ x, int C, int H,
                                                                      int W, TcGeom geo, float* __restrict__ part) {
    extern __shared__ __align__(1024) uint8_t wg_sm[];
    const int Cp = 16 * ((C + 15) / 16), R9 = 9 * Cp, RG = R9 / 8, nblk = (R9 + 127) / 128;
    const int Wt = geo.Wt, Wv = geo.Wv, XR = wg_xrows(Wv);
    uint8_t* sA = wg_sm;                                   // patch matrix, R9 x 128 positions
    uint16_t* sX = reinterpret_cast<uint16_t*>(wg_sm + (size_t)R9 * WG_TILE * 2);  // Cp x XR
    uint8_t* sB = reinterpret_cast<uint8_t*>(sX + (size_t)Cp * XR);               // 32 x 128 dy
    int* xoff = reinterpret_cast<int*>(sB + 32 * WG_TILE * 2);  // image offset of input row r, -1 outside
    int* yoff = xoff + XR + 2;                                  // image offset of output position r, -1 if none
    uint64_t* bar = reinterpret_cast<uint64_t*>(yoff + WG_TILE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long HW = (long long)H * W;
    // first pair (c, pair) of the input staging, first patch piece (kc, R),
    // and the steps between a thread's items
    const int HP = XR / 2;
    const int c0 = tid / HP, rp0 = tid - c0 * HP, dc = WG_THREADS / HP, drp = WG_THREADS - dc * HP;
    const int kc0 = tid / R9, R0 = tid - kc0 * R9, dk = WG_THREADS / R9, dR = WG_THREADS - dk * R9;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tc_smem(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

    bool ok = true;
    uint32_t it = 0;
    for (long long tile = blockIdx.x; tile < geo.tiles; tile += gridDim.x, ++it) {
        const long long bs = tile / geo.tps;
        const int k = (int)(tile - bs * geo.tps);
        const int b = (int)(bs / geo.strips), s = (int)(bs - (long long)b * geo.strips);
        const int v0 = Wv + k * WG_TILE, vlo = v0 - Wv - 1;
        const bf16* xb = x + (long long)b * C * HW;
        const bf16* db = dy + (long long)b * M * HW;
        // position tables (their previous readers finished before the barrier
        // ahead of the previous tile's MMAs)
        for (int r = tid; r < XR + WG_TILE; r += WG_THREADS) {
            if (r < XR) {
                xoff[r] = tc_offset(vlo + r, s, Wt, Wv, H, W);
            } else {
                const int v = v0 + (r - XR);
                const int i = v / Wv - 1, jj = v - (i + 1) * Wv - 1;
                yoff[r - XR] = (jj >= 0 && jj < Wt) ? tc_offset(v, s, Wt, Wv, H, W) : -1;
            }
        }
        __syncthreads();
        // input tile -> sX (pairs of positions); sX is free: the previous
        // tile's patch matrix was built before its MMAs were issued
        // (WG_BATCH pairs per thread in flight before their stores)
        const int npair = Cp * HP;
        int c = c0, rp = rp0;
        for (int e0 = 0; e0 < npair; e0 += WG_BATCH * WG_THREADS) {
            uint32_t h2[WG_BATCH];
            int dst[WG_BATCH];
#pragma unroll
            for (int u = 0; u < WG_BATCH; ++u) {
                const bool in = e0 + u * WG_THREADS + tid < npair;
                dst[u] = in ? c * HP + rp : -1;
                h2[u] = 0u;
                if (in && c < C) {
                    const int oa = xoff[2 * rp], ob = xoff[2 * rp + 1];
                    const bf16* xc = xb + (long long)c * HW;
                    if (oa >= 0) h2[u] = __bfloat16_as_ushort(xc[oa]);
                    if (ob >= 0) h2[u] |= (uint32_t)__bfloat16_as_ushort(xc[ob]) << 16;
                }
                rp += drp;
                c += dc;
                if (rp >= HP) {
                    rp -= HP;
                    ++c;
                }
            }
#pragma unroll
            for (int u = 0; u < WG_BATCH; ++u)
                if (dst[u] >= 0) reinterpret_cast<uint32_t*>(sX)[dst[u]] = h2[u];
        }
        // dy pieces (channel m, positions 8kc .. 8kc + 7) into registers
        uint4 dpc[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int p = tid + u * WG_THREADS, kc = p & 15, m = p >> 4;
            uint32_t w4[4] = {0u, 0u, 0u, 0u};
            if (m < M) {
                const bf16* dm = db + (long long)m * HW;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int o = yoff[8 * kc + e];
                    if (o >= 0) w4[e >> 1] |= (uint32_t)__bfloat16_as_ushort(dm[o]) << (16 * (e & 1));
                }
            }
            dpc[u] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        // the previous tile's MMAs must be done before sA and sB are rewritten
        if (it > 0) ok = wg_wait(bar, (it - 1) & 1u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int p = tid + u * WG_THREADS, kc = p & 15, m = p >> 4;
            *reinterpret_cast<uint4*>(sB + (kc * 4 + (m >> 3)) * 128 + (m & 7) * 16) = dpc[u];
        }
        // patch matrix: piece (row R = t Cp + c, position chunk kc)
        const uint32_t* sX32 = reinterpret_cast<const uint32_t*>(sX);
        int kc = kc0, R = R0;
        for (int p = tid; p < R9 * (WG_TILE / 8); p += WG_THREADS) {
            const int t = R / Cp, c = R - t * Cp;
            const int e0 = c * XR + (t / 3) * Wv + (t % 3) + 8 * kc;
            const uint32_t* w = sX32 + (e0 >> 1);
            const uint32_t w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
            uint4 v;
            if (e0 & 1) {
                const uint32_t w4 = w[4];
                v = make_uint4(__byte_perm(w0, w1, 0x5432), __byte_perm(w1, w2, 0x5432), __byte_perm(w2, w3, 0x5432),
                               __byte_perm(w3, w4, 0x5432));
            } else {
                v = make_uint4(w0, w1, w2, w3);
            }
            *reinterpret_cast<uint4*>(sA + (kc * RG + (R >> 3)) * 128 + (R & 7) * 16) = v;
            R += dR;
            kc += dk;
            if (R >= R9) {
                R -= R9;
                ++kc;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sB);
            for (int blk = 0; blk < nblk; ++blk)
                for (int kk = 0; kk < WG_TILE / 16; ++kk) {
                    const uint64_t ad = tc_desc(a0 + (2 * kk * RG + 16 * blk) * 128, RG * 128, 128);
                    const uint64_t bd = tc_desc(b0 + kk * 1024, 512, 128);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr + 32 * blk),
                        "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(it > 0 || kk > 0))
                        : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(bar))
                         : "memory");
        }
    }
    if (ok && it > 0) ok = wg_wait(bar, (it - 1) & 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = !__syncthreads_or(!ok);
    // partial: warp w reads tensor-memory lanes 32 (w % 4) .. of blocks w / 4, w / 4 + 2
    float* out = part + (long long)blockIdx.x * MAX_ROWS * 288;
    const int q = warp & 3;
    for (int blk = warp >> 2; blk < nblk; blk += 2) {
        uint32_t r[32];
        if (ok) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr + ((uint32_t)(32 * q) << 16) + 32 * blk));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
            for (int m = 0; m < 32; ++m) r[m] = 0x7fc00000u;  // NaN: a CTA that gave up poisons dW
        }
        const int R = blk * 128 + 32 * q + lane;
        if (R < R9) {
            const int t = R / Cp, c = R - t * Cp;
            if (c < C) {
#pragma unroll
                for (int m = 0; m < 32; ++m)
                    if (m < M) out[m * 288 + 9 * c + t] = __uint_as_float(r[m]);
            }
        }
    }
    if (!ok && tid == 0) atomicAdd(&g_conv_timeouts, 1ull);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(taddr) : "memory");
}

// dw[m][n] = sum_s part[s][m][n] in split order (deterministic), n < C*9; the
// loads run 8 partials ahead of the (sequential) sum.
__global__ void __launch_bounds__(64) wgrad_reduce_kernel(const float* __restrict__ part, int S, int M, int N,
                                                          float* __restrict__ dw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int m = idx / N, n = idx - m * N;
    const float* p = part + m * 288 + n;
    float s = 0.f;
    int k = 0;
    for (; k + 8 <= S; k += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[(long long)(k + u) * MAX_ROWS * 288];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; k < S; ++k) s += p[(long long)k * MAX_ROWS * 288];
    dw[idx] = s;
}

// db[m] = sum over (b, p) of dy32[b][m][p], in two fixed-order levels: block
// (sp, m) sums the sp-th of DB_SPLIT equal ranges of the flattened (b, p)
// index (each thread a strided subsequence, then a fixed tree) into
// partial[m][sp]; bias_grad_sum_kernel adds the DB_SPLIT partials in order.
constexpr int DB_SPLIT = 64;
__global__ void __launch_bounds__(256) bias_grad_kernel(const float* __restrict__ dy, int B, int M, long long HW,
                                                        float* __restrict__ partial) {
    __shared__ float sm[256];
    const int sp = blockIdx.x, m = blockIdx.y;
    const long long n = (long long)B * HW, L = (n + DB_SPLIT - 1) / DB_SPLIT;
    const long long q0 = sp * L, q1 = q0 + L < n ? q0 + L : n;
    float s = 0.f;
    long long q = q0 + threadIdx.x;
    long long b = q / HW, p = q - b * HW;
    for (; q + 768 < q1; q += 1024) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v[u] = dy[(b * M + m) * HW + p];
            p += 256;
            while (p >= HW) {
                p -= HW;
                ++b;
            }
        }
        s += v[0];
        s += v[1];
        s += v[2];
        s += v[3];
    }
    for (; q < q1; q += 256) {
        s += dy[(b * M + m) * HW + p];
        p += 256;
        while (p >= HW) {
            p -= HW;
            ++b;
        }
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[m * DB_SPLIT + sp] = sm[0];
}

__global__ void bias_grad_sum_kernel(const float* __restrict__ partial, int M, float* __restrict__ db) {
    const int m = threadIdx.x;
    if (m >= M) return;
    float s = 0.f;
    for (int k = 0; k < DB_SPLIT; ++k) s += partial[m * DB_SPLIT + k];
    db[m] = s;
}

// Element idx of the tensor-core weight operand (tile order of
// conv3x3_tc_kernel's shared memory): (tap t, chunk h, output row m, input
// channel c) with idx = 512 (t CH + h) + 256 (c' / 8) + 64 (m / 8) + 8 (m % 8)
// + c' % 8, c = 16 h + c'.
struct TapIndex {
    int t, m, c;
};
__device__ __forceinline__ TapIndex tap_index(int idx, int CH) {
    const int th = idx >> 9, e = idx & 511;
    const int t = th / CH, h = th - t * CH;
    return {t, 8 * ((e >> 6) & 3) + ((e >> 3) & 7), 16 * h + 8 * (e >> 8) + (e & 7)};
}

// Data-gradient operand: At(t, m = input channel, c = output channel)
// = W[c][m][2 - di][2 - dj] (t = 3 di + dj), zero where m >= M or c >= C.
__global__ void flip_transpose_kernel(const bf16* __restrict__ w, int C, int M, bf16* __restrict__ at) {
    const int CH = (C + 15) / 16;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9 * CH * 512) return;
    const TapIndex q = tap_index(idx, CH);
    at[idx] = (q.m < M && q.c < C) ? w[((q.c * M + q.m) * 3 + (2 - q.t / 3)) * 3 + (2 - q.t % 3)]
                                   : __float2bfloat16_rn(0.f);
}

// Forward operand: A(t, m, c) = W[m][c][di][dj] (FP32 master -> BF16), zero
// where m >= O or c >= C.
__global__ void pack_weights_kernel(const float* __restrict__ w, int O, int C, bf16* __restrict__ a) {
    const int CH = (C + 15) / 16;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9 * CH * 512) return;
    const TapIndex q = tap_index(idx, CH);
    a[idx] = __float2bfloat16_rn((q.m < O && q.c < C) ? w[(q.m * C + q.c) * 9 + q.t] : 0.f);
}

__global__ void relu_backward_kernel(const float* __restrict__ dx, const float* __restrict__ y, long long n,
                                     float* __restrict__ g32, bf16* __restrict__ g16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = y[i] > 0.f ? dx[i] : 0.f;
        g32[i] = v;
        g16[i] = __float2bfloat16_rn(v);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, long long n, bf16* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// grad = 2 (y - t) / n in FP32 and BF16; partial sums of (y - t)^2 per block.
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ tgt, long long n,
                           float* __restrict__ g32, bf16* __restrict__ g16, double* __restrict__ partial) {
    __shared__ double sm[256];
    double s = 0.0;
    const float sc = 2.0f / (float)n;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float d = y[i] - tgt[i];
        s += (double)d * d;
        g32[i] = sc * d;
        g16[i] = __float2bfloat16_rn(sc * d);
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int np, long long n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += partial[i];
        out[0] = s / (double)n;
    }
}

// Adam (Kingma & Ba 2015) on FP32 master weights.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Vertex-aligned bilinear upsampling of C planes (h x w) by an integer factor.
__global__ void upsample_kernel(const float* __restrict__ in, int C, int h, int w, int f, float* __restrict__ out) {
    const int H = (h - 1) * f + 1, Wd = (w - 1) * f + 1;
    const long long n = (long long)C * H * Wd;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / ((long long)H * Wd));
        const int r = (int)(idx - (long long)c * H * Wd);
        const int I = r / Wd, J = r - I * Wd;
        int i0 = I / f, j0 = J / f;
        if (i0 > h - 2) i0 = h - 2;
        if (j0 > w - 2) j0 = w - 2;
        const float ty = (float)(I - i0 * f) / f, tx = (float)(J - j0 * f) / f;
        const float* p = in + (long long)c * h * w;
        const float f00 = p[i0 * w + j0], f01 = p[i0 * w + j0 + 1];
        const float f10 = p[(i0 + 1) * w + j0], f11 = p[(i0 + 1) * w + j0 + 1];
        out[idx] = (1.f - ty) * ((1.f - tx) * f00 + tx * f01) + ty * ((1.f - tx) * f10 + tx * f11);
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? TLBM_OK : TLBM_ERR_CUDA; }

bool conv_shape_ok(int B, int C, int M, int H, int W) {
    return B > 0 && C > 0 && C <= 32 && M > 0 && M <= MAX_ROWS && H > 0 && W > 0 &&
           (long long)B * H * W < (1ll << 40) && (long long)H * W < (1ll << 31) && (long long)H * TC_PIX < (1ll << 30);
}

// Persistent launch: as many CTAs as fit the SMs at once (about 43 KB of
// shared memory each at 32 channels), never more than there are tiles.
// Tiles of 128 virtual positions (both tensor-core kernels walk the same layout).
TcGeom tc_geometry(int B, int H, int W) {
    TcGeom geo;
    geo.Wt = W < TC_WT ? W : TC_WT;
    geo.Wv = geo.Wt + 2;
    geo.strips = (W + geo.Wt - 1) / geo.Wt;
    geo.tps = (int)(((long long)H * geo.Wv + TC_PIX - 1) / TC_PIX);
    geo.tiles = (long long)B * geo.strips * geo.tps;
    return geo;
}

// Persistent grid: CTAs resident per SM as many as shared memory holds (228 KB
// per SM, 1 KB reserved per CTA), at most `cap` (tensor-memory columns: an SM
// has 512), never more CTAs than tiles.
int persistent_grid(long long tiles, size_t smem, long long cap, long long* grid) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TLBM_ERR_CUDA;
    long long per = (long long)(228 * 1024) / (long long)(smem + 1024);
    per = per < 1 ? 1 : (per > cap ? cap : per);
    *grid = tiles < sms * per ? tiles : sms * per;
    return TLBM_OK;
}

int launch_tc(const bf16* A, int M, const bf16* x, int B, int C, int H, int W, const float* bias, int relu,
              float* out, bf16* out_act, cudaStream_t s) {
    const TcGeom geo = tc_geometry(B, H, W);
    const size_t smem = tc_smem_bytes(C, geo.Wv);
    // launched with the largest shared-memory carveout so that the CTAs counted fit
    static const cudaError_t carve = cudaFuncSetAttribute(
        conv3x3_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    long long grid = 0;
    if (carve != cudaSuccess || persistent_grid(geo.tiles, smem, 8, &grid) != TLBM_OK) return TLBM_ERR_CUDA;
    conv3x3_tc_kernel<<<(unsigned)grid, TC_PIX, smem, s>>>(A, M, x, C, H, W, bias, relu, out, out_act, geo);
    return status_of(cudaGetLastError());
}

// Weight-gradient grid (the number of partials) for a shape.
int wgrad_grid(int B, int C, int H, int W, long long* grid) {
    const TcGeom geo = tc_geometry(B, H, W);
    return persistent_grid(geo.tiles, wg_smem_bytes(C, geo.Wv), 4, grid);
}

}  // namespace

extern "C" int tlbm_conv3x3_pack_weights(const float* w, int cout, int cin, void* a, void* stream) {
    if (!w || !a || cout < 1 || cout > MAX_ROWS || cin < 1 || cin > 32) return TLBM_ERR_ARG;
    const int n = 9 * 512 * ((cin + 15) / 16);
    pack_weights_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(w, cout, cin, (bf16*)a);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_conv3x3_forward(const void* x, const void* a, const float* bias, float* y, void* y_act,
                                    int B, int cin, int cout, int H, int W, int relu, void* stream) {
    if (!x || !a || !y || !conv_shape_ok(B, cin, cout, H, W)) return TLBM_ERR_ARG;
    return launch_tc((const bf16*)a, cout, (const bf16*)x, B, cin, H, W, bias, relu, y, (bf16*)y_act,
                     (cudaStream_t)stream);
}

extern "C" int tlbm_conv3x3_backward_data(const void* dy, const void* w_bf16, float* dx, int B, int cin, int cout,
                                          int H, int W, void* at_workspace, void* stream) {
    if (!dy || !w_bf16 || !dx || !at_workspace || !conv_shape_ok(B, cout, cin, H, W)) return TLBM_ERR_ARG;
    const int n = 9 * 512 * ((cout + 15) / 16);
    flip_transpose_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)w_bf16, cout, cin,
                                                                             (bf16*)at_workspace);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    return launch_tc((const bf16*)at_workspace, cin, (const bf16*)dy, B, cout, H, W, nullptr, 0, dx, nullptr,
                     (cudaStream_t)stream);
}

extern "C" int tlbm_conv3x3_weight_elems(int cin) { return cin < 1 || cin > 32 ? 0 : 9 * 512 * ((cin + 15) / 16); }

extern "C" int tlbm_conv3x3_status(unsigned long long* timeouts) {
    if (!timeouts) return TLBM_ERR_ARG;
    return status_of(cudaMemcpyFromSymbol(timeouts, g_conv_timeouts, sizeof(unsigned long long)));
}

extern "C" int tlbm_conv3x3_workspace_bytes(int B, int cin, int cout, int H, int W, size_t* bytes) {
    if (!bytes || !conv_shape_ok(B, cin, cout, H, W)) return TLBM_ERR_ARG;
    long long S = 0;
    if (wgrad_grid(B, cin, H, W, &S) != TLBM_OK) return TLBM_ERR_CUDA;
    const size_t part = ((size_t)S * MAX_ROWS * 288 + (size_t)MAX_ROWS * DB_SPLIT) * sizeof(float);
    const size_t at = (size_t)MAX_ROWS * 288 * sizeof(bf16);
    *bytes = part > at ? part : at;
    return TLBM_OK;
}

extern "C" int tlbm_conv3x3_backward_weight(const void* x, const void* dy_bf16, const float* dy, float* dw,
                                            float* db, int B, int cin, int cout, int H, int W, void* workspace,
                                            size_t workspace_bytes, void* stream) {
    if (!x || !dy_bf16 || !dw || !workspace || !conv_shape_ok(B, cin, cout, H, W)) return TLBM_ERR_ARG;
    size_t need = 0;
    tlbm_conv3x3_workspace_bytes(B, cin, cout, H, W, &need);
    if (workspace_bytes < need) return TLBM_ERR_OOM;
    const TcGeom geo = tc_geometry(B, H, W);
    const size_t smem = wg_smem_bytes(cin, geo.Wv);
    static const cudaError_t attr = cudaFuncSetAttribute(
        conv3x3_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wg_smem_bytes(32, TC_PIX));
    static const cudaError_t carve = cudaFuncSetAttribute(
        conv3x3_wgrad_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    long long S = 0;
    if (attr != cudaSuccess || carve != cudaSuccess || wgrad_grid(B, cin, H, W, &S) != TLBM_OK) return TLBM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    conv3x3_wgrad_tc_kernel<<<(unsigned)S, WG_THREADS, smem, s>>>((const bf16*)dy_bf16, cout, (const bf16*)x, cin, H,
                                                                  W, geo, (float*)workspace);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    wgrad_reduce_kernel<<<grid_for((long long)cout * cin * 9, 64), 64, 0, s>>>((const float*)workspace, (int)S,
                                                                             cout, cin * 9, dw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    if (db && dy) {
        float* partial = (float*)workspace + (size_t)S * MAX_ROWS * 288;
        bias_grad_kernel<<<dim3(DB_SPLIT, cout), 256, 0, s>>>(dy, B, cout, (long long)H * W, partial);
        e = cudaGetLastError();
        if (e != cudaSuccess) return TLBM_ERR_CUDA;
        bias_grad_sum_kernel<<<1, MAX_ROWS, 0, s>>>(partial, cout, db);
        e = cudaGetLastError();
    }
    return status_of(e);
}

extern "C" int tlbm_relu_backward(const float* dx, const float* y, long long n, float* g, void* g_bf16,
                                  void* stream) {
    if (!dx || !y || !g || !g_bf16 || n < 0) return TLBM_ERR_ARG;
    relu_backward_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(dx, y, n, g, (bf16*)g_bf16);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_to_bf16(const float* a, long long n, void* b, void* stream) {
    if (!a || !b || n < 0) return TLBM_ERR_ARG;
    to_bf16_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(a, n, (bf16*)b);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_mse_loss(const float* y, const float* target, long long n, float* g, void* g_bf16,
                             double* loss_dev, double* partial_dev, void* stream) {
    if (!y || !target || !g || !g_bf16 || !loss_dev || !partial_dev || n < 1) return TLBM_ERR_ARG;
    const int blocks = grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024;
    cudaStream_t s = (cudaStream_t)stream;
    mse_kernel<<<blocks, 256, 0, s>>>(y, target, n, g, (bf16*)g_bf16, partial_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    sum_partials_kernel<<<1, 32, 0, s>>>(partial_dev, blocks, n, loss_dev);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_adam_step(float* w, const float* g, float* m, float* v, long long n, float lr, float b1,
                              float b2, float eps, int t, void* stream) {
    if (!w || !g || !m || !v || n < 0 || t < 1) return TLBM_ERR_ARG;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_upsample_bilinear(const float* in, int channels, int h, int w, int factor, float* out,
                                      void* stream) {
    if (!in || !out || channels < 1 || h < 2 || w < 2 || factor < 1) return TLBM_ERR_ARG;
    const long long n = (long long)channels * ((h - 1) * factor + 1) * ((w - 1) * factor + 1);
    upsample_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, channels, h, w, factor, out);
    return status_of(cudaGetLastError());
}
