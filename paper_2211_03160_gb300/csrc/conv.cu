// Learned warm start: the layers of a small 3x3 convolutional network and the
// pieces of its training loop, as CUDA kernels behind the C ABI.
//
// Convolutions are implicit GEMMs on the tensor cores, BF16 operands with FP32
// accumulation:
//   forward   out[b][m][p] = bias[m] + sum_k A[m][k] col(x)[k][b, p]
//             with A = W reshaped to [Cout][Cin*9] and col(x) the 3x3 patches,
//             on the 5th-generation tensor cores (tcgen05.mma, accumulator in
//             tensor memory);
//   data grad the same kernel with A = W transposed and flipped, x = dL/dy;
//   weight grad  dW[m][n] = sum_{b,p} dy[b][m][p] col(x)[n][b, p], split over
//             pixel ranges and summed in a fixed order (deterministic), on the
//             warp-level mma.sync m16n8k16.
// Layout: NCHW, 3x3 kernel, stride 1, zero padding 1.  Channel counts up to 32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tlbm.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int CONV_THREADS = 128;     // 4 warps; each warp: 32 output rows x 32 pixels
constexpr int MAX_ROWS = 32;          // output channels per GEMM (two 16-row tiles)
constexpr int WG_SPLIT = 2048;        // pixels summed by one weight-gradient block
constexpr int WG_NT = 9;              // 8-column tiles per warp in the weight gradient (36 = 288 / 8 per block)

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D += A B for one 16x8x16 tile; fragment layouts as in the PTX ISA for
// mma.m16n8k16 with .bf16 inputs (g = lane/4, t = lane%4):
//   A regs: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
//   B regs: (k = 2t..2t+1, n = g), (k = 2t+8.., n = g)
//   D:      (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One element of the 3x3 patch matrix: row k = c*9 + di*3 + dj, pixel (b, i, j).
__device__ __forceinline__ bf16 patch(const bf16* __restrict__ x, int k, int K, int b, int i, int j, int C, int H,
                                      int W, bool pix_ok) {
    if (!pix_ok || k >= K) return __float2bfloat16_rn(0.f);
    const int c = k / 9, r = k - 9 * c;
    const int ii = i + r / 3 - 1, jj = j + r % 3 - 1;
    if (ii < 0 || ii >= H || jj < 0 || jj >= W) return __float2bfloat16_rn(0.f);
    return x[(((long long)b * C + c) * H + ii) * W + jj];
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
constexpr int TC_BATCH = 4;        // input-tile items a thread loads before storing them
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
__host__ __device__ inline size_t tc_smem_bytes(int C, int Wv) {
    const int CH = (C + 15) / 16;
    return (size_t)9 * CH * 1024 + (size_t)2 * CH * tc_rows(Wv) * 16 + 16;
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
    uint64_t* bar = reinterpret_cast<uint64_t*>(sX + (size_t)G * plane);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
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
        // input tile: item (g, r) = 8 channels of virtual position vlo + r;
        // TC_BATCH items per thread in flight before their stores
        for (int e0 = 0; e0 < G * rows; e0 += TC_BATCH * TC_PIX) {
            uint32_t w4[TC_BATCH][4];
#pragma unroll
            for (int u = 0; u < TC_BATCH; ++u) {
                const int e = e0 + u * TC_PIX + tid;
                const int g = e / rows, r = e - g * rows;
                const int v = vlo + r;
                w4[u][0] = w4[u][1] = w4[u][2] = w4[u][3] = 0u;
                if (e < G * rows && v >= 0 && 8 * g < C) {
                    const int i = v / Wv - 1, jj = v - (i + 1) * Wv - 1;
                    const int j = s * Wt + jj;
                    if (i >= 0 && i < H && j >= 0 && j < W) {
                        const bf16* p = xb + (long long)(8 * g) * HW + (long long)i * W + j;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c0 = 8 * g + 2 * q;
                            w4[u][q] = pack2(c0 < C ? p[(2 * q) * HW] : zero,
                                             c0 + 1 < C ? p[(2 * q + 1) * HW] : zero);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < TC_BATCH; ++u) {
                const int e = e0 + u * TC_PIX + tid;
                const int g = e / rows, r = e - g * rows;
                if (e < G * rows)
                    *reinterpret_cast<uint4*>(sX + g * plane + r * 16) =
                        make_uint4(w4[u][0], w4[u][1], w4[u][2], w4[u][3]);
            }
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

// Weight gradient partials: part[s][m][n] = sum over pixels q in split s of
// dy[b][m][p] * patch(x)[n][b, p], n < N = C*9 (padded to Np = 288 columns).
__global__ void __launch_bounds__(CONV_THREADS) conv3x3_wgrad_kernel(const bf16* __restrict__ dy, int M,
                                                                     const bf16* __restrict__ x, int B, int C,
                                                                     int H, int W, float* __restrict__ part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int N = C * 9;
    const long long HW = (long long)H * W, P = (long long)B * HW;
    const long long q0 = (long long)blockIdx.x * WG_SPLIT;
    const long long q1 = q0 + WG_SPLIT < P ? q0 + WG_SPLIT : P;
    float acc[2][WG_NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < WG_NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][j][e] = 0.f;

    for (long long qk = q0; qk < q1; qk += 16) {
        // pixels of this k-step handled by the thread: qk + 2t + {0, 1, 8, 9}
        long long qs[4] = {qk + 2 * t, qk + 2 * t + 1, qk + 2 * t + 8, qk + 2 * t + 9};
        int bq[4], iq[4], jq[4];
        bool ok[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ok[e] = qs[e] < q1;
            const long long qq = ok[e] ? qs[e] : q0;
            bq[e] = (int)(qq / HW);
            const long long r = qq - (long long)bq[e] * HW;
            iq[e] = (int)(r / W);
            jq[e] = (int)(r - (long long)iq[e] * W);
        }
        // A fragment from dy: rows m = mt*16 + g (+8), columns k = pixels
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            bf16 v[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = mt * 16 + g + 8 * h;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long long p = (long long)iq[e] * W + jq[e];
                    v[h * 4 + e] = (m < M && ok[e]) ? dy[((long long)bq[e] * M + m) * HW + p] : __float2bfloat16_rn(0.f);
                }
            }
            // v[h*4 + e]: h = row half (g / g+8), e = pixel slot (2t, 2t+1, 2t+8, 2t+9)
            a[mt][0] = pack2(v[0], v[1]);
            a[mt][1] = pack2(v[4], v[5]);
            a[mt][2] = pack2(v[2], v[3]);
            a[mt][3] = pack2(v[6], v[7]);
        }
#pragma unroll
        for (int j = 0; j < WG_NT; ++j) {
            const int n = (warp + 4 * j) * 8 + g;  // this thread's B column
            uint32_t b0 = pack2(patch(x, n, N, bq[0], iq[0], jq[0], C, H, W, ok[0]),
                                patch(x, n, N, bq[1], iq[1], jq[1], C, H, W, ok[1]));
            uint32_t b1 = pack2(patch(x, n, N, bq[2], iq[2], jq[2], C, H, W, ok[2]),
                                patch(x, n, N, bq[3], iq[3], jq[3], C, H, W, ok[3]));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][j], a[mt], b0, b1);
        }
    }
    float* out = part + (long long)blockIdx.x * MAX_ROWS * 288;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < WG_NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = mt * 16 + g + (e >= 2 ? 8 : 0);
                const int n = (warp + 4 * j) * 8 + 2 * t + (e & 1);
                out[m * 288 + n] = acc[mt][j][e];
            }
}

// dw[m][n] = sum_s part[s][m][n] in split order (deterministic), n < C*9.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int S, int M, int N, float* __restrict__ dw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int m = idx / N, n = idx - m * N;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += part[(long long)k * MAX_ROWS * 288 + m * 288 + n];
    dw[idx] = s;
}

// db[m] = sum over (b, p) of dy32[b][m][p]; one block per m, fixed tree.
__global__ void bias_grad_kernel(const float* __restrict__ dy, int B, int M, long long HW, float* __restrict__ db) {
    __shared__ float sm[256];
    const int m = blockIdx.x;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (long long p = threadIdx.x; p < HW; p += 256) s += dy[((long long)b * M + m) * HW + p];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[m] = sm[0];
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
           (long long)B * H * W < (1ll << 40) && (long long)H * TC_PIX < (1ll << 30);
}

// Persistent launch: as many CTAs as fit the SMs at once (about 43 KB of
// shared memory each at 32 channels), never more than there are tiles.
int launch_tc(const bf16* A, int M, const bf16* x, int B, int C, int H, int W, const float* bias, int relu,
              float* out, bf16* out_act, cudaStream_t s) {
    TcGeom geo;
    geo.Wt = W < TC_WT ? W : TC_WT;
    geo.Wv = geo.Wt + 2;
    geo.strips = (W + geo.Wt - 1) / geo.Wt;
    geo.tps = (int)(((long long)H * geo.Wv + TC_PIX - 1) / TC_PIX);
    geo.tiles = (long long)B * geo.strips * geo.tps;
    const size_t smem = tc_smem_bytes(C, geo.Wv);
    // CTAs resident per SM: as many as shared memory holds (228 KB per SM,
    // 1 KB reserved per CTA), at most 8 (each holds 32 of the SM's 512
    // tensor-memory columns); launched with the largest shared-memory carveout.
    static const cudaError_t carve = cudaFuncSetAttribute(
        conv3x3_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    int dev = 0, sms = 0;
    if (carve != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TLBM_ERR_CUDA;
    long long per = (long long)(228 * 1024) / (long long)(smem + 1024);
    per = per < 1 ? 1 : (per > 8 ? 8 : per);
    const long long grid = geo.tiles < sms * per ? geo.tiles : sms * per;
    conv3x3_tc_kernel<<<(unsigned)grid, TC_PIX, smem, s>>>(A, M, x, C, H, W, bias, relu, out, out_act, geo);
    return status_of(cudaGetLastError());
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
    const long long P = (long long)B * H * W;
    const long long S = (P + WG_SPLIT - 1) / WG_SPLIT;
    const size_t part = (size_t)S * MAX_ROWS * 288 * sizeof(float);
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
    const long long P = (long long)B * H * W;
    const int S = (int)((P + WG_SPLIT - 1) / WG_SPLIT);
    cudaStream_t s = (cudaStream_t)stream;
    conv3x3_wgrad_kernel<<<S, CONV_THREADS, 0, s>>>((const bf16*)dy_bf16, cout, (const bf16*)x, B, cin, H, W,
                                                    (float*)workspace);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    wgrad_reduce_kernel<<<grid_for((long long)cout * cin * 9, 256), 256, 0, s>>>((const float*)workspace, S, cout,
                                                                               cin * 9, dw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    if (db && dy) {
        bias_grad_kernel<<<cout, 256, 0, s>>>(dy, B, cout, (long long)H * W, db);
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
