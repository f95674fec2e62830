// Learned warm start: the layers of a small 3x3 convolutional network and the
// pieces of its training loop, as CUDA kernels behind the C ABI.
//
// Convolutions are implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation):
//   forward   out[b][m][p] = bias[m] + sum_k A[m][k] col(x)[k][b, p]
//             with A = W reshaped to [Cout][Cin*9] and col(x) the 3x3 patches;
//   data grad the same kernel with A = W transposed and flipped, x = dL/dy;
//   weight grad  dW[m][n] = sum_{b,p} dy[b][m][p] col(x)[n][b, p], split over
//             pixel ranges and summed in a fixed order (deterministic).
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

// out[b][m][p] (FP32) = bias[m] + sum_k A[m][k] * patch(x)[k][b, p];
// A: BF16 [M][Kp], zero for k >= K = C*9, Kp a multiple of 16, M <= 32.
// out_act (optional, BF16) = relu(out) if relu else out.
__global__ void __launch_bounds__(CONV_THREADS) conv3x3_igemm_kernel(const bf16* __restrict__ A, int M, int Kp,
                                                                     const bf16* __restrict__ x, int B, int C,
                                                                     int H, int W, const float* __restrict__ bias,
                                                                     int relu, float* __restrict__ out,
                                                                     bf16* __restrict__ out_act) {
    extern __shared__ uint32_t sA[];  // MAX_ROWS x Kp BF16 as 32-bit pairs
    const int words = MAX_ROWS * Kp / 2;
    const uint32_t* A32 = reinterpret_cast<const uint32_t*>(A);
    for (int w = threadIdx.x; w < words; w += CONV_THREADS) sA[w] = (w < M * Kp / 2) ? A32[w] : 0u;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int K = C * 9;
    const long long HW = (long long)H * W, P = (long long)B * HW;
    const long long pbase = (long long)blockIdx.x * CONV_THREADS + warp * 32;
    int pb[4], pi[4], pj[4];
    bool pok[4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const long long q = pbase + nt * 8 + g;
        pok[nt] = q < P;
        const long long qq = pok[nt] ? q : 0;
        pb[nt] = (int)(qq / HW);
        const long long r = qq - (long long)pb[nt] * HW;
        pi[nt] = (int)(r / W);
        pj[nt] = (int)(r - (long long)pi[nt] * W);
    }
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;

    for (int k0 = 0; k0 < Kp; k0 += 16) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = mt * 16 + g;
            a[mt][0] = sA[(r0 * Kp + k0 + 2 * t) >> 1];
            a[mt][1] = sA[((r0 + 8) * Kp + k0 + 2 * t) >> 1];
            a[mt][2] = sA[(r0 * Kp + k0 + 2 * t + 8) >> 1];
            a[mt][3] = sA[((r0 + 8) * Kp + k0 + 2 * t + 8) >> 1];
        }
        const int kb = k0 + 2 * t;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint32_t b0 = pack2(patch(x, kb, K, pb[nt], pi[nt], pj[nt], C, H, W, pok[nt]),
                                      patch(x, kb + 1, K, pb[nt], pi[nt], pj[nt], C, H, W, pok[nt]));
            const uint32_t b1 = pack2(patch(x, kb + 8, K, pb[nt], pi[nt], pj[nt], C, H, W, pok[nt]),
                                      patch(x, kb + 9, K, pb[nt], pi[nt], pj[nt], C, H, W, pok[nt]));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], a[mt], b0, b1);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = mt * 16 + g + (e >= 2 ? 8 : 0);
                const long long q = pbase + nt * 8 + 2 * t + (e & 1);
                if (m >= M || q >= P) continue;
                const long long b = q / HW, p = q - b * HW;
                const float v = acc[mt][nt][e] + (bias ? bias[m] : 0.f);
                const long long o = (b * M + m) * HW + p;
                out[o] = v;
                if (out_act) out_act[o] = __float2bfloat16_rn(relu ? fmaxf(v, 0.f) : v);
            }
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

// At[c][o*9 + di*3 + dj] = W[o][c][2-di][2-dj], zero-padded to Kp columns.
__global__ void flip_transpose_kernel(const bf16* __restrict__ w, int O, int C, int Kp, bf16* __restrict__ at) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C * Kp) return;
    const int c = idx / Kp, k = idx - c * Kp;
    if (k >= O * 9) {
        at[idx] = __float2bfloat16_rn(0.f);
        return;
    }
    const int o = k / 9, r = k - 9 * o, di = r / 3, dj = r % 3;
    at[idx] = w[((o * C + c) * 3 + (2 - di)) * 3 + (2 - dj)];
}

// W [O][C][3][3] (FP32 master) -> A [O][Kp] BF16, zero-padded.
__global__ void pack_weights_kernel(const float* __restrict__ w, int O, int C, int Kp, bf16* __restrict__ a) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= O * Kp) return;
    const int o = idx / Kp, k = idx - o * Kp;
    a[idx] = __float2bfloat16_rn(k < C * 9 ? w[o * C * 9 + k] : 0.f);
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
           (long long)B * H * W < (1ll << 40);
}

}  // namespace

extern "C" int tlbm_conv3x3_pack_weights(const float* w, int cout, int cin, void* a, void* stream) {
    if (!w || !a || cout < 1 || cout > MAX_ROWS || cin < 1 || cin > 32) return TLBM_ERR_ARG;
    const int Kp = (cin * 9 + 15) / 16 * 16;
    pack_weights_kernel<<<grid_for((long long)cout * Kp, 256), 256, 0, (cudaStream_t)stream>>>(w, cout, cin, Kp,
                                                                                            (bf16*)a);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_conv3x3_forward(const void* x, const void* a, const float* bias, float* y, void* y_act,
                                    int B, int cin, int cout, int H, int W, int relu, void* stream) {
    if (!x || !a || !y || !conv_shape_ok(B, cin, cout, H, W)) return TLBM_ERR_ARG;
    const int Kp = (cin * 9 + 15) / 16 * 16;
    const long long P = (long long)B * H * W;
    const size_t smem = (size_t)MAX_ROWS * Kp * sizeof(bf16);
    conv3x3_igemm_kernel<<<(unsigned)((P + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, smem,
                           (cudaStream_t)stream>>>((const bf16*)a, cout, Kp, (const bf16*)x, B, cin, H, W, bias, relu,
                                                   y, (bf16*)y_act);
    return status_of(cudaGetLastError());
}

extern "C" int tlbm_conv3x3_backward_data(const void* dy, const void* w_bf16, float* dx, int B, int cin, int cout,
                                          int H, int W, void* at_workspace, void* stream) {
    if (!dy || !w_bf16 || !dx || !at_workspace || !conv_shape_ok(B, cout, cin, H, W)) return TLBM_ERR_ARG;
    const int Kp = (cout * 9 + 15) / 16 * 16;
    flip_transpose_kernel<<<grid_for((long long)cin * Kp, 256), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)w_bf16, cout, cin, Kp, (bf16*)at_workspace);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TLBM_ERR_CUDA;
    const long long P = (long long)B * H * W;
    const size_t smem = (size_t)MAX_ROWS * Kp * sizeof(bf16);
    conv3x3_igemm_kernel<<<(unsigned)((P + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, smem,
                           (cudaStream_t)stream>>>((const bf16*)at_workspace, cin, Kp, (const bf16*)dy, B, cout, H,
                                                   W, nullptr, 0, dx, nullptr);
    return status_of(cudaGetLastError());
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
