// C ABI of the thermal lattice Boltzmann library (declared in include/tlbm.h):
// handle lifecycle, parameter mapping, memory binding, launches of the fused
// step, and the initial-state, population transfer, macro and reduction kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/tlbm.h"
#include "dispatch.h"
#include "handle.h"

using namespace tlbm;

namespace {

constexpr int RED_BLOCKS = 1024;   // fixed reduction grid: the summation order never changes
constexpr int RED_THREADS = 256;
constexpr int RED_FIELDS = 6;      // sum u_h T, sum 1/2 rho u^2, sum rho, max u^2, bad, sum T
constexpr long long STAGE_NODES = 1ll << 21;  // FP64 staging chunk for population transfers

thread_local char g_create_error[256] = "";

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace



// ------------------------------------------------------------------ errors

static int fail(tlbm_t h, int code, const char* fmt, ...) {
    char* dst = h ? h->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(tlbm_t h, cudaError_t e, const char* what) {
    return fail(h, TLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void drop_graph(tlbm_t h);
static int set_staged(tlbm_t h, int tile_width, int stages);

// The buffer (two-buffer pull) or the order (in place: 0 natural, 1 swapped)
// of the current state, and the matching state order for the diagnostic and
// transfer kernels.
static void set_cur(tlbm_t h, int c) {
    h->cur = c;
    h->kp.state = h->aa ? (c ? 2 : 1) : 0;
}

#define TLBM_CHECK_HANDLE(h)                                   \
    do {                                                       \
        if (!(h)) return fail(nullptr, TLBM_ERR_ARG, "NULL handle"); \
        (h)->err[0] = 0;                                       \
    } while (0)

#define TLBM_CHECK_BOUND(h)                                                         \
    do {                                                                            \
        if (!(h)->mem) return fail((h), TLBM_ERR_UNBOUND, "device memory not bound"); \
    } while (0)

// ------------------------------------------------------------------ kernels

namespace {

// splitmix64 output function (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A box of nodes [x0, x0 + wx) x [y0, y0 + wy) x [z0, z0 + wz), enumerated x fastest.
struct Window {
    int x0, y0, z0, wx, wy, wz;
};

__device__ __forceinline__ void window_xyz(long long k, const Window& w, int& x, int& y, int& z) {
    x = w.x0 + (int)(k % w.wx);
    long long r = k / w.wx;
    y = w.y0 + (int)(r % w.wy);
    z = w.z0 + (int)(r / w.wy);
}

__device__ __forceinline__ void node_xyz(long long n, const Layout& L, int& x, int& y, int& z) {
    x = (int)(n % L.nx);
    long long r = n / L.nx;
    y = (int)(r % L.ny);
    z = (int)(r / L.ny);
}

// Initial state: f = w (rho = 1, u = 0), g = g_eq(T, 0) with the conductive
// profile plus seeded uniform noise.  Every pre-collision value f_i(x) is
// written where the state order p.state keeps it (pre_index).
template <int DIM, class S>
__global__ void init_kernel(S* __restrict__ buf, const KParams p, uint64_t seed, double amp) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    const Layout& L = p.L;
    const long long N = (long long)L.nx * L.ny * L.nz;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(n, L, x, y, z);
        const int c = p.heat_axis == 0 ? x : (p.heat_axis == 1 ? y : z);
        const int len = p.heat_axis == 0 ? L.nx : (p.heat_axis == 1 ? L.ny : L.nz);
        const double r = (double)(splitmix64(seed ^ splitmix64((uint64_t)n)) >> 11) * 0x1.0p-53;
        double T = __dadd_rn(p.Th, __dmul_rn(p.Tc - p.Th, __ddiv_rn((double)c + 0.5, (double)len)));
        T = __dadd_rn(T, __dmul_rn(amp, 2.0 * r - 1.0));
        double nm[LG::Q];
        for (int k = 0; k < LG::Q; ++k) nm[k] = 0.0;
        nm[0] = T;
        nm[DIM == 2 ? 3 : 4] = p.a_T * T;
        double gq[LG::Q];
        populations<LG, double>(nm, gq);
        const C scale = (C)p.scale;
        static_for<LF::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            *TLBM_DBG(p, (buf + pre_index<LF, i>(p, x, y, z)), 0, 1) = enc_f<LF, S, C>(C(0), i, scale);
        });
        S* gb = buf + (long long)LF::Q * L.plane;
        static_for<LG::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            *TLBM_DBG(p, (gb + pre_index<LG, i>(p, x, y, z)), 0, 1) = enc_g<S, C>((C)gq[i], scale);
        });
    }
}

// Initial state from given fields (warm start): f = f_eq(rho = 1, u) and
// g = g_eq(T, u) at every node, written where p.state keeps them.
template <int DIM, class S>
__global__ void init_fields_kernel(S* __restrict__ buf, const KParams p, const float* __restrict__ Tf,
                                   const float* __restrict__ uxf, const float* __restrict__ uyf,
                                   const float* __restrict__ uzf) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    const Layout& L = p.L;
    const long long N = (long long)L.nx * L.ny * L.nz;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(n, L, x, y, z);
        const double T = Tf[n];
        const double u[3] = {uxf ? (double)uxf[n] : 0.0, uyf ? (double)uyf[n] : 0.0,
                             (DIM == 3 && uzf) ? (double)uzf[n] : 0.0};
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double nm[LG::Q];
        for (int k = 0; k < LG::Q; ++k) nm[k] = 0.0;
        nm[0] = T;
        nm[1] = u[0] * T;
        nm[2] = u[1] * T;
        if (DIM == 3) nm[3] = u[2] * T;
        nm[DIM == 2 ? 3 : 4] = p.a_T * T;
        double gq[LG::Q];
        populations<LG, double>(nm, gq);
        const C scale = (C)p.scale;
        static_for<LF::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const double eu = LF::e(i, 0) * u[0] + LF::e(i, 1) * u[1] + LF::e(i, 2) * u[2];
            const double dev = (LF::w36(i) / 36.0) * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            *TLBM_DBG(p, (buf + pre_index<LF, i>(p, x, y, z)), 0, 1) = enc_f<LF, S, C>((C)dev, i, scale);
        });
        S* gb = buf + (long long)LF::Q * L.plane;
        static_for<LG::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            *TLBM_DBG(p, (gb + pre_index<LG, i>(p, x, y, z)), 0, 1) = enc_g<S, C>((C)gq[i], scale);
        });
    }
}

// Host FP64 populations (one plane, nodes [n0, n0 + cnt)) -> the state's slots.
// dev: offset storage takes flow values as deviations f_i - w_i (the exact
// FP64 image of what it stores; checkpoints), otherwise as f_i.
template <int DIM, class S>
__global__ void scatter_kernel(S* __restrict__ buf, const double* __restrict__ stage, int pop, long long n0,
                               long long cnt, const Window w, const KParams p, bool dev) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    const Layout& L = p.L;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < cnt;
         k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        window_xyz(n0 + k, w, x, y, z);
        const double v = stage[k];
        static_for<LF::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (pop == i) {
                S s;
                if constexpr (Storage<S>::offset) s = from_c<S>((C)((dev ? v : v - LF::w36(i) / 36.0) * p.scale));
                else s = (S)v;
                *TLBM_DBG(p, (buf + pre_index<LF, i>(p, x, y, z)), 0, 1) = s;
            }
        });
        static_for<LG::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (pop == LF::Q + i) {
                S s;
                if constexpr (Storage<S>::offset) s = from_c<S>((C)(v * p.scale));
                else s = (S)v;
                *TLBM_DBG(p, (buf + ((long long)LF::Q * L.plane + pre_index<LG, i>(p, x, y, z))), 0, 1) = s;
            }
        });
    }
}

// The state's slots -> canonical FP64 populations (one plane, nodes [n0, n0 + cnt)).
// dev: offset storage hands out flow deviations f_i - w_i (exact) instead.
template <int DIM, class S>
__global__ void gather_kernel(const S* __restrict__ buf, double* __restrict__ stage, int pop, long long n0,
                              long long cnt, const Window w, const KParams p, bool dev) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const Layout& L = p.L;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < cnt;
         k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        window_xyz(n0 + k, w, x, y, z);
        double v = 0.0;
        static_for<LF::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (pop == i) {
                const double raw = to_c<double>(*TLBM_DBG(p, (buf + pre_index<LF, i>(p, x, y, z)), 0, 1));
                if constexpr (Storage<S>::offset) v = (dev ? 0.0 : LF::w36(i) / 36.0) + raw * (double)p.inv_scale;
                else v = raw;
            }
        });
        static_for<LG::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            if (pop == LF::Q + i) {
                const double raw =
                    to_c<double>(*TLBM_DBG(p, (buf + ((long long)LF::Q * L.plane + pre_index<LG, i>(p, x, y, z))), 0, 1));
                if constexpr (Storage<S>::offset) v = raw * (double)p.inv_scale;
                else v = raw;
            }
        });
        stage[k] = v;
    }
}

// rho, u, T of the current state into dense caller arrays.
template <int DIM, class S, class O>
__global__ void macros_kernel(const S* __restrict__ buf, const KParams p, O* rho, O* ux, O* uy, O* uz, O* T) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const Layout& L = p.L;
    const long long N = (long long)L.nx * L.ny * L.nz;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(n, L, x, y, z);
        double f[LF::Q], g[LG::Q], r, u[3], t;
        pull_node<DIM, S, double>(buf, p, x, y, z, f, g);
        node_macros<DIM, double>(f, g, p, r, u, t);
        if (rho) rho[n] = (O)r;
        if (ux) ux[n] = (O)u[0];
        if (uy) uy[n] = (O)u[1];
        if (uz) uz[n] = (O)u[2];
        if (T) T[n] = (O)t;
    }
}

// Deterministic FP64 reduction, pass 1: each block sums a fixed node subset in
// a fixed order (per-thread serial loop over every (RED_BLOCKS * RED_THREADS)-th
// node, then a fixed warp-shuffle tree and a fixed cross-warp order) and writes
// its partials.  The node coordinates advance by the stride's (x, y, z) digits
// with carries instead of a division per node.
template <int DIM, class S>
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(const S* __restrict__ buf, const KParams p,
                                                            double* __restrict__ partials) {
    const Layout& L = p.L;
    const long long N = (long long)L.nx * L.ny * L.nz;
    double acc[RED_FIELDS] = {0, 0, 0, 0, 0, 0};
    const long long n0 = blockIdx.x * (long long)RED_THREADS + threadIdx.x;
    if (n0 < N) {
        constexpr long long STR = (long long)RED_BLOCKS * RED_THREADS;
        int x, y, z;
        node_xyz(n0, L, x, y, z);
        int sx, sy, sz;
        node_xyz(STR, L, sx, sy, sz);  // the stride in mixed radix (nx, ny, .)
        while (z < L.nz) {
            double t[5];
            node_terms<DIM, S>(buf, p, x, y, z, t);
            acc[0] += t[0];
            acc[1] += t[1];
            acc[2] += t[2];
            acc[3] = fmax(acc[3], t[3]);
            if (!isfinite(t[2]) || !isfinite(t[4]) || !isfinite(t[3])) acc[4] = 1.0;
            acc[5] += t[4];
            x += sx;
            const int cx = x >= L.nx;
            x -= cx * L.nx;
            y += sy + cx;
            const int cy = y >= L.ny;
            y -= cy * L.ny;
            z += sz + cy;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < RED_FIELDS; ++k) {
            const double o = __shfl_down_sync(0xffffffffu, acc[k], off);
            acc[k] = (k == 3 || k == 4) ? fmax(acc[k], o) : acc[k] + o;
        }
    }
    __shared__ double sm[RED_THREADS / 32][RED_FIELDS];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < RED_FIELDS; ++k) sm[w][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double out[RED_FIELDS];
        for (int k = 0; k < RED_FIELDS; ++k) out[k] = sm[0][k];
        for (int j = 1; j < RED_THREADS / 32; ++j)
            for (int k = 0; k < RED_FIELDS; ++k)
                out[k] = (k == 3 || k == 4) ? fmax(out[k], sm[j][k]) : out[k] + sm[j][k];
        for (int k = 0; k < RED_FIELDS; ++k) partials[(long long)blockIdx.x * RED_FIELDS + k] = out[k];
    }
}

// Pass 2: one block combines the RED_BLOCKS partials in a fixed tree.
__global__ void __launch_bounds__(RED_BLOCKS) reduce_final_kernel(const double* __restrict__ partials,
                                                                 double* __restrict__ out) {
    __shared__ double sm[RED_BLOCKS];
    for (int k = 0; k < RED_FIELDS; ++k) {
        sm[threadIdx.x] = partials[(long long)threadIdx.x * RED_FIELDS + k];
        __syncthreads();
        for (int s = RED_BLOCKS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s)
                sm[threadIdx.x] = (k == 3 || k == 4) ? fmax(sm[threadIdx.x], sm[threadIdx.x + s])
                                                     : sm[threadIdx.x] + sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sm[0];
        __syncthreads();
    }
}

template <int DIM, class S>
struct DiagKernels {
    static cudaError_t init(void* buf, const KParams& p, uint64_t seed, double amp, cudaStream_t s) {
        init_kernel<DIM, S><<<2048, 256, 0, s>>>((S*)buf, p, seed, amp);
        return cudaGetLastError();
    }
    static cudaError_t init_fields(void* buf, const KParams& p, const float* T, const float* ux, const float* uy,
                                   const float* uz, cudaStream_t s) {
        init_fields_kernel<DIM, S><<<2048, 256, 0, s>>>((S*)buf, p, T, ux, uy, uz);
        return cudaGetLastError();
    }
    static cudaError_t scatter(void* buf, const double* st, int pop, long long n0, long long cnt, const Window& w,
                               const KParams& p, cudaStream_t s, bool dev = false) {
        scatter_kernel<DIM, S><<<1024, 256, 0, s>>>((S*)buf, st, pop, n0, cnt, w, p, dev);
        return cudaGetLastError();
    }
    static cudaError_t gather(const void* buf, double* st, int pop, long long n0, long long cnt, const Window& w,
                              const KParams& p, cudaStream_t s, bool dev = false) {
        gather_kernel<DIM, S><<<1024, 256, 0, s>>>((const S*)buf, st, pop, n0, cnt, w, p, dev);
        return cudaGetLastError();
    }
    static cudaError_t macros(const void* buf, const KParams& p, void* r, void* ux, void* uy, void* uz, void* T,
                              int dt, cudaStream_t s) {
        if (dt == TLBM_OUT_F64)
            macros_kernel<DIM, S, double><<<2048, 256, 0, s>>>((const S*)buf, p, (double*)r, (double*)ux,
                                                               (double*)uy, (double*)uz, (double*)T);
        else
            macros_kernel<DIM, S, float><<<2048, 256, 0, s>>>((const S*)buf, p, (float*)r, (float*)ux,
                                                              (float*)uy, (float*)uz, (float*)T);
        return cudaGetLastError();
    }
    static cudaError_t reduce(const void* buf, const KParams& p, double* partials, double* out, cudaStream_t s) {
        reduce_kernel<DIM, S><<<RED_BLOCKS, RED_THREADS, 0, s>>>((const S*)buf, p, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        reduce_final_kernel<<<1, RED_BLOCKS, 0, s>>>(partials, out);
        return cudaGetLastError();
    }
};

// dispatch a diagnostic call over (dim, precision)
template <class F>
cudaError_t with_types(int dim, int prec, F&& f) {
    if (dim == 2) {
        switch (prec) {
        case TLBM_FP64: return f(DiagKernels<2, double>{});
        case TLBM_FP32: return f(DiagKernels<2, float>{});
        case TLBM_FP16_OFFSET: return f(DiagKernels<2, __half>{});
        default: return f(DiagKernels<2, __nv_bfloat16>{});
        }
    }
    switch (prec) {
    case TLBM_FP64: return f(DiagKernels<3, double>{});
    case TLBM_FP32: return f(DiagKernels<3, float>{});
    case TLBM_FP16_OFFSET: return f(DiagKernels<3, __half>{});
    default: return f(DiagKernels<3, __nv_bfloat16>{});
    }
}

}  // namespace

// ------------------------------------------------------------------ setup

extern "C" void tlbm_default_params(tlbm_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->walls = TLBM_RB;
    const double nan = std::nan("");
    p->a_T = p->nu = p->alpha = p->gbeta = nan;
    p->s_rho = p->s_e = p->s_eps = p->s_j = p->s_q = p->s_pi = p->s_m = nan;
    p->q_e = p->q_v = nan;
    p->Th = p->Tc = nan;
    p->store_scale = nan;
}

static double pick(double v, double d) { return std::isnan(v) ? d : v; }

// Default step variant per (dimension, storage): nodes per thread and block
// shape, from a sweep on GB300 at 8193^2 (2D) and 385^3 (3D).
struct VariantDefault {
    int vec, bx, by, rows;
};
static VariantDefault default_variant(int dim, int prec) {
    if (dim == 2) {
        switch (prec) {
        case TLBM_FP64: return {2, 64, 1, 1};
        case TLBM_FP32: return {4, 32, 4, 2};
        default: return {4, 32, 1, 1};
        }
    }
    switch (prec) {
    case TLBM_FP64: return {1, 32, 4, 1};
    case TLBM_FP32: return {1, 32, 2, 1};
    default: return {2, 32, 1, 1};
    }
}
static int default_vec(int dim, int prec) { return default_variant(dim, prec).vec; }

extern "C" int tlbm_create(tlbm_t* out, int nx, int ny, int nz, int lattice, double Ra, double Pr, double Ma,
                           int precision, const tlbm_params* pin) {
    g_create_error[0] = 0;
    if (!out) return fail(nullptr, TLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (lattice != TLBM_D2Q9_D2Q5 && lattice != TLBM_D3Q19_D3Q7)
        return fail(nullptr, TLBM_ERR_ARG, "unknown lattice %d", lattice);
    if (precision < TLBM_FP64 || precision > TLBM_BF16_OFFSET)
        return fail(nullptr, TLBM_ERR_UNSUPPORTED, "unknown precision %d", precision);
    const int dim = lattice == TLBM_D2Q9_D2Q5 ? 2 : 3;
    if (dim == 2) nz = 1;
    if (nx < 3 || ny < 3 || (dim == 3 && nz < 3))
        return fail(nullptr, TLBM_ERR_ARG, "grid %d x %d x %d too small (each extent >= 3)", nx, ny, nz);
    if (nx > (1 << 24) || ny > 65535 || nz > 65535 || (double)nx * ny * nz > 4e10)
        return fail(nullptr, TLBM_ERR_ARG, "grid too large (nx <= 2^24, ny and nz <= 65535)");
    if (!(Ra > 0) || !(Pr > 0) || !(Ma > 0))
        return fail(nullptr, TLBM_ERR_ARG, "Ra, Pr and Ma must be > 0");
    tlbm_params prm;
    if (pin) prm = *pin;
    else tlbm_default_params(&prm);
    if (prm.walls != TLBM_RB && prm.walls != TLBM_SIDE_HEATED)
        return fail(nullptr, TLBM_ERR_ARG, "unknown walls %d", prm.walls);
    if (prm.periodic_mask < 0 || prm.periodic_mask > 7)
        return fail(nullptr, TLBM_ERR_ARG, "periodic_mask out of range");
    if (prm.streaming != TLBM_STREAM_PULL && prm.streaming != TLBM_STREAM_INPLACE)
        return fail(nullptr, TLBM_ERR_ARG, "unknown streaming %d", prm.streaming);

    tlbm_s* h = new (std::nothrow) tlbm_s();
    if (!h) return fail(nullptr, TLBM_ERR_OOM, "host allocation failed");
    h->nx = nx; h->ny = ny; h->nz = nz; h->dim = dim; h->lattice = lattice; h->prec = precision;
    h->qf = dim == 2 ? 9 : 19;
    h->qg = dim == 2 ? 5 : 7;
    h->Ra = Ra; h->Pr = Pr; h->Ma = Ma;
    h->prm = prm;

    // free-fall scaling, Eqs. (2)-(4)
    h->prm.Th = pick(prm.Th, 0.5);
    h->prm.Tc = pick(prm.Tc, -0.5);
    const double dT = h->prm.Th - h->prm.Tc;
    h->U = prm.u_is_ma ? Ma : Ma / std::sqrt(3.0);
    h->H = dim == 2 ? ny : nz;
    h->nu = pick(prm.nu, h->U * h->H * std::sqrt(Pr / Ra));
    h->alpha = pick(prm.alpha, h->U * h->H / std::sqrt(Pr * Ra));
    h->gbeta = pick(prm.gbeta, h->U * h->U / (h->H * dT));
    h->a_T = pick(prm.a_T, dim == 2 ? -2.0 / 3.0 : -0.75);
    h->omega = dim == 2 ? (4.0 + h->a_T) / 10.0 : (6.0 + h->a_T) / 21.0;
    if (!(3.0 * h->nu > 1e-6) || !(h->alpha > 0) || !(h->omega > 0) || !(dT != 0)) {
        delete h;
        return fail(nullptr, TLBM_ERR_ARG, "relaxation time out of range (3 nu = %g, alpha = %g)", 3.0 * h->nu,
                    h->alpha);
    }
    const double snu = 1.0 / (3.0 * h->nu + 0.5);
    const double sq = 8.0 * (2.0 - snu) / (8.0 - snu);
    const double s_rho = pick(prm.s_rho, 1.0), s_e = pick(prm.s_e, snu), s_eps = pick(prm.s_eps, snu);
    const double s_j = pick(prm.s_j, 1.0), s_q = pick(prm.s_q, sq), s_pi = pick(prm.s_pi, snu);
    const double s_m = pick(prm.s_m, sq);
    if (dim == 2) {
        const double S[9] = {s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, snu, snu};
        memcpy(h->S, S, sizeof(S));
    } else {
        const double S[19] = {s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_j, s_q, snu,
                              s_pi,  snu, s_pi,  snu, snu, snu, s_m, s_m, s_m};
        memcpy(h->S, S, sizeof(S));
    }
    const double qj = 1.0 / (h->alpha / h->omega + 0.5);
    const double qeven = 1.0 / (0.5 + 0.25 / (1.0 / qj - 0.5));
    const double q_e = pick(prm.q_e, qeven), q_v = pick(prm.q_v, qeven);
    if (dim == 2) {
        const double Q[5] = {1.0, qj, qj, q_e, q_v};
        memcpy(h->Q, Q, sizeof(Q));
    } else {
        const double Q[7] = {1.0, qj, qj, qj, q_e, q_v, q_v};
        memcpy(h->Q, Q, sizeof(Q));
    }

    // device layout
    KParams& kp = h->kp;
    memset(&kp, 0, sizeof(kp));
    kp.L.nx = nx; kp.L.ny = ny; kp.L.nz = nz; kp.L.dim = dim;
    kp.L.zg = dim == 3 ? 1 : 0;
    kp.L.P = (int)align_up((size_t)nx + 16, ROW_ALIGN);
    const long long rows = (long long)(ny + 2) * (dim == 3 ? nz + 2 : 1);
    kp.L.plane = (long long)align_up((size_t)(SLOT_OFF + rows * kp.L.P + TAIL), 64);
    kp.periodic = prm.periodic_mask;
    kp.grav_axis = dim - 1;
    kp.heat_axis = prm.walls == TLBM_RB ? dim - 1 : 0;
    // two-relaxation-time form applies when the even / odd non-conserved rates coincide
    {
        const int ev2[] = {1, 2, 7, 8}, od2[] = {4, 6};
        const int ev3[] = {1, 2, 9, 10, 11, 12, 13, 14, 15}, od3[] = {4, 6, 8, 16, 17, 18};
        const int* ev = dim == 2 ? ev2 : ev3;
        const int* od = dim == 2 ? od2 : od3;
        const int nev = dim == 2 ? 4 : 9, nod = dim == 2 ? 2 : 6;
        bool ok = true;
        for (int k = 1; k < nev; ++k) ok = ok && h->S[ev[k]] == h->S[ev[0]];
        for (int k = 1; k < nod; ++k) ok = ok && h->S[od[k]] == h->S[od[0]];
        const int tev = dim == 2 ? 3 : 4;  // first even non-conserved thermal moment
        for (int k = tev + 1; k < h->qg; ++k) ok = ok && h->Q[k] == h->Q[tev];
        for (int k = 2; k < tev; ++k) ok = ok && h->Q[k] == h->Q[1];
        kp.trt = ok ? 1 : 0;
        kp.sp = h->S[ev[0]];
        kp.sm = h->S[od[0]];
        kp.shp = 1.0 - 0.5 * kp.sp;
        kp.shm = 1.0 - 0.5 * kp.sm;
        kp.qp = h->Q[tev];
        kp.qm = h->Q[1];
        kp.spf = (float)kp.sp; kp.smf = (float)kp.sm; kp.shpf = (float)kp.shp; kp.shmf = (float)kp.shm;
        kp.qpf = (float)kp.qp; kp.qmf = (float)kp.qm;
    }
    h->trt = kp.trt;
    {
        // per-population pull / store offsets (elements, relative to a node's own
        // slot in plane 0): plane j, shifted back by the population's e_y, e_z
        // (the x-shift is taken by the kernel's loads)
        const long long P = kp.L.P, RP = (long long)(ny + 2) * kp.L.P;
        const int qf = h->qf;
        for (int j = 0; j < h->qf + h->qg; ++j) {
            int ey, ez;
            if (dim == 2) {
                ey = j < qf ? D2Q9::e(j, 1) : D2Q5::e(j - qf, 1);
                ez = 0;
            } else {
                ey = j < qf ? D3Q19::e(j, 1) : D3Q7::e(j - qf, 1);
                ez = j < qf ? D3Q19::e(j, 2) : D3Q7::e(j - qf, 2);
            }
            kp.soff[j] = (int)((long long)j * kp.L.plane);
            kp.loff[j] = (int)((long long)j * kp.L.plane - ey * P - ez * RP);
        }
        kp.plane32 = (int)kp.L.plane;
        kp.rp = (int)RP;
    }
    h->wait_ns = TILE_WAIT_NS;
    h->vec = default_variant(dim, precision).vec;
    h->bx = default_variant(dim, precision).bx;
    h->by = default_variant(dim, precision).by;
    h->rows = default_variant(dim, precision).rows;
    kp.xmax_load = kp.L.P - h->vec;
    kp.gbeta = h->gbeta; kp.omega = h->omega; kp.Th = h->prm.Th; kp.Tc = h->prm.Tc; kp.a_T = h->a_T;
    for (int a = 0; a < 3; ++a) {
        kp.body[a] = prm.body_force[a];
        kp.bodyf[a] = (float)prm.body_force[a];
    }
    for (int k = 0; k < MAXQ; ++k) {
        const double s = k < h->qf ? h->S[k] : 0.0;
        kp.S[k] = s;
        kp.Sh[k] = 1.0 - 0.5 * s;
        kp.Sf[k] = (float)s;
        kp.Shf[k] = (float)(1.0 - 0.5 * s);
    }
    for (int k = 0; k < 7; ++k) {
        const double q = k < h->qg ? h->Q[k] : 0.0;
        kp.Q[k] = q;
        kp.Qf[k] = (float)q;
    }
    kp.gbetaf = (float)h->gbeta; kp.omegaf = (float)h->omega; kp.Thf = (float)h->prm.Th;
    kp.Tcf = (float)h->prm.Tc; kp.a_Tf = (float)h->a_T;
    double scale = pick(prm.store_scale, precision == TLBM_FP16_OFFSET ? 1024.0 : 1.0);
    if (precision <= TLBM_FP32) scale = 1.0;
    int scale_exp = 0;
    if (!(scale > 0) || std::frexp(scale, &scale_exp) != 0.5) {
        delete h;
        return fail(nullptr, TLBM_ERR_ARG, "store_scale must be a power of two");
    }
    kp.scale = (float)scale;
    kp.inv_scale = (float)(1.0 / scale);
    {
        // FP32 constants of the two-relaxation-time collision (KParams::tf):
        // the in-kernel expressions, one operation per statement, so that the
        // host compiler forms each exactly as the kernel does
        const float sc = kp.scale;
        const int w0i = dim == 2 ? D2Q9::w36(0) : D3Q19::w36(0);
        const int wai = dim == 2 ? D2Q9::w36(1) : D3Q19::w36(1);
        const int wbi = dim == 2 ? D2Q9::w36(D2Q9::Q - 1) : D3Q19::w36(D3Q19::Q - 1);
        const float w0 = (float)w0i / 36.0f, wa = (float)wai / 36.0f, wb = (float)wbi / 36.0f;
        const float sp = kp.spf, sm = kp.smf, shp = kp.shpf, shm = kp.shmf, qp = kp.qpf, qm = kp.qmf;
        auto& t = kp.tf;
        t.m3shp = -3.0f * shp;
        t.r1 = 4.5f * sp;
        t.r3 = 3.0f * sm;
        const float spm = sp + sm;        // (sp + sm) / 2 and (sm - sp) / 2 are exact halvings
        t.c1 = 1.0f - 0.5f * spm;
        const float dsm = sm - sp;
        t.c2 = 0.5f * dsm;
        t.omsp = 1.0f - sp;
        t.w0s = w0 * sc;                  // sc is a power of two: exact
        t.was = wa * sc;
        t.wbs = wb * sc;
        const float s9 = 9.0f * shp, s3 = 3.0f * shm;
        t.f9a = s9 * t.was;
        t.f9b = s9 * t.wbs;
        t.f3a = s3 * t.was;
        t.f3b = s3 * t.wbs;
        const float wT = 0.5f * kp.omegaf;
        const float qpm = qp + qm;
        t.t1 = 1.0f - 0.5f * qpm;
        const float dq = qm - qp;
        t.t2 = 0.5f * dq;
        t.qpwT = qp * wT;
        t.hqm = 0.5f * qm;
        t.omqp = 1.0f - qp;
        const float rest = std::fma(-(float)(h->qg - 1), wT, 1.0f);
        t.g0c = qp * rest;
    }

    if ((long long)(h->qf + h->qg) * kp.L.plane + kp.L.P >= (1ll << 31)) {
        delete h;
        return fail(nullptr, TLBM_ERR_ARG, "cell too large: a population set must hold fewer than 2^31 elements");
    }
    h->elem = precision == TLBM_FP64 ? 8 : (precision == TLBM_FP32 ? 4 : 2);
    h->popset_bytes = align_up((size_t)(h->qf + h->qg) * (size_t)kp.L.plane * h->elem, 256);
    h->aa = prm.streaming == TLBM_STREAM_INPLACE;
    h->nbuf = h->aa ? 1 : 2;
    if (h->aa) {
        h->rows = 1;  // the in-place halves have no multi-row variant
        if (dim == 2 && precision == TLBM_FP32) h->by = 1;  // 57.4 vs 56.0 GLUPS with 32 x 4 at 8193^2
    }
    h->red_off = h->nbuf * h->popset_bytes;
    h->res_off = h->red_off + align_up((size_t)RED_BLOCKS * RED_FIELDS * sizeof(double), 256);
    h->status_off = h->res_off + 128;
    h->stage_off = h->res_off + 256;
    const long long N = (long long)nx * ny * nz;
    h->total_bytes = h->stage_off + align_up((size_t)std::min<long long>(N, STAGE_NODES) * sizeof(double), 256);
    h->stream = nullptr;
    set_cur(h, 0);
    h->t = 0;
    h->graph_steps = 16;
    *out = h;
    return TLBM_OK;
}

extern "C" int tlbm_required_bytes(tlbm_t h, size_t* bytes) {
    TLBM_CHECK_HANDLE(h);
    if (!bytes) return fail(h, TLBM_ERR_ARG, "bytes is NULL");
    *bytes = h->total_bytes;
    return TLBM_OK;
}

extern "C" int tlbm_bind_memory(tlbm_t h, void* dev_ptr, size_t bytes) {
    TLBM_CHECK_HANDLE(h);
    if (!dev_ptr) return fail(h, TLBM_ERR_ARG, "dev_ptr is NULL");
    if (((uintptr_t)dev_ptr) % 256) return fail(h, TLBM_ERR_ARG, "dev_ptr must be 256-byte aligned");
    if (bytes < h->total_bytes)
        return fail(h, TLBM_ERR_OOM, "bound block has %zu bytes, %zu needed", bytes, h->total_bytes);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, dev_ptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaPointerGetAttributes");
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(h, TLBM_ERR_ARG, "dev_ptr is not device memory");
    // the staged kernel's status word starts cleared
    e = cudaMemset((char*)dev_ptr + h->status_off, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset");
    drop_graph(h);
    h->mem = (char*)dev_ptr;
    h->mem_bytes = bytes;
    h->buf[0] = h->mem;
    h->buf[1] = h->aa ? h->mem : h->mem + h->popset_bytes;
#ifdef TLBM_DEBUG_BOUNDS
    h->kp.dbg_lo = h->mem;
    h->kp.dbg_hi = h->mem + h->nbuf * h->popset_bytes;
    h->kp.dbg_count = (unsigned long long*)(h->mem + h->status_off + 64);
    e = cudaMemset(h->kp.dbg_count, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset");
#endif
    set_cur(h, 0);
    // FP16/BF16 storage with two-relaxation-time rates defaults to the
    // shared-memory staged kernel: in 2D 512-node tiles with the stages chosen
    // as above (2 stages and three blocks per SM on GB300, the fastest there),
    // in 3D whole rows with 2 stages and two blocks per SM (385^3 FP16: 46.5
    // GLUPS against 46.3 with 3 stages and 44.4 for the register kernel); the
    // register kernel stays if the device cannot host it
    if (!h->variant_chosen && !h->aa && (h->prec == TLBM_FP16_OFFSET || h->prec == TLBM_BF16_OFFSET) &&
        h->kp.trt && set_staged(h, 0, h->dim == 3 ? 2 : 0) != TLBM_OK) {
        h->staged = 0;
        h->err[0] = 0;
    }
    return TLBM_OK;
}

extern "C" int tlbm_set_stream(tlbm_t h, void* s) {
    TLBM_CHECK_HANDLE(h);
    h->stream = (cudaStream_t)s;
    return TLBM_OK;
}

extern "C" int tlbm_init(tlbm_t h, uint64_t seed, double noise_amp) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!std::isfinite(noise_amp) || noise_amp < 0) return fail(h, TLBM_ERR_ARG, "noise_amp must be finite, >= 0");
    cudaError_t e = cudaMemsetAsync(h->mem, 0, h->nbuf * h->popset_bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    e = cudaMemsetAsync(h->mem + h->status_off, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    set_cur(h, 0);
    e = with_types(h->dim, h->prec, [&](auto K) { return decltype(K)::init(h->buf[0], h->kp, seed, noise_amp, h->stream); });
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    h->launches += 1;
    h->t = 0;
    return TLBM_OK;
}

extern "C" int tlbm_init_fields(tlbm_t h, const float* T, const float* ux, const float* uy, const float* uz) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!T) return fail(h, TLBM_ERR_ARG, "T is required");
    cudaError_t e = cudaMemsetAsync(h->mem, 0, h->nbuf * h->popset_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->mem + h->status_off, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    set_cur(h, 0);
    e = with_types(h->dim, h->prec, [&](auto K) {
        return decltype(K)::init_fields(h->buf[0], h->kp, T, ux, uy, uz, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "init_fields kernel");
    h->launches += 1;
    h->t = 0;
    return TLBM_OK;
}

// Launch one step reading buffer `parity` and writing the other, on stream s
// (no bookkeeping).
static cudaError_t launch_step_raw(tlbm_t h, int parity, cudaStream_t s) {
    const KParams& kp = h->kp;
    const void* src = h->buf[parity];
    void* dst = h->buf[parity ^ 1];
    if (h->staged) {
        StagedInfo si;
        si.tw = h->staged_tw;
        si.tiles_per_row = (h->nx + si.tw - 1) / si.tw;
        si.tiles = h->ny * h->nz * si.tiles_per_row;
        si.stages = h->staged_stages;
        si.status = (int*)(h->mem + h->status_off);
        si.wait_ns = h->wait_ns;
        return launch_staged(h->dim, h->prec, h->staged_nc, src, dst, kp, si, h->staged_grid, h->staged_smem, s);
    }
    const int vec = h->vec;
    const int bx = h->bx, by = h->by, rows = h->rows;
    const int threads_x = (h->nx + vec - 1) / vec;
    dim3 block(bx, by, 1);
    dim3 grid((threads_x + bx - 1) / bx, (h->ny + by * rows - 1) / (by * rows), h->dim == 3 ? h->nz : 1);
    // in place: natural order -> the AA_EVEN half, swapped -> AA_ODD, one buffer
    if (h->aa) return launch_step(h->dim, h->prec, vec, h->trt != 0, parity ? -AA_ODD : -AA_EVEN, src, h->buf[0], kp,
                                  grid, block, s);
    return launch_step(h->dim, h->prec, vec, h->trt != 0, rows, src, dst, kp, grid, block, s);
}

static void drop_graph(tlbm_t h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

// Capture graph_steps steps starting from buffer 0 into a CUDA graph (on a
// private stream; the graph is replayed on the handle's stream).
static int build_graph(tlbm_t h) {
    drop_graph(h);
    cudaError_t e = cudaSuccess;
    if (!h->capture_stream) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
    e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < h->graph_steps && le == cudaSuccess; ++k) le = launch_step_raw(h, k & 1, h->capture_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->capture_stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, le != cudaSuccess ? le : e, "step graph capture");
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    return TLBM_OK;
}

static cudaError_t launch_one_step(tlbm_t h) {
    cudaError_t e = launch_step_raw(h, h->cur, h->stream);
    if (e == cudaSuccess) {
        set_cur(h, h->cur ^ 1);
        h->t += 1;
        h->launches += 1;
    }
    return e;
}

extern "C" int tlbm_step(tlbm_t h, int64_t n) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (n < 0) return fail(h, TLBM_ERR_ARG, "n must be >= 0");
    while (n > 0) {
        if (h->graph_steps >= 2 && h->cur == 0 && n >= h->graph_steps) {
            if (!h->graph) {
                int rc = build_graph(h);
                if (rc != TLBM_OK) return rc;
            }
            cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            h->t += h->graph_steps;  // an even number of steps: the state is back in buffer 0
            h->launches += h->graph_steps;
            n -= h->graph_steps;
        } else {
            cudaError_t e = launch_one_step(h);
            if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
            n -= 1;
        }
    }
    return TLBM_OK;
}

extern "C" int tlbm_set_graph(tlbm_t h, int steps) {
    TLBM_CHECK_HANDLE(h);
    if (steps < 0 || steps % 2 || steps > 4096) return fail(h, TLBM_ERR_ARG, "steps must be even, in [0, 4096]");
    drop_graph(h);
    h->graph_steps = steps;
    return TLBM_OK;
}

extern "C" int tlbm_macros(tlbm_t h, void* rho, void* ux, void* uy, void* uz, void* T, int out_dtype) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (out_dtype != TLBM_OUT_F64 && out_dtype != TLBM_OUT_F32) return fail(h, TLBM_ERR_ARG, "bad out_dtype");
    if (h->dim == 2) uz = nullptr;
    cudaError_t e = with_types(h->dim, h->prec, [&](auto K) {
        return decltype(K)::macros(h->buf[h->cur], h->kp, rho, ux, uy, uz, T, out_dtype, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "macros kernel");
    h->launches += 1;
    return TLBM_OK;
}

// runs the two-pass reduction and copies the six results to the host
static int run_reduce(tlbm_t h, double* res) {
    double* partials = (double*)(h->mem + h->red_off);
    double* out = (double*)(h->mem + h->res_off);
    cudaError_t e = with_types(h->dim, h->prec, [&](auto K) {
        return decltype(K)::reduce(h->buf[h->cur], h->kp, partials, out, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction kernel");
    h->launches += 2;
    e = cudaMemcpyAsync(res, out, RED_FIELDS * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
    int status = 0;
    e = cudaMemcpyAsync(&status, h->mem + h->status_off, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    if (status) return fail(h, TLBM_ERR_TIMEOUT, "a staged step gave up waiting for its copies");
    return TLBM_OK;
}

// the reduction found a non-finite value or |u| > 0.5 (|u|^2 > 0.25)
static bool reduce_diverged(const double* r) { return r[4] != 0.0 || !(r[3] <= 0.25); }

extern "C" int tlbm_nusselt(tlbm_t h, double* nu) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!nu) return fail(h, TLBM_ERR_ARG, "nu is NULL");
    double r[RED_FIELDS];
    int rc = run_reduce(h, r);
    if (rc) return rc;
    const double N = (double)h->nx * h->ny * h->nz;
    const int ax = h->kp.heat_axis;
    const double L = ax == 0 ? h->nx : (ax == 1 ? h->ny : h->nz);
    *nu = 1.0 + L * (r[0] / N) / (h->alpha * (h->prm.Th - h->prm.Tc));
    if (reduce_diverged(r)) return fail(h, TLBM_ERR_DIVERGED, "the state has diverged (the value is written)");
    return TLBM_OK;
}

extern "C" int tlbm_energy(tlbm_t h, double* ekin, double* mass) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    double r[RED_FIELDS];
    int rc = run_reduce(h, r);
    if (rc) return rc;
    if (ekin) *ekin = r[1];
    if (mass) *mass = r[2];
    if (reduce_diverged(r)) return fail(h, TLBM_ERR_DIVERGED, "the state has diverged (the values are written)");
    return TLBM_OK;
}

extern "C" int tlbm_status(tlbm_t h, int* diverged, int64_t* step) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    double r[RED_FIELDS];
    int rc = run_reduce(h, r);
    if (rc) return rc;
    if (diverged) *diverged = reduce_diverged(r) ? 1 : 0;
    if (step) *step = h->t;
    return TLBM_OK;
}

static int get_window(tlbm_t h, const Window& w, double* host_f, double* host_g) {
    const long long N = (long long)w.wx * w.wy * w.wz;
    double* stage = (double*)(h->mem + h->stage_off);
    for (int pop = 0; pop < h->qf + h->qg; ++pop) {
        double* dst = pop < h->qf ? (host_f ? host_f + (long long)pop * N : nullptr)
                                  : (host_g ? host_g + (long long)(pop - h->qf) * N : nullptr);
        if (!dst) continue;
        for (long long n0 = 0; n0 < N; n0 += STAGE_NODES) {
            const long long cnt = std::min(STAGE_NODES, N - n0);
            cudaError_t e = with_types(h->dim, h->prec, [&](auto K) {
                return decltype(K)::gather(h->buf[h->cur], stage, pop, n0, cnt, w, h->kp, h->stream);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "gather kernel");
            h->launches += 1;
            e = cudaMemcpyAsync(dst + n0, stage, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync D2H");
            e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        }
    }
    return TLBM_OK;
}

extern "C" int tlbm_get_populations(tlbm_t h, double* host_f, double* host_g) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    const Window w = {0, 0, 0, h->nx, h->ny, h->nz};
    return get_window(h, w, host_f, host_g);
}

extern "C" int tlbm_get_populations_window(tlbm_t h, int x0, int y0, int z0, int wx, int wy, int wz,
                                           double* host_f, double* host_g) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (h->dim == 2) {
        z0 = 0;
        wz = 1;
    }
    if (x0 < 0 || y0 < 0 || z0 < 0 || wx < 1 || wy < 1 || wz < 1 || x0 + wx > h->nx || y0 + wy > h->ny ||
        z0 + wz > h->nz)
        return fail(h, TLBM_ERR_ARG, "window out of the cell");
    const Window w = {x0, y0, z0, wx, wy, wz};
    return get_window(h, w, host_f, host_g);
}

// Replace the state by FP64 populations delivered chunk by chunk: src(pop, n0,
// cnt, chunk) points chunk at nodes n0 .. n0 + cnt of population pop (flow
// planes first) and returns TLBM_OK or an error code.  reuse: src hands out
// one host buffer again and again, so each chunk's copy must finish before the
// next call.  Synchronises.
template <class Src>
static int put_state(tlbm_t h, Src src, bool reuse, bool dev = false) {
    const long long N = (long long)h->nx * h->ny * h->nz;
    const Window full = {0, 0, 0, h->nx, h->ny, h->nz};
    double* stage = (double*)(h->mem + h->stage_off);
    cudaError_t e = cudaMemsetAsync(h->mem, 0, h->nbuf * h->popset_bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    e = cudaMemsetAsync(h->mem + h->status_off, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    set_cur(h, 0);
    for (int pop = 0; pop < h->qf + h->qg; ++pop) {
        for (long long n0 = 0; n0 < N; n0 += STAGE_NODES) {
            const long long cnt = std::min(STAGE_NODES, N - n0);
            const double* chunk = nullptr;
            const int rc = src(pop, n0, cnt, chunk);
            if (rc != TLBM_OK) return rc;
            e = cudaMemcpyAsync(stage, chunk, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync H2D");
            e = with_types(h->dim, h->prec, [&](auto K) {
                return decltype(K)::scatter(h->buf[0], stage, pop, n0, cnt, full, h->kp, h->stream, dev);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "scatter kernel");
            h->launches += 1;
            if (reuse) {
                e = cudaStreamSynchronize(h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
            }
        }
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    h->t = 0;
    return TLBM_OK;
}

extern "C" int tlbm_set_populations(tlbm_t h, const double* host_f, const double* host_g) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!host_f || !host_g) return fail(h, TLBM_ERR_ARG, "host_f and host_g are required");
    const long long N = (long long)h->nx * h->ny * h->nz;
    return put_state(h, [&](int pop, long long n0, long long, const double*& chunk) {
        chunk = (pop < h->qf ? host_f + (long long)pop * N : host_g + (long long)(pop - h->qf) * N) + n0;
        return (int)TLBM_OK;
    }, false);
}

// ------------------------------------------------------------------ checkpoint files

namespace {
// File header of tlbm_save: native byte order, checked by `order`.
struct CkptHeader {
    char magic[8];          // "TLBMCKP1"
    uint32_t order;         // 0x01020304 as written
    int32_t version;        // 1
    int32_t lattice, nx, ny, nz, precision, walls, periodic_mask, nderived;
    int32_t flow_dev;       // 1: flow planes hold f_i - w_i (offset storage), 0: f_i
    int32_t pad;
    double Ra, Pr, Ma, Th, Tc, scale;
    double body[3];
    double derived[7 + MAXQ + 7];  // tlbm_derived: U, H, nu, alpha, gbeta, a_T, omega, S, Q
    int64_t t;              // steps taken since the initial state
    int64_t nodes;          // nx * ny * nz
};
}  // namespace

static void ckpt_fill(tlbm_t h, CkptHeader& c) {
    memset(&c, 0, sizeof(c));
    memcpy(c.magic, "TLBMCKP1", 8);
    c.order = 0x01020304u;
    c.version = 1;
    c.lattice = h->lattice;
    c.nx = h->nx;
    c.ny = h->ny;
    c.nz = h->nz;
    c.precision = h->prec;
    c.walls = h->prm.walls;
    c.periodic_mask = h->prm.periodic_mask;
    c.Ra = h->Ra;
    c.Pr = h->Pr;
    c.Ma = h->Ma;
    c.Th = h->prm.Th;
    c.Tc = h->prm.Tc;
    c.scale = h->kp.scale;
    for (int a = 0; a < 3; ++a) c.body[a] = h->prm.body_force[a];
    int n = 0;
    tlbm_derived(h, c.derived, 7 + MAXQ + 7, &n);
    c.nderived = n;
    c.flow_dev = h->prec == TLBM_FP64 ? 0 : 1;  // offset storage (FP32, FP16, BF16)
    c.t = h->t;
    c.nodes = (int64_t)h->nx * h->ny * h->nz;
}

extern "C" int tlbm_save(tlbm_t h, const char* path) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!path) return fail(h, TLBM_ERR_ARG, "path is NULL");
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(h, TLBM_ERR_ARG, "cannot open %s for writing", path);
    CkptHeader c;
    ckpt_fill(h, c);
    int rc = TLBM_OK;
    if (fwrite(&c, sizeof(c), 1, fp) != 1) rc = fail(h, TLBM_ERR_ARG, "write to %s failed", path);
    const long long N = c.nodes;
    const Window full = {0, 0, 0, h->nx, h->ny, h->nz};
    double* stage = (double*)(h->mem + h->stage_off);
    double* buf = rc == TLBM_OK ? (double*)malloc((size_t)std::min(STAGE_NODES, N) * sizeof(double)) : nullptr;
    if (rc == TLBM_OK && !buf) rc = fail(h, TLBM_ERR_OOM, "host buffer");
    for (int pop = 0; rc == TLBM_OK && pop < h->qf + h->qg; ++pop) {
        for (long long n0 = 0; rc == TLBM_OK && n0 < N; n0 += STAGE_NODES) {
            const long long cnt = std::min(STAGE_NODES, N - n0);
            cudaError_t e = with_types(h->dim, h->prec, [&](auto K) {
                return decltype(K)::gather(h->buf[h->cur], stage, pop, n0, cnt, full, h->kp, h->stream, true);
            });
            h->launches += 1;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(buf, stage, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) rc = cuda_fail(h, e, "checkpoint gather");
            else if (fwrite(buf, sizeof(double), (size_t)cnt, fp) != (size_t)cnt)
                rc = fail(h, TLBM_ERR_ARG, "write to %s failed", path);
        }
    }
    free(buf);
    if (fclose(fp) != 0 && rc == TLBM_OK) rc = fail(h, TLBM_ERR_ARG, "closing %s failed", path);
    return rc;
}

extern "C" int tlbm_load(tlbm_t h, const char* path) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!path) return fail(h, TLBM_ERR_ARG, "path is NULL");
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(h, TLBM_ERR_ARG, "cannot open %s", path);
    CkptHeader c, mine;
    ckpt_fill(h, mine);
    int rc = TLBM_OK;
    if (fread(&c, sizeof(c), 1, fp) != 1 || memcmp(c.magic, "TLBMCKP1", 8) != 0 || c.order != 0x01020304u ||
        c.version != 1)
        rc = fail(h, TLBM_ERR_ARG, "%s is not a checkpoint of this format", path);
    else if (c.lattice != mine.lattice || c.nx != mine.nx || c.ny != mine.ny || c.nz != mine.nz ||
             c.precision != mine.precision)
        rc = fail(h, TLBM_ERR_ARG, "checkpoint lattice / size / storage differ from the handle's");
    else if (c.walls != mine.walls || c.periodic_mask != mine.periodic_mask || c.nderived != mine.nderived ||
             c.flow_dev != mine.flow_dev ||
             memcmp(&c.Ra, &mine.Ra, offsetof(CkptHeader, t) - offsetof(CkptHeader, Ra)) != 0)
        rc = fail(h, TLBM_ERR_ARG, "checkpoint parameters differ from the handle's");
    const long long N = c.nodes;
    double* buf = rc == TLBM_OK ? (double*)malloc((size_t)std::min(STAGE_NODES, N) * sizeof(double)) : nullptr;
    if (rc == TLBM_OK && !buf) rc = fail(h, TLBM_ERR_OOM, "host buffer");
    if (rc == TLBM_OK) {
        rc = put_state(h, [&](int, long long, long long cnt, const double*& chunk) {
            if (fread(buf, sizeof(double), (size_t)cnt, fp) != (size_t)cnt)
                return fail(h, TLBM_ERR_ARG, "%s is shorter than its header says", path);
            chunk = buf;
            return (int)TLBM_OK;
        }, true, true);
        if (rc == TLBM_OK) {
            char extra;
            if (fread(&extra, 1, 1, fp) != 0) rc = fail(h, TLBM_ERR_ARG, "%s is longer than its header says", path);
        }
        if (rc == TLBM_OK) {
            h->t = c.t;
            // 16-bit storage: the step counter the time steps keep in word 0 of
            // the current buffer (their stochastic rounding salt), as the
            // uninterrupted run had it
            if (h->elem == 2) {
                const uint32_t t32 = (uint32_t)c.t;
                cudaError_t e = cudaMemcpyAsync(h->buf[0], &t32, sizeof(t32), cudaMemcpyHostToDevice, h->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                if (e != cudaSuccess) rc = cuda_fail(h, e, "cudaMemcpyAsync (step counter)");
            }
        }
    }
    free(buf);
    fclose(fp);
    return rc;
}

extern "C" int tlbm_set_variant(tlbm_t h, int vec, int form, int block_x, int block_y, int rows) {
    TLBM_CHECK_HANDLE(h);
    const int v = vec > 0 ? vec : default_vec(h->dim, h->prec);
    if (form < 0 || form > 2) return fail(h, TLBM_ERR_ARG, "form must be 0 (auto), 1 (MRT) or 2 (TRT)");
    if (form == 2 && !h->kp.trt)
        return fail(h, TLBM_ERR_ARG, "the relaxation rates are not of two-relaxation-time form");
    const int trt = form == 1 ? 0 : h->kp.trt;
    const int bx = block_x > 0 ? block_x : default_variant(h->dim, h->prec).bx;
    const int by = block_y > 0 ? block_y : default_variant(h->dim, h->prec).by;
    if (bx % 32 || bx * by > 1024) return fail(h, TLBM_ERR_ARG, "block_x must be a multiple of 32, bx*by <= 1024");
    const int nr = rows > 0 ? rows : 1;
    if (h->aa && nr != 1) return fail(h, TLBM_ERR_UNSUPPORTED, "in-place streaming has no multi-row variant");
    // the in-place scheme alternates two kernels; both must exist
    const int kinds[2] = {h->aa ? -AA_EVEN : nr, h->aa ? -AA_ODD : nr};
    for (int kind : kinds) {
        if (!step_variant_available(h->dim, h->prec, v, trt != 0, kind))
            return fail(h, TLBM_ERR_UNSUPPORTED, "step variant (vec %d, %s, %d rows%s) not built", v,
                        trt ? "TRT" : "MRT", nr, h->aa ? ", in place" : "");
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, step_function(h->dim, h->prec, v, trt != 0, kind));
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncGetAttributes");
        if (bx * by > fa.maxThreadsPerBlock)
            return fail(h, TLBM_ERR_ARG, "block of %d threads exceeds the variant's limit of %d", bx * by,
                        fa.maxThreadsPerBlock);
    }
    h->vec = v;
    h->trt = trt;
    h->bx = bx;
    h->by = by;
    h->rows = nr;
    h->staged = 0;
    h->variant_chosen = 1;
    h->kp.xmax_load = h->kp.L.P - v;
    drop_graph(h);
    return TLBM_OK;
}

static int set_staged(tlbm_t h, int tile_width, int stages) {
    if (h->aa) return fail(h, TLBM_ERR_UNSUPPORTED, "the staged kernel uses two buffers (no in-place variant)");
    if (h->prec == TLBM_FP64) return fail(h, TLBM_ERR_UNSUPPORTED, "the staged kernel has no FP64 variant");
    if (!h->kp.trt) return fail(h, TLBM_ERR_UNSUPPORTED, "the staged kernel needs two-relaxation-time rates");
    const int A = 16 / (int)h->elem;
    const int nx_a = (h->nx + A - 1) / A * A;
    // default: whole rows up to the widest tile (512 nodes in 2D, 448 in 3D),
    // else segments of that width
    const int twmax = h->dim == 3 ? 448 : 512;
    int tw = tile_width > 0 ? tile_width : std::min(twmax, nx_a);
    if (tw % A || tw < A || tw > twmax)
        return fail(h, TLBM_ERR_ARG, "tile_width must be a multiple of %d in [%d, %d]", A, A, twmax);
    if (tw > nx_a) tw = nx_a;
    // consumer warps (one pair of nodes per thread): 4 for tiles up to 256
    // nodes, else 8 in 2D and 7 in 3D
    const int nc = tw > 256 ? (h->dim == 3 ? 7 : 8) : 4;
    const int lw = 64 * nc + 2 * A;   // shared row length per population (elements)
    const size_t stage_bytes = (size_t)(h->qf + h->qg) * lw * h->elem;
    const void* fn = staged_function(h->dim, h->prec, nc);
    if (!fn) return fail(h, TLBM_ERR_UNSUPPORTED, "staged kernel not built for this precision");
    int dev = 0, optin = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceGetAttribute");
    // allow the device's full opt-in shared memory for this kernel, so that
    // handles with different tile shapes can share it
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute (shared memory size)");
    const int threads = 32 * (nc + 1);
    int ns = stages;
    if (ns <= 0) {
        // the most tiles in flight per SM (blocks per SM x stages) up to six,
        // more blocks first (else the fewest stages that fit): on GB300 2 x 3
        // was best for 96-register consumers, 3 x 2 for 72-register ones, and
        // more in flight was slower
        int first = 0, best_in = 0, best_b = 0;
        for (int k = 2; k <= TILE_MAX_STAGES; ++k) {
            int b = 0;
            const size_t sm = 512 + (size_t)k * stage_bytes;
            if (sm > (size_t)optin) break;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, sm);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (b < 1) break;
            if (!first) first = k;
            const int in = b * k;
            if (in <= 6 && (in > best_in || (in == best_in && b > best_b))) {
                ns = k;
                best_in = in;
                best_b = b;
            }
        }
        if (ns == 0) ns = first;
        if (ns == 0) return fail(h, TLBM_ERR_ARG, "two stages of %zu bytes do not fit in shared memory", stage_bytes);
    }
    if (ns < 2 || ns > TILE_MAX_STAGES) return fail(h, TLBM_ERR_ARG, "stages must be in [2, %d]", TILE_MAX_STAGES);
    const size_t smem = 512 + (size_t)ns * stage_bytes;
    if (smem > (size_t)optin) return fail(h, TLBM_ERR_ARG, "%zu bytes of shared memory per block exceed %d", smem, optin);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(h, TLBM_ERR_ARG, "%zu bytes of shared memory per block do not fit", smem);
    const long long tiles = (long long)h->ny * h->nz * ((h->nx + tw - 1) / tw);
    if (tiles >= (1ll << 31)) return fail(h, TLBM_ERR_ARG, "too many tiles for the staged kernel");
    h->staged = 1;
    h->staged_tw = tw;
    h->staged_nc = nc;
    h->staged_stages = ns;
    h->staged_smem = smem;
    h->staged_grid = (int)std::min<long long>(tiles, (long long)per_sm * sms);
    drop_graph(h);
    return TLBM_OK;
}

extern "C" int tlbm_set_staged(tlbm_t h, int tile_width, int stages) {
    TLBM_CHECK_HANDLE(h);
    const int rc = set_staged(h, tile_width, stages);
    if (rc == TLBM_OK) h->variant_chosen = 1;
    return rc;
}

extern "C" int tlbm_set_wait_limit(tlbm_t h, double seconds) {
    TLBM_CHECK_HANDLE(h);
    if (!(seconds >= 0.0 && seconds <= 10.0)) return fail(h, TLBM_ERR_ARG, "seconds must be in [0, 10]");
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    drop_graph(h);
    return TLBM_OK;
}

extern "C" int tlbm_get_staged(tlbm_t h, int* tile_width, int* stages, int* blocks) {
    TLBM_CHECK_HANDLE(h);
    if (tile_width) *tile_width = h->staged ? h->staged_tw : 0;
    if (stages) *stages = h->staged ? h->staged_stages : 0;
    if (blocks) *blocks = h->staged ? h->staged_grid : 0;
    return TLBM_OK;
}

extern "C" int tlbm_get_variant(tlbm_t h, int* vec, int* form, int* block_x, int* block_y, int* rows) {
    TLBM_CHECK_HANDLE(h);
    if (rows) *rows = h->rows;
    if (vec) *vec = h->staged ? 0 : h->vec;
    if (form) *form = h->trt ? 2 : 1;
    if (block_x) *block_x = h->bx;
    if (block_y) *block_y = h->by;
    return TLBM_OK;
}

extern "C" int tlbm_derived(tlbm_t h, double* out, int cap, int* count) {
    TLBM_CHECK_HANDLE(h);
    if (!out && cap > 0) return fail(h, TLBM_ERR_ARG, "out is NULL");
    double v[7 + MAXQ + 7];
    int n = 0;
    v[n++] = h->U; v[n++] = h->H; v[n++] = h->nu; v[n++] = h->alpha;
    v[n++] = h->gbeta; v[n++] = h->a_T; v[n++] = h->omega;
    for (int k = 0; k < h->qf; ++k) v[n++] = h->S[k];
    for (int k = 0; k < h->qg; ++k) v[n++] = h->Q[k];
    for (int i = 0; i < n && i < cap; ++i) out[i] = v[i];
    if (count) *count = n < cap ? n : cap;
    return TLBM_OK;
}

extern "C" int tlbm_bounds_violations(tlbm_t h, int64_t* count) {
    TLBM_CHECK_HANDLE(h);
    TLBM_CHECK_BOUND(h);
    if (!count) return fail(h, TLBM_ERR_ARG, "count is NULL");
#ifdef TLBM_DEBUG_BOUNDS
    unsigned long long c = 0;
    cudaError_t e = cudaMemcpyAsync(&c, h->kp.dbg_count, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading the violation counter");
    *count = (int64_t)c;
    return TLBM_OK;
#else
    *count = 0;
    return fail(h, TLBM_ERR_UNSUPPORTED, "this library is built without bounds checks (TLBM_DEBUG_BOUNDS)");
#endif
}

extern "C" const char* tlbm_last_error(tlbm_t h) { return h ? h->err : g_create_error; }

extern "C" int tlbm_launch_count(tlbm_t h, int64_t* count) {
    TLBM_CHECK_HANDLE(h);
    if (!count) return fail(h, TLBM_ERR_ARG, "count is NULL");
    *count = h->launches;
    return TLBM_OK;
}

extern "C" void tlbm_destroy(tlbm_t h) {
    if (!h) return;
    drop_graph(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
}
