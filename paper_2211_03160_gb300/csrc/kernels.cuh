// Fused stream + collide kernels of the DDF thermal lattice Boltzmann step
// (Xu & Li, §2.2 Eqs. (5)-(7), split form Eqs. (10)-(11), fused here).
//
// Data layout ("pull buffer with a ghost halo").  Each population i of a set
// lives in its own plane (SoA, x fastest, §3.1).  A plane has one ghost layer
// around the cell: slots x in [-1, nx], y in [-1, ny] (and z in [-1, nz] in 3D),
//     slot(x, y, z) = OFF + ((z + zg) * (ny + 2) + (y + 1)) * P + x,
// zg = 1 in 3D and 0 in 2D, P = row pitch (multiple of 32, >= nx + 16).
// Slot (s, i) holds the value that node s + e_i pulls as its pre-collision
// f_i.  So a time step is a pure pull, f_i(x) = slot(x - e_i, i), with no
// branch, and the wall rules are applied when the post-collision values are
// written: a value leaving the cell through a wall (half-way bounce-back,
// anti-bounce-back, adiabatic bounce-back, §2.2) is written into the ghost slot
// that its own node will pull from in the next step; a value leaving through a
// periodic face is written into the ghost slot its periodic image pulls from.
// Every ghost slot that is ever read has exactly one writer.
//
// Precision variants: storage S in {double, float, __half, __nv_bfloat16};
// collision in C = double for double storage, float otherwise.  The collision
// works on deviations d_i = f_i - w_i; FP16/BF16 storage keeps d_i * scale
// (flow) and g_i * scale (temperature), the "offset" storage.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"

namespace tlbm {

constexpr int MAXQ = 19;
constexpr int ROW_ALIGN = 32;   // row pitch multiple (elements)
constexpr int SLOT_OFF = 64;    // offset of slot (0, -1[, -1]) row start (elements)
constexpr int TAIL = 64;        // padding after the last row of a plane (elements)

struct Layout {
    int nx, ny, nz;          // nz = 1 in 2D
    int dim;
    int P;                   // row pitch in elements
    int zg;                  // 1 in 3D, 0 in 2D
    long long plane;         // elements per population plane (padded)
    __host__ __device__ __forceinline__ long long row(int y, int z) const {
        return (long long)SLOT_OFF + ((long long)(z + zg) * (ny + 2) + (y + 1)) * P;
    }
    __host__ __device__ __forceinline__ long long slot(int x, int y, int z) const {
        return row(y, z) + x;
    }
};

// Kernel parameters (passed by value).
struct KParams {
    Layout L;
    int periodic;            // bit0 x, bit1 y, bit2 z
    int heat_axis;           // axis normal to the isothermal walls
    int grav_axis;           // 1 (2D) or 2 (3D)
    int xmax_load;           // largest safe vector start for lanes past the row end
    double gbeta, omega, Th, Tc, a_T;
    double body[3];
    double S[MAXQ], Sh[MAXQ];  // flow rates and 1 - S/2
    double Q[7];
    float Sf[MAXQ], Shf[MAXQ], Qf[7];
    float gbetaf, omegaf, Thf, Tcf, a_Tf, bodyf[3];
    float scale, inv_scale;  // offset-storage scale
    // two-relaxation-time form of the same collision (valid when every even
    // non-conserved rate equals sp and every odd one equals sm; the rates of the
    // conserved moments do not enter the result)
    int trt;
    double sp, sm, shp, shm, qp, qm;
    float spf, smf, shpf, shmf, qpf, qmf;
    // element offsets, relative to a node's own slot in plane 0, of the slot
    // each population j (flow planes first, then thermal) is pulled from, and
    // of the plane it is stored to
    // (32-bit: a population set holds fewer than 2^31 elements)
    int loff[2 * MAXQ];
    int soff[2 * MAXQ];
    // the same offsets as arithmetic on compile-time coefficients (off_plane,
    // off_shift): plane32 = plane, rp = (ny + 2) P
    int plane32, rp;
    // where the state's pre-collision f_i(x) lives, for the diagnostic and
    // transfer kernels: 0 two-buffer pull layout (slot x - e_i of plane i),
    // 1 in-place natural order (slot x of plane i), 2 in-place swapped order
    // (slot x - e_i of plane ibar)
    int state;
    // FP32 constants of the two-relaxation-time collision (collide_trt_v with
    // HC), formed once on the host, with the same operations in the same order
    // as the in-kernel form, and sc = scale (1 unless offset storage, whose
    // two-relaxation-time collision always runs on the scaled values):
    // m3shp = -3 shp, r1 = 4.5 sp, r3 = 3 sm, c1 = 1 - (sp + sm)/2,
    // c2 = (sm - sp)/2, omsp = 1 - sp, w0s/was/wbs = w_0/w_a/w_b sc,
    // f9x = 9 shp w_x sc, f3x = 3 shm w_x sc (x = a, b: the two weight classes);
    // thermal, with wT = omega/2: t1 = 1 - (qp + qm)/2, t2 = (qm - qp)/2,
    // qpwT = qp wT, hqm = qm/2, omqp = 1 - qp, g0c = qp fma(-(Q_g - 1), wT, 1)
    struct {
        float m3shp, r1, r3, c1, c2, omsp, w0s, was, wbs, f9a, f9b, f3a, f3b;
        float t1, t2, qpwT, hqm, omqp, g0c;
    } tf;
#ifdef TLBM_DEBUG_BOUNDS
    // the population buffers of the handle and the violation counter
    const char* dbg_lo;
    const char* dbg_hi;
    unsigned long long* dbg_count;
#endif
};

// Bounds check of the debug build (TLBM_DEBUG_BOUNDS; compiled out otherwise):
// the access of elements q[-before .. n - before) must lie in the population
// buffers [p.dbg_lo, p.dbg_hi).  One that does not is counted in *p.dbg_count
// and redirected to element 16 of the buffers (aligned for every vector
// width), so that nothing outside the allocation is touched.
// TLBM_DBG(p, q, before, n) is the checked pointer in the debug build and q
// itself otherwise (a macro, so that the release build's code, including what
// the compiler knows about pointer aliasing, is exactly the unchecked one).
#ifdef TLBM_DEBUG_BOUNDS
template <class T>
__device__ __forceinline__ T* dbg_ptr(const KParams& p, T* q, int before, int n) {
    const char* a = reinterpret_cast<const char*>(q - before);
    if (a >= p.dbg_lo && a + (long long)n * (long long)sizeof(T) <= p.dbg_hi) return q;
    atomicAdd(p.dbg_count, 1ull);
    using B = typename std::conditional<std::is_const<T>::value, const char, char>::type;
    return reinterpret_cast<T*>(const_cast<B*>(p.dbg_lo)) + 16;
}
#define TLBM_DBG(p, q, before, n) ::tlbm::dbg_ptr((p), (q), (before), (n))
#else
#define TLBM_DBG(p, q, before, n) (q)
#endif

template <int j, int dy, int dz>
__device__ __forceinline__ int off_shift(const KParams& p) {
    return j * p.plane32 + dy * p.L.P + dz * p.rp;
}

// Element offset, relative to a node's own slot in plane 0, of plane j (both
// sets numbered flow first) shifted by dy rows and dz row planes.  The in-place
// halves form their addresses from these (three per-launch values held by a
// thread) rather than from the offset tables: measured 6-10 % faster there,
// while the two-buffer kernels stay with the tables (0.4-1.3 % faster).
template <int j, int dy = 0, int dz = 0>
__device__ __forceinline__ int off_shift(const struct KParams& p);

// ------------------------------------------------------------------ storage

template <class S>
struct Storage;
// offset: the flow planes hold the deviations d_i = f_i - w_i (times the
// storage scale) rather than f_i, so that a stored value keeps the precision of
// the deviation instead of rounding at the ulp of w_i; scaled: that scale may
// differ from 1 (FP32 deviations are stored as they are).
template <>
struct Storage<double> {
    using C = double;
    static constexpr bool offset = false;
    static constexpr bool scaled = false;
};
template <>
struct Storage<float> {
    using C = float;
    static constexpr bool offset = true;
    static constexpr bool scaled = false;
};
template <>
struct Storage<__half> {
    using C = float;
    static constexpr bool offset = true;
    static constexpr bool scaled = true;
};
template <>
struct Storage<__nv_bfloat16> {
    using C = float;
    static constexpr bool offset = true;
    static constexpr bool scaled = true;
};

// The collision works on the stored values directly (KS) with two-relaxation-
// time rates on offset storage; it has to unscale them only if the storage
// scale may differ from 1.
template <class S, bool TRT>
constexpr bool collide_scaled = TRT && Storage<S>::offset && Storage<S>::scaled;

template <class C, class S>
__device__ __forceinline__ C to_c(S s) {
    if constexpr (std::is_same<S, __half>::value) return __half2float(s);
    else if constexpr (std::is_same<S, __nv_bfloat16>::value) return __bfloat162float(s);
    else return C(s);
}
template <class S, class C>
__device__ __forceinline__ S from_c(C c) {
    if constexpr (std::is_same<S, __half>::value) return __float2half_rn(c);
    else if constexpr (std::is_same<S, __nv_bfloat16>::value) return __float2bfloat16_rn(c);
    else return S(c);
}

// ------------------------------------------------------------------ stochastic rounding
//
// FP16/BF16 storage rounds every value a time step stores stochastically: up
// with probability equal to the dropped fraction of an ulp, so that a stored
// value is exact in expectation.  Round to nearest drops every per-step change
// below half an ulp; in a Rayleigh-Benard cell at 257^2 (about 4450 steps per
// free-fall time, so populations change by ~2e-4 of their value per step) the
// FP16 state then froze into a steady roll whose time-averaged Nusselt number
// was 40 % below FP64, and convection never started from the noisy conductive
// state.  The hardware conversion cvt.rs takes its random bits from a 32-bit
// operand: for two packed values the upper value uses bits 31..16 (FP16: the 13
// bits 28..16), the lower one bits 15..0 (FP16: 12..0); it rounds up when the
// dropped bits plus those bits carry into the kept ones.  The bits of a value
// are the top 16 bits of its FP32 pattern times 0x9E3779B1 (2^32 / golden
// ratio): a deterministic function of the value alone, so every kernel variant
// stores bitwise the same state, and a Weyl sequence in the value's low bits, so
// that a value changing by a few units in its last place per step meets
// equidistributed thresholds.  A value that does not change at all would meet
// the same threshold every step (and round the same way, so that a nearly
// frozen state stays frozen: a 129^2 cell at Ra = 2e4 never left its noisy
// conductive start), so the key also adds a per-step salt, t times the same
// constant, t being the step counter that the time steps keep in the first word
// of each population buffer (step_count / advance_count below): the threshold
// of a constant value then runs through a Weyl sequence over the steps.
// Initial states and transfers (tlbm_init, tlbm_set_populations) round to
// nearest.
__device__ __forceinline__ uint32_t sr_key(float v, uint32_t salt) { return __float_as_uint(v) * 0x9E3779B1u + salt; }

// (hi, lo) -> packed 16-bit pair, lo in the low half, stochastically rounded
template <class S>
__device__ __forceinline__ uint32_t cvt_rs2(float hi, float lo, uint32_t salt) {
    const uint32_t r = __byte_perm(sr_key(lo, salt), sr_key(hi, salt), 0x7632);  // top16(hi) << 16 | top16(lo)
    uint32_t d;
    if constexpr (std::is_same<S, __half>::value)
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}

// the value a time step stores: stochastically rounded for 16-bit storage (the
// same threshold as it would get in the low half of a pair)
template <class S, class C>
__device__ __forceinline__ S from_c_step(C c, uint32_t salt) {
    if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) {
        const unsigned short b = (unsigned short)(cvt_rs2<S>(0.0f, (float)c, salt) & 0xffffu);
        S v;
        memcpy(&v, &b, 2);
        return v;
    } else {
        return S(c);
    }
}

template <class S>
constexpr bool is16 = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;

// The step counter of 16-bit storage: a 32-bit word at the start of each
// population buffer (in the padding before slot (0, -1, -1), which no kernel
// touches).  A two-buffer step reads word 0 of its source and writes the count
// plus one into word 0 of its destination; the in-place halves alternate
// between words 0 and 1 of their single buffer (AA_EVEN reads 0 and writes 1,
// AA_ODD the reverse).  tlbm_init and tlbm_set_populations clear it with the
// buffers, tlbm_load sets it to the restored step count.
template <class S, bool CG = false>
__device__ __forceinline__ uint32_t step_count(const S* buf, int word) {
    if constexpr (!is16<S>) return 0u;
    const uint32_t* w = reinterpret_cast<const uint32_t*>(buf) + word;
    if constexpr (CG) return __ldcg(w);
    else return __ldg(w);
}
template <class S>
__device__ __forceinline__ void advance_count(S* buf, int word, uint32_t t, bool writer) {
    if constexpr (is16<S>) {
        if (writer) reinterpret_cast<uint32_t*>(buf)[word] = t + 1u;
    }
}
// the per-step salt of the stochastic rounding key
__device__ __forceinline__ uint32_t step_salt(uint32_t t) { return t * 0x9E3779B9u; }

// parameter accessors in the compute precision
template <class C> struct PV;
template <> struct PV<double> {
    __device__ static double sp(const KParams& p) { return p.sp; }
    __device__ static double sm(const KParams& p) { return p.sm; }
    __device__ static double shp(const KParams& p) { return p.shp; }
    __device__ static double shm(const KParams& p) { return p.shm; }
    __device__ static double qp(const KParams& p) { return p.qp; }
    __device__ static double qm(const KParams& p) { return p.qm; }
    __device__ static double S(const KParams& p, int k) { return p.S[k]; }
    __device__ static double Sh(const KParams& p, int k) { return p.Sh[k]; }
    __device__ static double Q(const KParams& p, int k) { return p.Q[k]; }
    __device__ static double gbeta(const KParams& p) { return p.gbeta; }
    __device__ static double omega(const KParams& p) { return p.omega; }
    __device__ static double Th(const KParams& p) { return p.Th; }
    __device__ static double Tc(const KParams& p) { return p.Tc; }
    __device__ static double aT(const KParams& p) { return p.a_T; }
    __device__ static double body(const KParams& p, int a) { return p.body[a]; }
};
template <> struct PV<float> {
    __device__ static float sp(const KParams& p) { return p.spf; }
    __device__ static float sm(const KParams& p) { return p.smf; }
    __device__ static float shp(const KParams& p) { return p.shpf; }
    __device__ static float shm(const KParams& p) { return p.shmf; }
    __device__ static float qp(const KParams& p) { return p.qpf; }
    __device__ static float qm(const KParams& p) { return p.qmf; }
    __device__ static float S(const KParams& p, int k) { return p.Sf[k]; }
    __device__ static float Sh(const KParams& p, int k) { return p.Shf[k]; }
    __device__ static float Q(const KParams& p, int k) { return p.Qf[k]; }
    __device__ static float gbeta(const KParams& p) { return p.gbetaf; }
    __device__ static float omega(const KParams& p) { return p.omegaf; }
    __device__ static float Th(const KParams& p) { return p.Thf; }
    __device__ static float Tc(const KParams& p) { return p.Tcf; }
    __device__ static float aT(const KParams& p) { return p.a_Tf; }
    __device__ static float body(const KParams& p, int a) { return p.bodyf[a]; }
};

// flow weight w_i in precision C
template <class L, class C>
__device__ __forceinline__ constexpr C weight(int i) {
    return C(L::w36(i)) / C(36);
}

// decode a stored flow value into its deviation d_i = f_i - w_i
template <class LF, class S, class C>
__device__ __forceinline__ C dec_f(S s, int i, C inv_scale) {
    if constexpr (Storage<S>::offset) return to_c<C>(s) * inv_scale;
    else return to_c<C>(s) - weight<LF, C>(i);
}
template <class LF, class S, class C>
__device__ __forceinline__ S enc_f(C d, int i, C scale) {
    if constexpr (Storage<S>::offset) return from_c<S>(d * scale);
    else return from_c<S>(weight<LF, C>(i) + d);
}
template <class S, class C>
__device__ __forceinline__ C dec_g(S s, C inv_scale) {
    if constexpr (Storage<S>::offset) return to_c<C>(s) * inv_scale;
    else return to_c<C>(s);
}
template <class S, class C>
__device__ __forceinline__ S enc_g(C g, C scale) {
    if constexpr (Storage<S>::offset) return from_c<S>(g * scale);
    else return from_c<S>(g);
}
// the same as stored by a time step (stochastic rounding for 16-bit storage)
template <class LF, class S, class C>
__device__ __forceinline__ S enc_f_step(C d, int i, C scale, uint32_t salt) {
    if constexpr (Storage<S>::offset) return from_c_step<S>(d * scale, salt);
    else return from_c_step<S>(weight<LF, C>(i) + d, salt);
}
template <class S, class C>
__device__ __forceinline__ S enc_g_step(C g, C scale, uint32_t salt) {
    if constexpr (Storage<S>::offset) return from_c_step<S>(g * scale, salt);
    else return from_c_step<S>(g, salt);
}

template <class C> struct ScaleOf;
template <> struct ScaleOf<float> {
    __device__ static float s(const KParams& p) { return p.scale; }
    __device__ static float inv(const KParams& p) { return p.inv_scale; }
};
template <> struct ScaleOf<double> {
    __device__ static double s(const KParams& p) { return (double)p.scale; }
    __device__ static double inv(const KParams& p) { return (double)p.inv_scale; }
};

// ------------------------------------------------------------------ collision

// 1/x, correctly rounded in both precisions
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Macroscopic moments of one node from deviations (§2.2):
// rho = 1 + sum d, T = sum g, F = rho (g beta T ghat + a), u = (sum e f + F/2)/rho.
// 2D flow MRT + Guo forcing (Eq. (5), Eq. (6a)) and D2Q5 thermal MRT (Eq. (7)),
// in deviation form: every moment is taken relative to the rest state
// (rho = 1, u = 0), m_w = M w = [1, -2, 1, 0, ...].
template <class C>
__device__ __forceinline__ void collide_2d(C (&d)[9], C (&g)[5], const KParams& p) {
    using P = PV<C>;
    C m[9], n[5];
    moments<D2Q9>(d, m);
    moments<D2Q5>(g, n);
    const C drho = m[0];
    const C rho = C(1) + drho;
    const C T = n[0];
    const C Fx = rho * P::body(p, 0);
    const C Fy = rho * (P::gbeta(p) * T + P::body(p, 1));
    const C ir = C(1) / rho;
    const C ux = (m[3] + C(0.5) * Fx) * ir;
    const C uy = (m[5] + C(0.5) * Fy) * ir;
    const C ru2 = rho * (ux * ux + uy * uy);
    // m_eq - m_w (Lallemand & Luo basis)
    const C meq[9] = {drho,
                      C(-2) * drho + C(3) * ru2,
                      drho - C(3) * ru2,
                      rho * ux,
                      -rho * ux,
                      rho * uy,
                      -rho * uy,
                      rho * (ux * ux - uy * uy),
                      rho * ux * uy};
    // M Ftilde, Eq. (6a) (last entry read as u Fy + v Fx)
    const C uF = ux * Fx + uy * Fy;
    const C mF[9] = {C(0),     C(6) * uF, C(-6) * uF, Fx, -Fx, Fy, -Fy,
                     C(2) * (ux * Fx - uy * Fy), ux * Fy + uy * Fx};
    static_for<9>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        m[k] = m[k] - P::S(p, k) * (m[k] - meq[k]) + P::Sh(p, k) * mF[k];
    });
    populations<D2Q9>(m, d);
    // thermal: n_eq = [T, uT, vT, a_T T, 0]
    const C neq[5] = {T, ux * T, uy * T, P::aT(p) * T, C(0)};
    static_for<5>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        if constexpr (k > 0) n[k] = n[k] - P::Q(p, k) * (n[k] - neq[k]);
    });
    populations<D2Q5>(n, g);
}

// 3D: D3Q19 MRT (d'Humieres basis) + Guo forcing Eq. (6b), D3Q7 thermal MRT.
// m_w = M w = [1, -11, 3, 0, ...].
template <class C>
__device__ __forceinline__ void collide_3d(C (&d)[19], C (&g)[7], const KParams& p) {
    using P = PV<C>;
    C m[19], n[7];
    moments<D3Q19>(d, m);
    moments<D3Q7>(g, n);
    const C drho = m[0];
    const C rho = C(1) + drho;
    const C T = n[0];
    const C Fx = rho * P::body(p, 0);
    const C Fy = rho * P::body(p, 1);
    const C Fz = rho * (P::gbeta(p) * T + P::body(p, 2));
    const C ir = C(1) / rho;
    const C ux = (m[3] + C(0.5) * Fx) * ir;
    const C uy = (m[5] + C(0.5) * Fy) * ir;
    const C uz = (m[7] + C(0.5) * Fz) * ir;
    const C ru2 = rho * (ux * ux + uy * uy + uz * uz);
    const C pxx = rho * (C(2) * ux * ux - uy * uy - uz * uz);
    const C pww = rho * (uy * uy - uz * uz);
    const C meq[19] = {drho,
                       C(-11) * drho + C(19) * ru2,
                       C(3) * drho - C(5.5) * ru2,
                       rho * ux, C(-2) / C(3) * (rho * ux),
                       rho * uy, C(-2) / C(3) * (rho * uy),
                       rho * uz, C(-2) / C(3) * (rho * uz),
                       pxx, C(-0.5) * pxx, pww, C(-0.5) * pww,
                       rho * ux * uy, rho * uy * uz, rho * ux * uz,
                       C(0), C(0), C(0)};
    const C uF = ux * Fx + uy * Fy + uz * Fz;
    const C mF[19] = {C(0), C(38) * uF, C(-11) * uF,
                      Fx, C(-2) / C(3) * Fx, Fy, C(-2) / C(3) * Fy, Fz, C(-2) / C(3) * Fz,
                      C(4) * ux * Fx - C(2) * uy * Fy - C(2) * uz * Fz,
                      C(-2) * ux * Fx + uy * Fy + uz * Fz,
                      C(2) * uy * Fy - C(2) * uz * Fz,
                      -uy * Fy + uz * Fz,
                      ux * Fy + uy * Fx, uy * Fz + uz * Fy, ux * Fz + uz * Fx,
                      C(0), C(0), C(0)};
    static_for<19>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        m[k] = m[k] - P::S(p, k) * (m[k] - meq[k]) + P::Sh(p, k) * mF[k];
    });
    populations<D3Q19>(m, d);
    const C neq[7] = {T, ux * T, uy * T, uz * T, P::aT(p) * T, C(0), C(0)};
    static_for<7>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        if constexpr (k > 0) n[k] = n[k] - P::Q(p, k) * (n[k] - neq[k]);
    });
    populations<D3Q7>(n, g);
}

template <int DIM> struct Lat;
template <> struct Lat<2> { using F = D2Q9; using G = D2Q5; };
template <> struct Lat<3> { using F = D3Q19; using G = D3Q7; };


// Two-relaxation-time evaluation of the same collision.  When every even
// non-conserved moment relaxes with sp and every odd one with sm, the MRT
// operator M^-1 S M of Eq. (5) equals sp on the symmetric part and sm on the
// antisymmetric part of each pair (i, ibar), and M^-1 (I - S/2) M Ftilde
// splits the same way (the conserved moments' rates cancel out, see the MRT
// form above).  Likewise for the thermal operator of Eq. (7).  In deviation
// form, with E_i = f_eq,i - w_i = w_i [drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)]
// and the Guo source G_i = w_i [3 (e - u).F + 9 (e.u)(e.F)], a pair updates as
//   d_i+    = c1 d_i + c2 d_ibar + Ks + Ka,   d_ibar+ = c1 d_ibar + c2 d_i + Ks - Ka,
//   c1 = 1 - (sp + sm)/2,  c2 = (sm - sp)/2,
//   Ks = sp E_i^s + (1 - sp/2) G_i^s = w_i [K0 + e.u (4.5 sp rho e.u + 9 (1 - sp/2) e.F)],
//   Ka = sm E_i^a + (1 - sm/2) G_i^a = w_i [3 sm rho e.u + 3 (1 - sm/2) e.F],
//   K0 = sp drho - 1.5 sp rho u^2 - 3 (1 - sp/2) u.F   (one value per node),
// and the rest population as d_0+ = (1 - sp) d_0 + w_0 K0.  The thermal pairs:
//   g_i+ = t1 g_i + t2 g_ibar + qp wT T + (qm/2) e.u T  (and - for ibar),
//   t1 = 1 - (qp + qm)/2, t2 = (qm - qp)/2, wT = omega/2;  g_0+ = (1 - qp) g_0 + qp (1 - (q-1) wT) T.
// SCALED: the inputs and outputs are the stored values d_i * scale and
// g_i * scale (offset storage); every term is linear in them except through the
// node's rho, u and T, which are formed unscaled.
template <int DIM, class C, bool SCALED>
__device__ __forceinline__ void collide_trt(C (&d)[Lat<DIM>::F::Q], C (&g)[Lat<DIM>::G::Q], const KParams& p) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using P = PV<C>;
    C drs = C(0), jx = C(0), jy = C(0), jz = C(0), Ts = C(0);
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        drs += d[i];
        if constexpr (LF::e(i, 0) == 1) jx += d[i];
        if constexpr (LF::e(i, 0) == -1) jx -= d[i];
        if constexpr (LF::e(i, 1) == 1) jy += d[i];
        if constexpr (LF::e(i, 1) == -1) jy -= d[i];
        if constexpr (LF::e(i, 2) == 1) jz += d[i];
        if constexpr (LF::e(i, 2) == -1) jz -= d[i];
    });
    static_for<LG::Q>([&](auto ii) { Ts += g[decltype(ii)::value]; });
    C sc = C(1), inv = C(1);
    if constexpr (SCALED) {
        sc = ScaleOf<C>::s(p);
        inv = ScaleOf<C>::inv(p);
    }
    const C drho = SCALED ? drs * inv : drs;
    const C T = SCALED ? Ts * inv : Ts;
    const C rho = C(1) + drho;
    const C buoy = P::gbeta(p) * T;
    const C Fx = rho * P::body(p, 0);
    const C Fy = rho * (DIM == 2 ? buoy + P::body(p, 1) : P::body(p, 1));
    const C Fz = DIM == 3 ? rho * (buoy + P::body(p, 2)) : C(0);
    const C ir = recip(rho);
    const C hx = C(0.5) * Fx, hy = C(0.5) * Fy, hz = C(0.5) * Fz;
    const C ux = (SCALED ? fma(jx, inv, hx) : jx + hx) * ir;
    const C uy = (SCALED ? fma(jy, inv, hy) : jy + hy) * ir;
    const C uz = DIM == 3 ? (SCALED ? fma(jz, inv, hz) : jz + hz) * ir : C(0);
    const C sp = P::sp(p), sm = P::sm(p), shp = P::shp(p), shm = P::shm(p);
    const C uu15 = C(1.5) * (ux * ux + uy * uy + uz * uz);
    const C uF3 = C(3) * (ux * Fx + uy * Fy + uz * Fz);
    const C K0 = sp * (drho - rho * uu15) - shp * uF3;
    const C R1 = C(4.5) * sp * rho, R2 = C(9) * shp;
    const C R3 = C(3) * sm * rho, R4 = C(3) * shm;
    const C c1 = C(1) - C(0.5) * (sp + sm), c2 = C(0.5) * (sm - sp);
    {
        constexpr C w0 = weight<LF, C>(0);
        d[0] = (C(1) - sp) * d[0] + (w0 * sc) * K0;
    }
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        constexpr int o = LF::opp(i);
        if constexpr (i != 0 && i < o) {
            constexpr int ex = LF::e(i, 0), ey = LF::e(i, 1), ez = LF::e(i, 2);
            const C ws = weight<LF, C>(i) * sc;
            C eu = C(0), eF = C(0);
            if constexpr (ex != 0) { eu += C(ex) * ux; eF += C(ex) * Fx; }
            if constexpr (ey != 0) { eu += C(ey) * uy; eF += C(ey) * Fy; }
            if constexpr (ez != 0) { eu += C(ez) * uz; eF += C(ez) * Fz; }
            const C Ks = ws * (K0 + eu * (R1 * eu + R2 * eF));
            const C Ka = ws * (R3 * eu + R4 * eF);
            const C di = d[i], dob = d[o];
            d[i] = c1 * di + c2 * dob + (Ks + Ka);
            d[o] = c1 * dob + c2 * di + (Ks - Ka);
        }
    });
    // thermal
    const C qp = P::qp(p), qm = P::qm(p);
    const C wT = C(0.5) * P::omega(p);
    const C t1 = C(1) - C(0.5) * (qp + qm), t2 = C(0.5) * (qm - qp);
    const C Ks_T = qp * wT * Ts;        // scaled like g
    const C ka_T = C(0.5) * qm * Ts;    // times e.u
    g[0] = (C(1) - qp) * g[0] + qp * (C(1) - C(LG::Q - 1) * wT) * Ts;
    static_for<LG::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        constexpr int o = LG::opp(i);
        if constexpr (i != 0 && i < o) {
            constexpr int ex = LG::e(i, 0), ey = LG::e(i, 1), ez = LG::e(i, 2);
            const C eu = ex != 0 ? C(ex) * ux : (ey != 0 ? C(ey) * uy : C(ez) * uz);
            const C Ka = ka_T * eu;
            const C gi = g[i], go = g[o];
            g[i] = t1 * gi + t2 * go + (Ks_T + Ka);
            g[o] = t1 * go + t2 * gi + (Ks_T - Ka);
        }
    });
}

// ------------------------------------------------------------------ FP32 pairs
//
// sm_100-class SMs execute two independent FP32 operations per instruction on a
// register pair (FADD2 / FMUL2 / FFMA2; each half is an ordinary IEEE
// round-to-nearest operation).  The FP32 two-relaxation-time collision is
// therefore written once over V = float (one node) and V = float2 (two
// x-adjacent nodes of one thread), with explicit, never-contracted operations,
// so that a node gets bitwise the same result whichever form updates it.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
template <class V> __device__ __forceinline__ V vbc(float x);
template <> __device__ __forceinline__ float vbc<float>(float x) { return x; }
template <> __device__ __forceinline__ float2 vbc<float2>(float x) { return make_float2(x, x); }
// a - b as one rounding (b * -1 is exact)
template <class V> __device__ __forceinline__ V vsub(V a, V b) { return vfma(b, vbc<V>(-1.0f), a); }

// Sum over the velocity components with coefficients c in {-1, 0, 1}; the first
// non-zero coefficient must be +1.
template <class V, int CX, int CY, int CZ>
__device__ __forceinline__ V vdot_unit(V x, V y, V z) {
    static_assert(CX == 1 || (CX == 0 && CY == 1) || (CX == 0 && CY == 0 && CZ == 1), "first coefficient +1");
    V r = CX ? x : (CY ? y : z);
    if constexpr (CX != 0 && CY == 1) r = vadd(r, y);
    if constexpr (CX != 0 && CY == -1) r = vsub(r, y);
    if constexpr ((CX != 0 || CY != 0) && CZ == 1) r = vadd(r, z);
    if constexpr ((CX != 0 || CY != 0) && CZ == -1) r = vsub(r, z);
    return r;
}

// The collision of collide_trt above in FP32, over V = float or float2.  Per
// pair (i, ibar) the direction with a leading +1 component, e*, carries the
// antisymmetric part: with sg = +1 if e_i = e*, -1 otherwise,
//   d_i+ = c1 d_i + c2 d_ibar + Ks + sg Ka*,  d_ibar+ = c1 d_ibar + c2 d_i + Ks - sg Ka*,
//   Ks  = ws K0 + e*.u (R1w e*.u + R2w e*.F),   Ka* = R3w e*.u + R4w e*.F,
// where R1w = 4.5 sp rho ws, R2w = 9 (1 - sp/2) ws, R3w = 3 sm rho ws,
// R4w = 3 (1 - sm/2) ws and ws = w_i * scale (the same terms as above, with
// the lattice weight folded in per weight class).
//
// HC: take the per-launch constants from p.tf (formed on the host, bitwise the
// same values) instead of forming them in every thread.  Measured on GB300:
// +4 % for the staged 2D FP16 kernel, +1.6 % for the in-place 2D FP32 kernel;
// -1 % to -7 % for the 3D FP16 kernels held to 96 registers and the batched
// FP32 kernel, within 0.3 % elsewhere.
template <int DIM, class V, bool SCALED, bool HC = false>
__device__ __forceinline__ void collide_trt_v(V (&d)[Lat<DIM>::F::Q], V (&g)[Lat<DIM>::G::Q], const KParams& p) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using P = PV<float>;
    const V zero = vbc<V>(0.0f);
    V drs = d[0], jx = zero, jy = zero, jz = zero;
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        if constexpr (i > 0) drs = vadd(drs, d[i]);
        if constexpr (LF::e(i, 0) == 1) jx = vadd(jx, d[i]);
        if constexpr (LF::e(i, 0) == -1) jx = vsub(jx, d[i]);
        if constexpr (LF::e(i, 1) == 1) jy = vadd(jy, d[i]);
        if constexpr (LF::e(i, 1) == -1) jy = vsub(jy, d[i]);
        if constexpr (LF::e(i, 2) == 1) jz = vadd(jz, d[i]);
        if constexpr (LF::e(i, 2) == -1) jz = vsub(jz, d[i]);
    });
    V Ts = g[0];
    static_for<LG::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        if constexpr (i > 0) Ts = vadd(Ts, g[i]);
    });
    const float sc = SCALED ? ScaleOf<float>::s(p) : 1.0f;
    const V inv = vbc<V>(SCALED ? ScaleOf<float>::inv(p) : 1.0f);
    const V drho = SCALED ? vmul(drs, inv) : drs;
    const V T = SCALED ? vmul(Ts, inv) : Ts;
    const V rho = vadd(vbc<V>(1.0f), drho);
    const V buoy = vmul(vbc<V>(P::gbeta(p)), T);
    const V Fx = vmul(rho, vbc<V>(P::body(p, 0)));
    const V Fy = vmul(rho, DIM == 2 ? vadd(buoy, vbc<V>(P::body(p, 1))) : vbc<V>(P::body(p, 1)));
    const V Fz = DIM == 3 ? vmul(rho, vadd(buoy, vbc<V>(P::body(p, 2)))) : zero;
    const V ir = vrcp(rho);
    const V half = vbc<V>(0.5f);
    const V ux = vmul(vfma(jx, inv, vmul(half, Fx)), ir);
    const V uy = vmul(vfma(jy, inv, vmul(half, Fy)), ir);
    const V uz = DIM == 3 ? vmul(vfma(jz, inv, vmul(half, Fz)), ir) : zero;
    const float sp = P::sp(p), sm = P::sm(p), shp = P::shp(p), shm = P::shm(p);
    const V uu = DIM == 3 ? vfma(ux, ux, vfma(uy, uy, vmul(uz, uz))) : vfma(ux, ux, vmul(uy, uy));
    const V uF = DIM == 3 ? vfma(ux, Fx, vfma(uy, Fy, vmul(uz, Fz))) : vfma(ux, Fx, vmul(uy, Fy));
    // K0 = sp (drho - 1.5 rho u^2) - 3 (1 - sp/2) u.F
    const V K0 = vfma(vbc<V>(sp), vfma(rho, vmul(vbc<V>(-1.5f), uu), drho), vmul(vbc<V>(HC ? p.tf.m3shp : -3.0f * shp), uF));
    const V R1 = vmul(vbc<V>(HC ? p.tf.r1 : 4.5f * sp), rho), R3 = vmul(vbc<V>(HC ? p.tf.r3 : 3.0f * sm), rho);
    const float c1 = HC ? p.tf.c1 : 1.0f - 0.5f * (sp + sm), c2 = HC ? p.tf.c2 : 0.5f * (sm - sp);
    {
        constexpr float w0 = weight<LF, float>(0);
        d[0] = vfma(vbc<V>(HC ? p.tf.omsp : 1.0f - sp), d[0], vmul(vbc<V>(HC ? p.tf.w0s : w0 * sc), K0));
    }
    // per weight class (D2Q9: 1/9, 1/36; D3Q19: 1/18, 1/36)
    constexpr float wa = weight<LF, float>(1), wb = weight<LF, float>(LF::Q - 1);
    const float was = HC ? p.tf.was : wa * sc, wbs = HC ? p.tf.wbs : wb * sc;
    const V wKa = vmul(vbc<V>(was), K0), wKb = vmul(vbc<V>(wbs), K0);
    const V R1a = vmul(vbc<V>(was), R1), R1b = vmul(vbc<V>(wbs), R1);
    const V R3a = vmul(vbc<V>(was), R3), R3b = vmul(vbc<V>(wbs), R3);
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        constexpr int o = LF::opp(i);
        if constexpr (i != 0 && i < o) {
            constexpr int ex = LF::e(i, 0), ey = LF::e(i, 1), ez = LF::e(i, 2);
            constexpr int sg = ex != 0 ? ex : (ey != 0 ? ey : ez);
            constexpr bool cls_a = LF::w36(i) == LF::w36(1);
            static_assert(cls_a || LF::w36(i) == LF::w36(LF::Q - 1), "two weight classes");
            const float ws = (cls_a ? wa : wb) * sc;
            const V eu = vdot_unit<V, sg * ex, sg * ey, sg * ez>(ux, uy, uz);
            const V eF = vdot_unit<V, sg * ex, sg * ey, sg * ez>(Fx, Fy, Fz);
            const V Ks = vfma(eu, vfma(cls_a ? R1a : R1b, eu, vmul(vbc<V>(HC ? (cls_a ? p.tf.f9a : p.tf.f9b) : 9.0f * shp * ws), eF)), cls_a ? wKa : wKb);
            const V Ka = vfma(cls_a ? R3a : R3b, eu, vmul(vbc<V>(HC ? (cls_a ? p.tf.f3a : p.tf.f3b) : 3.0f * shm * ws), eF));
            const V sum = sg > 0 ? vadd(Ks, Ka) : vsub(Ks, Ka);
            const V dif = sg > 0 ? vsub(Ks, Ka) : vadd(Ks, Ka);
            const V di = d[i], dob = d[o];
            d[i] = vfma(vbc<V>(c1), di, vfma(vbc<V>(c2), dob, sum));
            d[o] = vfma(vbc<V>(c1), dob, vfma(vbc<V>(c2), di, dif));
        }
    });
    // thermal
    const float qp = P::qp(p), qm = P::qm(p);
    const float wT = 0.5f * P::omega(p);
    const float t1 = HC ? p.tf.t1 : 1.0f - 0.5f * (qp + qm), t2 = HC ? p.tf.t2 : 0.5f * (qm - qp);
    const V Ks_T = vmul(vbc<V>(HC ? p.tf.qpwT : qp * wT), Ts);  // scaled like g
    const V ka_T = vmul(vbc<V>(HC ? p.tf.hqm : 0.5f * qm), Ts); // times e.u
    const float g0c = HC ? p.tf.g0c : qp * __fmaf_rn(-float(LG::Q - 1), wT, 1.0f);
    g[0] = vfma(vbc<V>(HC ? p.tf.omqp : 1.0f - qp), g[0], vmul(vbc<V>(g0c), Ts));
    static_for<LG::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        constexpr int o = LG::opp(i);
        if constexpr (i != 0 && i < o) {
            constexpr int ex = LG::e(i, 0), ey = LG::e(i, 1), ez = LG::e(i, 2);
            constexpr int sg = ex != 0 ? ex : (ey != 0 ? ey : ez);
            const V eu = ex != 0 ? ux : (ey != 0 ? uy : uz);
            const V Ka = vmul(ka_T, eu);
            const V sum = sg > 0 ? vadd(Ks_T, Ka) : vsub(Ks_T, Ka);
            const V dif = sg > 0 ? vsub(Ks_T, Ka) : vadd(Ks_T, Ka);
            const V gi = g[i], go = g[o];
            g[i] = vfma(vbc<V>(t1), gi, vfma(vbc<V>(t2), go, sum));
            g[o] = vfma(vbc<V>(t1), go, vfma(vbc<V>(t2), gi, dif));
        }
    });
}

template <int DIM, bool TRT, class C, bool SCALED = false, bool HC = false>
__device__ __forceinline__ void collide(C (&d)[Lat<DIM>::F::Q], C (&g)[Lat<DIM>::G::Q], const KParams& p) {
    if constexpr (TRT && std::is_same<C, float>::value) collide_trt_v<DIM, float, SCALED, HC>(d, g, p);
    else if constexpr (TRT) collide_trt<DIM, C, SCALED>(d, g, p);
    else if constexpr (DIM == 2) collide_2d<C>(d, g, p);
    else collide_3d<C>(d, g, p);
}

// Collide the nodes k = 0 .. VEC-1 of f[i][k], g[i][k]; two at a time on the
// FP32 pair instructions where the form and the count allow.  HC as for
// collide_trt_v.
template <int DIM, bool TRT, class C, bool KS, int VEC, bool HC = false>
__device__ __forceinline__ void collide_vec(C (&f)[Lat<DIM>::F::Q][VEC], C (&g)[Lat<DIM>::G::Q][VEC],
                                            const KParams& p) {
    constexpr int QF = Lat<DIM>::F::Q, QG = Lat<DIM>::G::Q;
    if constexpr (TRT && std::is_same<C, float>::value && VEC % 2 == 0) {
#pragma unroll
        for (int k = 0; k < VEC; k += 2) {
            float2 fd[QF], gd[QG];
#pragma unroll
            for (int i = 0; i < QF; ++i) fd[i] = make_float2(f[i][k], f[i][k + 1]);
#pragma unroll
            for (int i = 0; i < QG; ++i) gd[i] = make_float2(g[i][k], g[i][k + 1]);
            collide_trt_v<DIM, float2, KS, HC>(fd, gd, p);
#pragma unroll
            for (int i = 0; i < QF; ++i) { f[i][k] = fd[i].x; f[i][k + 1] = fd[i].y; }
#pragma unroll
            for (int i = 0; i < QG; ++i) { g[i][k] = gd[i].x; g[i][k + 1] = gd[i].y; }
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            C fd[QF], gd[QG];
#pragma unroll
            for (int i = 0; i < QF; ++i) fd[i] = f[i][k];
#pragma unroll
            for (int i = 0; i < QG; ++i) gd[i] = g[i][k];
            collide<DIM, TRT, C, KS, HC>(fd, gd, p);
#pragma unroll
            for (int i = 0; i < QF; ++i) f[i][k] = fd[i];
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i][k] = gd[i];
        }
    }
}

// Node macros from deviations (used by the diagnostic kernels).
template <int DIM, class C>
__device__ __forceinline__ void node_macros(const C (&d)[Lat<DIM>::F::Q], const C (&g)[Lat<DIM>::G::Q],
                                            const KParams& p, C& rho, C (&u)[3], C& T) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using P = PV<C>;
    C drho = C(0), j[3] = {C(0), C(0), C(0)}, t = C(0);
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        drho += d[i];
        if constexpr (LF::e(i, 0) == 1) j[0] += d[i];
        if constexpr (LF::e(i, 0) == -1) j[0] -= d[i];
        if constexpr (LF::e(i, 1) == 1) j[1] += d[i];
        if constexpr (LF::e(i, 1) == -1) j[1] -= d[i];
        if constexpr (LF::e(i, 2) == 1) j[2] += d[i];
        if constexpr (LF::e(i, 2) == -1) j[2] -= d[i];
    });
    static_for<LG::Q>([&](auto ii) { t += g[decltype(ii)::value]; });
    rho = C(1) + drho;
    T = t;
    C F[3] = {rho * P::body(p, 0), rho * P::body(p, 1), rho * P::body(p, 2)};
    F[DIM - 1] += rho * P::gbeta(p) * t;
    const C ir = C(1) / rho;
    u[0] = (j[0] + C(0.5) * F[0]) * ir;
    u[1] = (j[1] + C(0.5) * F[1]) * ir;
    u[2] = DIM == 3 ? (j[2] + C(0.5) * F[2]) * ir : C(0);
}

// ------------------------------------------------------------------ vector IO

// Loads of the populations: through the read-only path (ld.global.nc) when the
// source buffer is not written during the kernel; CG: cached in L2 only
// (ld.global.cg), for a kernel that reads, after a grid barrier, what other
// blocks of the same launch wrote.
template <bool CG, class T>
__device__ __forceinline__ T ld_pop(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}
template <class S, bool CG>
__device__ __forceinline__ S ld_one(const S* p) {
    if constexpr (sizeof(S) == 2) {
        const unsigned short t = ld_pop<CG>(reinterpret_cast<const unsigned short*>(p));
        S v;
        memcpy(&v, &t, 2);
        return v;
    } else {
        return ld_pop<CG>(p);
    }
}

template <class S, int VEC, bool CG = false>
__device__ __forceinline__ void ld_vec(const S* __restrict__ p, S (&v)[VEC]) {
    constexpr int B = VEC * (int)sizeof(S);
    static_assert(B == 2 || B == 4 || B == 8 || B == 16, "vector width");
    if constexpr (B == 16) {
        uint4 t = ld_pop<CG>(reinterpret_cast<const uint4*>(p));
        memcpy(v, &t, 16);
    } else if constexpr (B == 8) {
        uint2 t = ld_pop<CG>(reinterpret_cast<const uint2*>(p));
        memcpy(v, &t, 8);
    } else if constexpr (B == 4) {
        unsigned int t = ld_pop<CG>(reinterpret_cast<const unsigned int*>(p));
        memcpy(v, &t, 4);
    } else {
        unsigned short t = ld_pop<CG>(reinterpret_cast<const unsigned short*>(p));
        memcpy(v, &t, 2);
    }
}

// Stores of the populations, always to global memory (st.global): a buffer
// pointer the batched kernels read from their instance table would otherwise
// give generic stores.
template <class S, int VEC>
__device__ __forceinline__ void st_vec(S* __restrict__ p, const S (&v)[VEC]) {
    constexpr int B = VEC * (int)sizeof(S);
    if constexpr (B == 16) {
        uint4 t;
        memcpy(&t, v, 16);
        __stwb(reinterpret_cast<uint4*>(p), t);
    } else if constexpr (B == 8) {
        uint2 t;
        memcpy(&t, v, 8);
        __stwb(reinterpret_cast<uint2*>(p), t);
    } else if constexpr (B == 4) {
        unsigned int t;
        memcpy(&t, v, 4);
        __stwb(reinterpret_cast<unsigned int*>(p), t);
    } else {
        unsigned short t;
        memcpy(&t, v, 2);
        __stwb(reinterpret_cast<unsigned short*>(p), t);
    }
}

// Load the VEC consecutive stored values that nodes x0 .. x0+VEC-1 pull in a
// direction with x-component EX; `q` points at the slot of the source row
// (y - e_y, z - e_z) under x0 (16-byte aligned for VEC > 1).  The aligned
// vector at q is loaded and shifted by one element through a warp shuffle; the
// warp's edge lane fetches the one element beyond its vector directly.  All 32
// lanes must call this together.
template <class S, int VEC, int EX, class C, bool CG = false>
__device__ __forceinline__ void pull_row(const S* __restrict__ q, int lane, C (&out)[VEC]) {
    if constexpr (VEC == 1) {
        // one node per thread: a scalar load needs no alignment, fetch the
        // shifted element directly
        out[0] = to_c<C>(ld_one<S, CG>(q - EX));
        return;
    }
    S v[VEC];
    ld_vec<S, VEC, CG>(q, v);
    if constexpr (EX == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) out[k] = to_c<C>(v[k]);
    } else if constexpr (EX == 1) {
        // node x pulls from x - 1
        C left = __shfl_up_sync(0xffffffffu, to_c<C>(v[VEC - 1]), 1);
        if (lane == 0) left = to_c<C>(ld_one<S, CG>(q - 1));
        out[0] = left;
#pragma unroll
        for (int k = 1; k < VEC; ++k) out[k] = to_c<C>(v[k - 1]);
    } else {
        // node x pulls from x + 1
        C right = __shfl_down_sync(0xffffffffu, to_c<C>(v[0]), 1);
        if (lane == 31) right = to_c<C>(ld_one<S, CG>(q + VEC));
#pragma unroll
        for (int k = 0; k < VEC - 1; ++k) out[k] = to_c<C>(v[k + 1]);
        out[VEC - 1] = right;
    }
}

// ------------------------------------------------------------------ wall rules

// Streaming schemes (the MODE of the wall rules and of the step body):
//   PULL    two buffers; slot (s, i) holds what node s + e_i pulls next step.
//   AA_EVEN in place, first half of a step pair: every node reads its own slots
//           (x, i), collides, and writes f+_i back into its own slot (x, ibar).
//   AA_ODD  in place, second half: node x reads f_i from (x - e_i, ibar), collides
//           and pushes f+_i to (x + e_i, i), which restores the natural order.
// In both in-place halves every node reads and writes one and the same set of
// slots, so the update is race-free in a single buffer.
constexpr int PULL = 0, AA_EVEN = 1, AA_ODD = 2;

// Write the post-collision value `val` of population i (set LS, flow or
// thermal) of node (x, y, z) where the next step will read it, if it leaves
// the cell.  THERMAL selects the temperature rules of §2.2.  PULL: into the
// ghost slot the node (wall) or its periodic image pulls from.  AA_EVEN: into
// the ghost slot the following AA_ODD half reads it from.  AA_ODD: into the slot
// the next AA_EVEN half reads (the node's own slot of the opposite direction
// for a wall, the image's own slot for a periodic face).
template <class LS, bool THERMAL, int i, class S, class C, int MODE = PULL>
__device__ __forceinline__ void ghost_write(S* __restrict__ base, const KParams& p, int x, int y, int z, C val,
                                            C scale, uint32_t salt) {
    constexpr int ex = LS::e(i, 0), ey = LS::e(i, 1), ez = LS::e(i, 2);
    if constexpr (ex == 0 && ey == 0 && ez == 0) return;
    const Layout& L = p.L;
    const int dx = x + ex, dy = y + ey, dz = z + ez;
    const bool ox = dx < 0 || dx >= L.nx;
    const bool oy = dy < 0 || dy >= L.ny;
    const bool oz = (ez != 0) && (dz < 0 || dz >= L.nz);
    if (!(ox || oy || oz)) return;
    const bool wall = (ox && !(p.periodic & 1)) || (oy && !(p.periodic & 2)) || (oz && !(p.periodic & 4));
    constexpr int o = LS::opp(i);
    if (wall) {
        // bounce-back: the value returns to the node as f_ibar of the next step
        C out = val;
        if constexpr (THERMAL) {
            // axis-aligned: exactly one axis is crossed
            const int ax = ox ? 0 : (oy ? 1 : 2);
            if (ax == p.heat_axis) {
                const bool hi = ox ? (dx >= L.nx) : (oy ? (dy >= L.ny) : (dz >= L.nz));
                const C Tw = hi ? PV<C>::Tc(p) : PV<C>::Th(p);
                out = -val + PV<C>::omega(p) * Tw;  // anti-bounce-back
            }
        }
        // written by PULL: slot (x + e_i) of plane ibar, where the node pulls
        // ibar from; by AA_EVEN: slot (x + e_i) of plane i, where the next
        // AA_ODD half reads it; by AA_ODD: the node's own slot of plane ibar,
        // where the next AA_EVEN half reads it
        constexpr int plane = MODE == AA_EVEN ? i : o;
        const long long s = MODE == AA_ODD ? L.slot(x, y, z) : L.slot(dx, dy, dz);
        if constexpr (THERMAL) *TLBM_DBG(p, (base + ((long long)plane * L.plane + s)), 0, 1) = enc_g_step<S, C>(out, scale, salt);
        else *TLBM_DBG(p, (base + ((long long)plane * L.plane + s)), 0, 1) = enc_f_step<LS, S, C>(out, plane, scale, salt);
    } else {
        // periodic: the value reaches the image node w = wrap(x + e_i) as f_i;
        // written by PULL: slot (w - e_i) of plane i; by AA_EVEN: slot (w - e_i)
        // of plane ibar (the next AA_ODD half reads there); by AA_ODD: w's own
        // slot of plane i (the next AA_EVEN half reads there)
        const int wx = ox ? (dx < 0 ? dx + L.nx : dx - L.nx) : dx;
        const int wy = oy ? (dy < 0 ? dy + L.ny : dy - L.ny) : dy;
        const int wz = oz ? (dz < 0 ? dz + L.nz : dz - L.nz) : dz;
        constexpr int plane = MODE == AA_EVEN ? o : i;
        const long long s = MODE == AA_ODD ? L.slot(wx, wy, wz) : L.slot(wx - ex, wy - ey, wz - ez);
        if constexpr (THERMAL) *TLBM_DBG(p, (base + ((long long)plane * L.plane + s)), 0, 1) = enc_g_step<S, C>(val, scale, salt);
        else *TLBM_DBG(p, (base + ((long long)plane * L.plane + s)), 0, 1) = enc_f_step<LS, S, C>(val, plane, scale, salt);
    }
}

// ------------------------------------------------------------------ step kernel

// decode a raw stored value (already converted to C) into the flow deviation;
// with KS (keep scaled) offset storage stays in its scaled domain
template <class LF, class S, class C, bool KS>
__device__ __forceinline__ C raw_to_dev_k(C raw, int i, C inv_scale) {
    if constexpr (Storage<S>::offset) return KS ? raw : raw * inv_scale;
    else return raw - weight<LF, C>(i);
}
template <class S, class C, bool KS>
__device__ __forceinline__ C raw_to_g_k(C raw, C inv_scale) {
    if constexpr (Storage<S>::offset) return KS ? raw : raw * inv_scale;
    else return raw;
}
template <class LF, class S, class C, bool KS>
__device__ __forceinline__ S enc_f_k(C d, int i, C scale, uint32_t salt) {
    if constexpr (Storage<S>::offset) return from_c_step<S>(KS ? d : d * scale, salt);
    else return from_c_step<S>(weight<LF, C>(i) + d, salt);
}
template <class S, class C, bool KS>
__device__ __forceinline__ S enc_g_k(C g, C scale, uint32_t salt) {
    if constexpr (Storage<S>::offset) return from_c_step<S>(KS ? g : g * scale, salt);
    else return from_c_step<S>(g, salt);
}
// The VEC values a thread stores for one population, encoded as enc_f_k /
// enc_g_k would (flow: i >= 0 is its index; thermal: i < 0); 16-bit storage
// converts them two at a time (one cvt.rs per pair, bitwise the scalar result).
template <class LF, class S, class C, bool KS, int VEC>
__device__ __forceinline__ void enc_vec(const C (&v)[VEC], int i, C scale, uint32_t salt, S (&out)[VEC]) {
    constexpr bool h16 = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
    if constexpr (h16 && VEC % 2 == 0) {
        static_assert(Storage<S>::offset, "16-bit storage is offset storage");
#pragma unroll
        for (int k = 0; k < VEC; k += 2) {
            const float a = (float)(KS ? v[k] : v[k] * scale), b = (float)(KS ? v[k + 1] : v[k + 1] * scale);
            const uint32_t d = cvt_rs2<S>(b, a, salt);
            memcpy(&out[k], &d, 4);
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            out[k] = i >= 0 ? enc_f_k<LF, S, C, KS>(v[k], i, scale, salt) : enc_g_k<S, C, KS>(v[k], scale, salt);
    }
}

template <class LF, class S, class C>
__device__ __forceinline__ C raw_to_dev(C raw, int i, C inv_scale) {
    if constexpr (Storage<S>::offset) return raw * inv_scale;
    else return raw - weight<LF, C>(i);
}
template <class S, class C>
__device__ __forceinline__ C raw_to_g(C raw, C inv_scale) {
    if constexpr (Storage<S>::offset) return raw * inv_scale;
    else return raw;
}

// Pull the pre-collision populations of nodes x0 .. x0+VEC-1 whose own slot in
// plane 0 is `own`: f as deviations d_i = f_i - w_i, g as values.
template <int DIM, class S, int VEC, class C, bool KS, bool CG = false>
__device__ __forceinline__ void pull_node_vec(const S* __restrict__ own, const KParams& p, int lane,
                                              C (&f)[Lat<DIM>::F::Q][VEC], C (&g)[Lat<DIM>::G::Q][VEC]) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const C inv_scale = ScaleOf<C>::inv(p);
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        C t[VEC];
        pull_row<S, VEC, LF::e(i, 0), C, CG>(TLBM_DBG(p, (own + p.loff[i]), 1, VEC + 2), lane, t);
#pragma unroll
        for (int k = 0; k < VEC; ++k) f[i][k] = raw_to_dev_k<LF, S, C, KS>(t[k], i, inv_scale);
    });
    static_for<LG::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        C t[VEC];
        pull_row<S, VEC, LG::e(i, 0), C, CG>(TLBM_DBG(p, (own + p.loff[LF::Q + i]), 1, VEC + 2), lane, t);
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[i][k] = raw_to_g_k<S, C, KS>(t[k], inv_scale);
    });
}

// Wall and periodic rules for the nodes of a thread at the edge of the cell.
// Kept out of line: only edge threads call it, and its fully unrolled body
// would otherwise crowd the instruction cache of the hot path.
template <int DIM, class S, int VEC, class C, int MODE = PULL>
__device__ __noinline__ void edge_writes(S* __restrict__ dst, const KParams& p, int x0, int y, int z,
                                         const C* __restrict__ post, uint32_t salt) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    constexpr int QF = LF::Q, QG = LG::Q;
    const C scale = ScaleOf<C>::s(p);
    S* __restrict__ gdst = dst + (long long)QF * p.L.plane;
    for (int k = 0; k < VEC; ++k) {
        const int x = x0 + k;
        if (x >= p.L.nx) break;
        static_for<QF>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            ghost_write<LF, false, i, S, C, MODE>(dst, p, x, y, z, post[i * VEC + k], scale, salt);
        });
        static_for<QG>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            ghost_write<LG, true, i, S, C, MODE>(gdst, p, x, y, z, post[(QF + i) * VEC + k], scale, salt);
        });
    }
}

// The populations with e_x = SIDE of node k of a thread's VEC nodes, for a node
// on the x face SIDE of an inner row (y, z away from the faces) with x not
// periodic: those, and only those, leave the cell, through that face.
template <class LS, bool THERMAL, int SIDE, class S, int VEC, class C, bool KS, int MODE = PULL>
__device__ __forceinline__ void x_face(S* __restrict__ base, const KParams& p, int x, int y, int z, int k,
                                       const C (&v)[LS::Q][VEC], uint32_t salt) {
    const C scale = ScaleOf<C>::s(p);
    const C un = KS ? ScaleOf<C>::inv(p) : C(1);  // the wall rules take unscaled values
    static_for<LS::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        if constexpr (LS::e(i, 0) == SIDE) {
            C val = v[i][0];
#pragma unroll
            for (int kk = 1; kk < VEC; ++kk)
                if (k == kk) val = v[i][kk];
            ghost_write<LS, THERMAL, i, S, C, MODE>(base, p, x, y, z, KS ? val * un : val, scale, salt);
        }
    });
}

// Wall and periodic rules for the post-collision values of a thread's nodes.
// Threads holding x = 0 or x = nx - 1 of an inner row only have the x-face
// populations to place (inline); rows on a y or z face, and periodic x, take the
// general out-of-line path.
template <int DIM, class S, int VEC, class C, bool KS, int MODE = PULL>
__device__ __forceinline__ void wall_writes(S* __restrict__ dst, const KParams& p, int x0, int y, int z,
                                            const C (&f)[Lat<DIM>::F::Q][VEC], const C (&g)[Lat<DIM>::G::Q][VEC],
                                            uint32_t salt) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    constexpr int QF = LF::Q, QG = LG::Q;
    const Layout& L = p.L;
    const bool xlo = x0 == 0, xhi = x0 + VEC >= L.nx;
    const bool face_row = (y == 0) || (y == L.ny - 1) || (DIM == 3 && (z == 0 || z == L.nz - 1));
    if (face_row || ((xlo || xhi) && (p.periodic & 1))) {
        C post[(QF + QG) * VEC];
        const C un = KS ? ScaleOf<C>::inv(p) : C(1);  // the wall rules take unscaled values
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
#pragma unroll
            for (int i = 0; i < QF; ++i) post[i * VEC + k] = KS ? f[i][k] * un : f[i][k];
#pragma unroll
            for (int i = 0; i < QG; ++i) post[(QF + i) * VEC + k] = KS ? g[i][k] * un : g[i][k];
        }
        edge_writes<DIM, S, VEC, C, MODE>(dst, p, x0, y, z, post, salt);
        return;
    }
    S* __restrict__ gdst = dst + (long long)QF * L.plane;
    if (xlo) {
        x_face<LF, false, -1, S, VEC, C, KS, MODE>(dst, p, 0, y, z, 0, f, salt);
        x_face<LG, true, -1, S, VEC, C, KS, MODE>(gdst, p, 0, y, z, 0, g, salt);
    }
    if (xhi) {
        const int k = L.nx - 1 - x0;
        x_face<LF, false, 1, S, VEC, C, KS, MODE>(dst, p, L.nx - 1, y, z, k, f, salt);
        x_face<LG, true, 1, S, VEC, C, KS, MODE>(gdst, p, L.nx - 1, y, z, k, g, salt);
    }
}

// One thread updates VEC consecutive nodes of one row.  blockDim.x must be a
// multiple of 32 so that a warp covers 32*VEC consecutive nodes of one row.
// Body of the step for the block at grid position (bx, by, bz) of one cell.
template <int DIM, class S, int VEC, bool TRT, bool CG = false>
__device__ __forceinline__ void step_block(const S* __restrict__ src, S* __restrict__ dst, const KParams& p, int bx,
                                           int by, int bz) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    constexpr int QF = LF::Q, QG = LG::Q;
    const Layout& L = p.L;
    const int lane = threadIdx.x & 31;
    const int y = by * blockDim.y + threadIdx.y;
    const int z = DIM == 3 ? bz : 0;
    if (y >= L.ny) return;  // uniform across the warp
    const int x0 = (bx * blockDim.x + threadIdx.x) * VEC;
    if (x0 - lane * VEC >= L.nx) return;  // the whole warp lies past the row end
    const int x0ld = min(x0, p.xmax_load);
    const C scale = ScaleOf<C>::s(p);
    const long long row = L.row(y, z);
    constexpr bool KS = TRT && Storage<S>::offset;  // TRT works on the stored, scaled values
    const uint32_t tcount = step_count<S, CG>(src, 0);
    const uint32_t salt = step_salt(tcount);
    advance_count<S>(dst, 0, tcount, bx == 0 && by == 0 && bz == 0 && threadIdx.x == 0 && threadIdx.y == 0);

    C f[QF][VEC], g[QG][VEC];
    pull_node_vec<DIM, S, VEC, C, KS, CG>(src + row + x0ld, p, lane, f, g);

    collide_vec<DIM, TRT, C, collide_scaled<S, TRT>, VEC>(f, g, p);

    if (x0 >= L.nx) return;
    S* __restrict__ own = dst + row + x0;
    if (x0 + VEC <= L.nx) {
        static_for<QF>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            S v[VEC];
            enc_vec<LF, S, C, KS, VEC>(f[i], i, scale, salt, v);
            st_vec<S, VEC>(TLBM_DBG(p, (own + p.soff[i]), 0, VEC), v);
        });
        static_for<QG>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            S v[VEC];
            enc_vec<LF, S, C, KS, VEC>(g[i], -1, scale, salt, v);
            st_vec<S, VEC>(TLBM_DBG(p, (own + p.soff[QF + i]), 0, VEC), v);
        });
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if (x0 + k < L.nx) {
                static_for<QF>([&](auto ii) {
                    constexpr int i = decltype(ii)::value;
                    *TLBM_DBG(p, (own + (p.soff[i] + k)), 0, 1) = enc_f_k<LF, S, C, KS>(f[i][k], i, scale, salt);
                });
                static_for<QG>([&](auto ii) {
                    constexpr int i = decltype(ii)::value;
                    *TLBM_DBG(p, (own + (p.soff[QF + i] + k)), 0, 1) = enc_g_k<S, C, KS>(g[i][k], scale, salt);
                });
            }
        }
    }

    // wall and periodic rules for values that leave the cell
    wall_writes<DIM, S, VEC, C, KS>(dst, p, x0, y, z, f, g, salt);
}

// ------------------------------------------------------------------ in-place (AA) streaming

// Push the post-collision values v[k] of nodes x0 + k (direction with
// x-component EX) to x0 + k + EX.  `q` points at column x0 of the target row;
// `enc` turns a value into its stored form.  The aligned vector at q receives
// the values of nodes x0 - EX .. x0 + VEC - 1 - EX through a warp shuffle; the
// one value that crosses into the neighbouring warp's columns is stored by the
// edge lane as a scalar, and only values of nodes inside the row are written
// (the in-place update must leave every other slot to its own writer).  All 32
// lanes must call this together.
template <class S, int VEC, int EX, class C, class Enc>
__device__ __forceinline__ void push_row(S* q, int lane, int x0, int nx, const C (&v)[VEC], Enc enc) {
    if constexpr (VEC == 1) {
        if (x0 < nx) q[EX] = enc(v[0]);
        return;
    }
    C w[VEC];
    if constexpr (EX == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) w[k] = v[k];
    } else if constexpr (EX == 1) {
        w[0] = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
#pragma unroll
        for (int k = 1; k < VEC; ++k) w[k] = v[k - 1];
    } else {
#pragma unroll
        for (int k = 0; k < VEC - 1; ++k) w[k] = v[k + 1];
        w[VEC - 1] = __shfl_down_sync(0xffffffffu, v[0], 1);
    }
    if (x0 >= nx) return;
    // every source node x0 + k - EX inside the row and held by this warp
    const bool whole = EX == 0 ? x0 + VEC <= nx : (EX == 1 ? (lane != 0 && x0 + VEC - 1 <= nx) : (lane != 31 && x0 + VEC < nx));
    if (whole) {
        S t[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) t[k] = enc(w[k]);
        st_vec<S, VEC>(q, t);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const int src = x0 + k - EX;
            const bool held = !(EX == 1 && k == 0 && lane == 0) && !(EX == -1 && k == VEC - 1 && lane == 31);
            if (held && src >= 0 && src < nx) q[k] = enc(w[k]);
        }
    }
    if constexpr (EX == 1) {
        if (lane == 31 && x0 + VEC - 1 < nx) q[VEC] = enc(v[VEC - 1]);
    } else if constexpr (EX == -1) {
        if (lane == 0) q[-1] = enc(v[0]);
    }
}

// One half of an in-place step pair for the block at (bx, by, bz): MODE =
// AA_EVEN reads every node's own slots and writes the post-collision values back
// into the slots of the opposite directions; MODE = AA_ODD reads f_i from
// (x - e_i) of plane ibar and pushes f+_i to (x + e_i) of plane i.  The
// collision is the one of step_block; the wall rules go where the next half
// reads them (ghost_write).  One buffer: `buf` is read and written.
template <int DIM, class S, int VEC, bool TRT, int MODE>
__device__ __forceinline__ void step_block_aa(S* buf, const KParams& p, int bx, int by, int bz) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    using C = typename Storage<S>::C;
    constexpr int QF = LF::Q, QG = LG::Q;
    const Layout& L = p.L;
    const int lane = threadIdx.x & 31;
    const int y = by * blockDim.y + threadIdx.y;
    const int z = DIM == 3 ? bz : 0;
    if (y >= L.ny) return;  // uniform across the warp
    const int x0 = (bx * blockDim.x + threadIdx.x) * VEC;
    if (x0 - lane * VEC >= L.nx) return;  // the whole warp lies past the row end
    const int x0ld = min(x0, p.xmax_load);
    const C scale = ScaleOf<C>::s(p);
    const C inv_scale = ScaleOf<C>::inv(p);
    const long long row = L.row(y, z);
    constexpr bool KS = TRT && Storage<S>::offset;
    // the step counter alternates between words 0 and 1 of the single buffer
    const uint32_t tcount = step_count<S>(buf, MODE == AA_ODD ? 1 : 0);
    const uint32_t salt = step_salt(tcount);
    advance_count<S>(buf, MODE == AA_ODD ? 0 : 1, tcount,
                     bx == 0 && by == 0 && bz == 0 && threadIdx.x == 0 && threadIdx.y == 0);

    C f[QF][VEC], g[QG][VEC];
    const S* own_ld = buf + row + x0ld;
    static_for<QF>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        C t[VEC];
        if constexpr (MODE == AA_EVEN) pull_row<S, VEC, 0, C>(TLBM_DBG(p, (own_ld + off_shift<i>(p)), 1, VEC + 2), lane, t);
        else pull_row<S, VEC, LF::e(i, 0), C>(TLBM_DBG(p, (own_ld + off_shift<LF::opp(i), -LF::e(i, 1), -LF::e(i, 2)>(p)), 1, VEC + 2),
                                               lane, t);
#pragma unroll
        for (int k = 0; k < VEC; ++k) f[i][k] = raw_to_dev_k<LF, S, C, KS>(t[k], i, inv_scale);
    });
    static_for<QG>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        C t[VEC];
        if constexpr (MODE == AA_EVEN) pull_row<S, VEC, 0, C>(TLBM_DBG(p, (own_ld + off_shift<QF + i>(p)), 1, VEC + 2), lane, t);
        else pull_row<S, VEC, LG::e(i, 0), C>(
                TLBM_DBG(p, (own_ld + off_shift<QF + LG::opp(i), -LG::e(i, 1), -LG::e(i, 2)>(p)), 1, VEC + 2), lane, t);
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[i][k] = raw_to_g_k<S, C, KS>(t[k], inv_scale);
    });

    // 2D: constants formed on the host (1.6 % faster for 2D FP32 on GB300, 1 %
    // slower for 3D FP16)
    collide_vec<DIM, TRT, C, collide_scaled<S, TRT>, VEC, DIM == 2>(f, g, p);

    S* own = buf + row + x0;
    if constexpr (MODE == AA_EVEN) {
        if (x0 >= L.nx) return;
        // own slots, opposite planes
        if (x0 + VEC <= L.nx) {
            static_for<QF>([&](auto ii) {
                constexpr int i = decltype(ii)::value;
                S v[VEC];
                enc_vec<LF, S, C, KS, VEC>(f[i], i, scale, salt, v);
                st_vec<S, VEC>(TLBM_DBG(p, (own + off_shift<LF::opp(i)>(p)), 0, VEC), v);
            });
            static_for<QG>([&](auto ii) {
                constexpr int i = decltype(ii)::value;
                S v[VEC];
                enc_vec<LF, S, C, KS, VEC>(g[i], -1, scale, salt, v);
                st_vec<S, VEC>(TLBM_DBG(p, (own + off_shift<QF + LG::opp(i)>(p)), 0, VEC), v);
            });
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                if (x0 + k < L.nx) {
                    static_for<QF>([&](auto ii) {
                        constexpr int i = decltype(ii)::value;
                        *TLBM_DBG(p, (own + (off_shift<LF::opp(i)>(p) + k)), 0, 1) = enc_f_k<LF, S, C, KS>(f[i][k], i, scale, salt);
                    });
                    static_for<QG>([&](auto ii) {
                        constexpr int i = decltype(ii)::value;
                        *TLBM_DBG(p, (own + (off_shift<QF + LG::opp(i)>(p) + k)), 0, 1) = enc_g_k<S, C, KS>(g[i][k], scale, salt);
                    });
                }
            }
        }
    } else {
        // push to x + e_i of plane i (all lanes take part in the shuffles; lanes
        // past the row end store nothing)
#ifdef TLBM_DEBUG_BOUNDS
#define TLBM_AIM(q) (x0 < L.nx ? TLBM_DBG(p, (q), 1, VEC + 2) : (q))
#else
#define TLBM_AIM(q) (q)
#endif
        static_for<QF>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            push_row<S, VEC, LF::e(i, 0), C>(TLBM_AIM((own + off_shift<i, LF::e(i, 1), LF::e(i, 2)>(p))), lane, x0, L.nx, f[i],
                                             [&](C d) { return enc_f_k<LF, S, C, KS>(d, i, scale, salt); });
        });
        static_for<QG>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            push_row<S, VEC, LG::e(i, 0), C>(TLBM_AIM((own + off_shift<QF + i, LG::e(i, 1), LG::e(i, 2)>(p))), lane, x0, L.nx, g[i],
                                             [&](C d) { return enc_g_k<S, C, KS>(d, scale, salt); });
        });
#undef TLBM_AIM
        if (x0 >= L.nx) return;
    }
    wall_writes<DIM, S, VEC, C, KS, MODE>(buf, p, x0, y, z, f, g, salt);
}

template <int DIM, class S, int VEC, bool TRT, int MODE>
__global__ void step_kernel_aa(S* buf, const KParams p) {
    step_block_aa<DIM, S, VEC, TRT, MODE>(buf, p, blockIdx.x, blockIdx.y, blockIdx.z);
}
template <int DIM, class S, int VEC, bool TRT, int MODE>
__global__ void __maxnreg__(96) step_kernel_aa_r96(S* buf, const KParams p) {
    step_block_aa<DIM, S, VEC, TRT, MODE>(buf, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ------------------------------------------------------------------ software-pipelined rows

// The raw stored values one thread pulls for one row: the aligned vector of
// every population and, for the warp's edge lane, the one element beyond it.
template <int DIM, class S, int VEC>
struct RawRow {
    static constexpr int Q = Lat<DIM>::F::Q + Lat<DIM>::G::Q;
    S v[Q][VEC];
    S h[Q];
};

// Issue the loads of one row (no use of the loaded values yet).
template <int DIM, class S, int VEC>
__device__ __forceinline__ void fetch_row(const S* __restrict__ own, const KParams& p, int lane,
                                          RawRow<DIM, S, VEC>& r) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    static_for<LF::Q + LG::Q>([&](auto jj) {
        constexpr int j = decltype(jj)::value;
        constexpr int ex = j < LF::Q ? LF::e(j < LF::Q ? j : 0, 0) : LG::e(j < LF::Q ? 0 : j - LF::Q, 0);
        const S* __restrict__ q = TLBM_DBG(p, (own + p.loff[j]), 1, VEC + 2);
        if constexpr (VEC == 1) {
            r.v[j][0] = ld_one<S, false>(q - ex);
        } else {
            ld_vec<S, VEC>(q, r.v[j]);
            if constexpr (ex == 1) {
                if (lane == 0) r.h[j] = ld_one<S, false>(q - 1);
            } else if constexpr (ex == -1) {
                if (lane == 31) r.h[j] = ld_one<S, false>(q + VEC);
            }
        }
    });
}

// Shift, convert and decode a fetched row (all 32 lanes together).
template <int DIM, class S, int VEC, class C, bool KS>
__device__ __forceinline__ void decode_row(const RawRow<DIM, S, VEC>& r, const KParams& p, int lane,
                                           C (&f)[Lat<DIM>::F::Q][VEC], C (&g)[Lat<DIM>::G::Q][VEC]) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const C inv_scale = ScaleOf<C>::inv(p);
    static_for<LF::Q + LG::Q>([&](auto jj) {
        constexpr int j = decltype(jj)::value;
        constexpr bool flow = j < LF::Q;
        constexpr int ex = flow ? LF::e(flow ? j : 0, 0) : LG::e(flow ? 0 : j - LF::Q, 0);
        C t[VEC];
        if constexpr (VEC == 1 || ex == 0) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) t[k] = to_c<C>(r.v[j][k]);
        } else if constexpr (ex == 1) {
            C left = __shfl_up_sync(0xffffffffu, to_c<C>(r.v[j][VEC - 1]), 1);
            if (lane == 0) left = to_c<C>(r.h[j]);
            t[0] = left;
#pragma unroll
            for (int k = 1; k < VEC; ++k) t[k] = to_c<C>(r.v[j][k - 1]);
        } else {
            C right = __shfl_down_sync(0xffffffffu, to_c<C>(r.v[j][0]), 1);
            if (lane == 31) right = to_c<C>(r.h[j]);
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) t[k] = to_c<C>(r.v[j][k + 1]);
            t[VEC - 1] = right;
        }
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if constexpr (flow) f[j][k] = raw_to_dev_k<LF, S, C, KS>(t[k], j, inv_scale);
            else g[j - LF::Q][k] = raw_to_g_k<S, C, KS>(t[k], inv_scale);
        }
    });
}

// Collide and store one decoded row (all lanes participate; stores predicated).
template <int DIM, class S, int VEC, bool TRT, class C, bool KS>
__device__ __forceinline__ void finish_row(S* __restrict__ dst, const KParams& p, int x0, int y, int z,
                                           long long row, C (&f)[Lat<DIM>::F::Q][VEC],
                                           C (&g)[Lat<DIM>::G::Q][VEC], uint32_t salt) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    constexpr int QF = LF::Q, QG = LG::Q;
    const Layout& L = p.L;
    const C scale = ScaleOf<C>::s(p);
    collide_vec<DIM, TRT, C, collide_scaled<S, TRT>, VEC>(f, g, p);
    if (x0 >= L.nx) return;
    S* __restrict__ own = dst + row + x0;
    if (x0 + VEC <= L.nx) {
        static_for<QF>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            S v[VEC];
            enc_vec<LF, S, C, KS, VEC>(f[i], i, scale, salt, v);
            st_vec<S, VEC>(TLBM_DBG(p, (own + p.soff[i]), 0, VEC), v);
        });
        static_for<QG>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            S v[VEC];
            enc_vec<LF, S, C, KS, VEC>(g[i], -1, scale, salt, v);
            st_vec<S, VEC>(TLBM_DBG(p, (own + p.soff[QF + i]), 0, VEC), v);
        });
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if (x0 + k < L.nx) {
                static_for<QF>([&](auto ii) {
                    constexpr int i = decltype(ii)::value;
                    *TLBM_DBG(p, (own + (p.soff[i] + k)), 0, 1) = enc_f_k<LF, S, C, KS>(f[i][k], i, scale, salt);
                });
                static_for<QG>([&](auto ii) {
                    constexpr int i = decltype(ii)::value;
                    *TLBM_DBG(p, (own + (p.soff[QF + i] + k)), 0, 1) = enc_g_k<S, C, KS>(g[i][k], scale, salt);
                });
            }
        }
    }
    wall_writes<DIM, S, VEC, C, KS>(dst, p, x0, y, z, f, g, salt);
}

// ROWS consecutive rows per thread, software-pipelined: the loads of the next
// row are issued before the current row is collided, so every warp keeps loads
// in flight while it computes.
// Body of the software-pipelined kernel for the block at grid position (bx, by, bz).
template <int DIM, class S, int VEC, bool TRT, int ROWS>
__device__ __forceinline__ void step_rows_block(const S* __restrict__ src, S* __restrict__ dst, const KParams& p,
                                                int bx, int by, int bz) {
    using C = typename Storage<S>::C;
    constexpr int QF = Lat<DIM>::F::Q, QG = Lat<DIM>::G::Q;
    constexpr bool KS = TRT && Storage<S>::offset;
    const Layout& L = p.L;
    const int lane = threadIdx.x & 31;
    const int y0 = (by * blockDim.y + threadIdx.y) * ROWS;
    const int z = DIM == 3 ? bz : 0;
    if (y0 >= L.ny) return;  // uniform across the warp
    const int x0 = (bx * blockDim.x + threadIdx.x) * VEC;
    if (x0 - lane * VEC >= L.nx) return;  // the whole warp lies past the row end
    const int x0ld = min(x0, p.xmax_load);
    const long long row0 = L.row(y0, z);
    const uint32_t tcount = step_count<S>(src, 0);
    const uint32_t salt = step_salt(tcount);
    advance_count<S>(dst, 0, tcount, bx == 0 && by == 0 && bz == 0 && threadIdx.x == 0 && threadIdx.y == 0);
    RawRow<DIM, S, VEC> A, B;
    fetch_row<DIM, S, VEC>(src + row0 + x0ld, p, lane, A);
#pragma unroll
    for (int r = 0; r < ROWS; r += 2) {
        const int ya = y0 + r, yb = ya + 1;
        const long long rowa = row0 + (long long)r * L.P;
        if (r + 1 < ROWS && yb < L.ny) fetch_row<DIM, S, VEC>(src + rowa + L.P + x0ld, p, lane, B);
        {
            C f[QF][VEC], g[QG][VEC];
            decode_row<DIM, S, VEC, C, KS>(A, p, lane, f, g);
            finish_row<DIM, S, VEC, TRT, C, KS>(dst, p, x0, ya, z, rowa, f, g, salt);
        }
        if (r + 1 >= ROWS || yb >= L.ny) break;
        if (r + 2 < ROWS && yb + 1 < L.ny) fetch_row<DIM, S, VEC>(src + rowa + 2 * L.P + x0ld, p, lane, A);
        {
            C f[QF][VEC], g[QG][VEC];
            decode_row<DIM, S, VEC, C, KS>(B, p, lane, f, g);
            finish_row<DIM, S, VEC, TRT, C, KS>(dst, p, x0, yb, z, rowa + L.P, f, g, salt);
        }
        if (yb + 1 >= L.ny) break;
    }
}

template <int DIM, class S, int VEC, bool TRT, int ROWS>
__global__ void step_kernel_rows(const S* __restrict__ src, S* __restrict__ dst, const KParams p) {
    step_rows_block<DIM, S, VEC, TRT, ROWS>(src, dst, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int DIM, class S, int VEC, bool TRT>
__global__ void step_kernel(const S* __restrict__ src, S* __restrict__ dst, const KParams p) {
    step_block<DIM, S, VEC, TRT>(src, dst, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The same kernels held to 96 registers per thread.  For the 3D two-node
// FP16/BF16 variants the extra resident warps (21 instead of 16 per SM with
// one-warp blocks) outweigh the few values the cap spills: 45.1 instead of
// 43.0 GLUPS at 385^3 on GB300, same box, same process.
template <int DIM, class S, int VEC, bool TRT>
__global__ void __maxnreg__(96) step_kernel_r96(const S* __restrict__ src, S* __restrict__ dst, const KParams p) {
    step_block<DIM, S, VEC, TRT>(src, dst, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ------------------------------------------------------------------ diagnostics

// Element index (within the planes of set LS) of the pre-collision value
// f_j(x) of the state, in the order p.state names.
template <class LS, int j>
__device__ __forceinline__ long long pre_index(const KParams& p, int x, int y, int z) {
    const Layout& L = p.L;
    constexpr int ex = LS::e(j, 0), ey = LS::e(j, 1), ez = LS::e(j, 2);
    if (p.state == 1) return (long long)j * L.plane + L.slot(x, y, z);
    const int plane = p.state == 2 ? LS::opp(j) : j;
    return (long long)plane * L.plane + L.slot(x - ex, y - ey, z - ez);
}

// Canonical pre-collision populations of one node (scalar reads).
template <int DIM, class S, class C>
__device__ __forceinline__ void pull_node(const S* __restrict__ src, const KParams& p, int x, int y, int z,
                                          C (&f)[Lat<DIM>::F::Q], C (&g)[Lat<DIM>::G::Q]) {
    using LF = typename Lat<DIM>::F;
    using LG = typename Lat<DIM>::G;
    const Layout& L = p.L;
    const C inv_scale = ScaleOf<C>::inv(p);
    const S* __restrict__ gsrc = src + (long long)LF::Q * L.plane;
    static_for<LF::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const C raw = to_c<C>(*TLBM_DBG(p, (src + pre_index<LF, i>(p, x, y, z)), 0, 1));
        f[i] = raw_to_dev<LF, S, C>(raw, i, inv_scale);
    });
    static_for<LG::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const C raw = to_c<C>(*TLBM_DBG(p, (gsrc + pre_index<LG, i>(p, x, y, z)), 0, 1));
        g[i] = raw_to_g<S, C>(raw, inv_scale);
    });
}

// Per-node terms of the reductions (a6): u_h T, 1/2 rho |u|^2, rho, |u|^2, T,
// formed in the storage's collision precision (FP64 storage: FP64; otherwise
// FP32, the precision the state was computed in) and handed over in FP64 for
// the FP64 sums.
template <int DIM, class S>
__device__ __forceinline__ void node_terms(const S* __restrict__ buf, const KParams& p, int x, int y, int z,
                                           double (&t)[5]) {
    using C = typename Storage<S>::C;
    C f[Lat<DIM>::F::Q], g[Lat<DIM>::G::Q], r, u[3], T;
    pull_node<DIM, S, C>(buf, p, x, y, z, f, g);
    node_macros<DIM, C>(f, g, p, r, u, T);
    const C u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    t[0] = (double)(u[p.heat_axis] * T);
    t[1] = (double)(C(0.5) * r * u2);
    t[2] = (double)r;
    t[3] = (double)u2;
    t[4] = (double)T;
}

}  // namespace tlbm
