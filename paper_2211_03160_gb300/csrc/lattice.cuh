// Lattice tables and moment-space algebra for the CUDA path.
//
// Velocity sets (Fig. 1 of Xu & Li): D2Q9 + D2Q5 in 2D, D3Q19 + D3Q7 in 3D.
// D2Q9 numbering follows the halo sets of §3.1 (directions 2, 5, 6 move +y;
// 4, 7, 8 move -y).  Moment bases: Lallemand & Luo (2000) for D2Q9,
// d'Humieres et al. (2002) for D3Q19; the thermal bases are
// [1, ex, ey, 5|e|^2-4, ex^2-ey^2] (D2Q5) and
// [1, ex, ey, ez, 7|e|^2-6, 3ex^2-|e|^2, ey^2-ez^2] (D3Q7).
// All rows are mutually orthogonal, so M^-1 = M^T diag(1/|row|^2).
//
// Everything here is constexpr so that the unrolled moment transforms in the
// kernels reduce to additions of the non-zero integer coefficients.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace tlbm {

template <int N, class F, int... I>
__host__ __device__ __forceinline__ constexpr void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
// Calls f(std::integral_constant<int, i>) for i = 0 .. N-1, fully unrolled.
template <int N, class F>
__host__ __device__ __forceinline__ constexpr void static_for(F&& f) {
    static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------------------ 2D sets
struct D2Q9 {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return E[i][a];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int O[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return O[i];
    }
    // weights as exact rationals: numerator / 36
    __host__ __device__ static constexpr int w36(int i) {
        constexpr int W[9] = {16, 4, 4, 4, 4, 1, 1, 1, 1};
        return W[i];
    }
    // moment rows: rho, e, eps, jx, qx, jy, qy, pxx, pxy
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int T[9][9] = {
            {1, 1, 1, 1, 1, 1, 1, 1, 1},          {-4, -1, -1, -1, -1, 2, 2, 2, 2},
            {4, -2, -2, -2, -2, 1, 1, 1, 1},      {0, 1, 0, -1, 0, 1, -1, -1, 1},
            {0, -2, 0, 2, 0, 1, -1, -1, 1},       {0, 0, 1, 0, -1, 1, 1, -1, -1},
            {0, 0, -2, 0, 2, 1, 1, -1, -1},       {0, 1, -1, 1, -1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 1, -1, 1, -1}};
        return T[k][i];
    }
};

struct D2Q5 {
    static constexpr int Q = 5;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
        return E[i][a];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int O[5] = {0, 3, 4, 1, 2};
        return O[i];
    }
    // rows: T, jx, jy, e (5|e|^2 - 4), nu (ex^2 - ey^2)
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int T[5][5] = {{1, 1, 1, 1, 1},
                                 {0, 1, 0, -1, 0},
                                 {0, 0, 1, 0, -1},
                                 {-4, 1, 1, 1, 1},
                                 {0, 1, -1, 1, -1}};
        return T[k][i];
    }
};

// ------------------------------------------------------------------ 3D sets
struct D3Q19 {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
        return E[i][a];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int O[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return O[i];
    }
    __host__ __device__ static constexpr int w36(int i) {
        constexpr int W[19] = {12, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
        return W[i];
    }
    // rows: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww,
    //       pxy, pyz, pxz, mx, my, mz
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int T[19][19] = {
            // 0  1   2   3   4   5   6   7   8   9  10  11  12  13  14  15  16  17  18
            {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
            {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
            {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
            {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
            {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
            {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, -4, 4, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
            {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
            {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
            {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
            {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
            {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, -1, 1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1}};
        return T[k][i];
    }
};

struct D3Q7 {
    static constexpr int Q = 7;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int E[7][3] = {{0, 0, 0},  {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                 {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        return E[i][a];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int O[7] = {0, 2, 1, 4, 3, 6, 5};
        return O[i];
    }
    // rows: T, jx, jy, jz, e (7|e|^2 - 6), 3ex^2 - |e|^2, ey^2 - ez^2
    __host__ __device__ static constexpr int M(int k, int i) {
        constexpr int T[7][7] = {{1, 1, 1, 1, 1, 1, 1},     {0, 1, -1, 0, 0, 0, 0},
                                 {0, 0, 0, 1, -1, 0, 0},    {0, 0, 0, 0, 0, 1, -1},
                                 {-6, 1, 1, 1, 1, 1, 1},    {0, 2, 2, -1, -1, -1, -1},
                                 {0, 0, 0, 1, 1, -1, -1}};
        return T[k][i];
    }
};

template <class L>
__host__ __device__ constexpr int row_norm2(int k) {
    int s = 0;
    for (int i = 0; i < L::Q; ++i) s += L::M(k, i) * L::M(k, i);
    return s;
}

// m = M x  (x in population space, m in moment space), unrolled over the
// non-zero integer coefficients.
template <class L, class C>
__device__ __forceinline__ void moments(const C (&x)[L::Q], C (&m)[L::Q]) {
    static_for<L::Q>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        C acc = C(0);
        static_for<L::Q>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            constexpr int c = L::M(k, i);
            if constexpr (c == 1) acc += x[i];
            else if constexpr (c == -1) acc -= x[i];
            else if constexpr (c != 0) acc += C(c) * x[i];
        });
        m[k] = acc;
    });
}

// x = M^-1 m = M^T diag(1/|row|^2) m
template <class L, class C>
__device__ __forceinline__ void populations(const C (&m)[L::Q], C (&x)[L::Q]) {
    C ms[L::Q];
    static_for<L::Q>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr int n2 = row_norm2<L>(k);
        ms[k] = m[k] * (C(1) / C(n2));
    });
    static_for<L::Q>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        C acc = C(0);
        static_for<L::Q>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            constexpr int c = L::M(k, i);
            if constexpr (c == 1) acc += ms[k];
            else if constexpr (c == -1) acc -= ms[k];
            else if constexpr (c != 0) acc += C(c) * ms[k];
        });
        x[i] = acc;
    });
}

}  // namespace tlbm
