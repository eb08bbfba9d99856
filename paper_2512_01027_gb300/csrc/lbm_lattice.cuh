// Lattice tables for the device path (D2Q9, D3Q19, D3Q27; T = 1/3, Sec. II).
//
// Direction order: rest first, then pairs (c, -c): axis directions, then face
// diagonals, then (D3Q27) corners.  Weights: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3,
// 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.  Everything here is constexpr so
// that per-direction coefficients fold into the instruction stream.
#pragma once

#include <cstdint>
#include <utility>

namespace lbm {

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

struct D2Q9 {
    static constexpr int id = 0, D = 2, Q = 9;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

namespace detail {
__host__ __device__ constexpr int c3(int i, int a)
{
    constexpr int t[27][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
        {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
        {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    return t[i][a];
}
}  // namespace detail

struct D3Q19 {
    static constexpr int id = 1, D = 3, Q = 19;
    __host__ __device__ static constexpr int c(int i, int a) { return detail::c3(i, a); }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

struct D3Q27 {
    static constexpr int id = 2, D = 3, Q = 27;
    __host__ __device__ static constexpr int c(int i, int a) { return detail::c3(i, a); }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
};

// Opposite direction: pairs (c, -c) sit at (2k-1, 2k).
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

}  // namespace lbm
