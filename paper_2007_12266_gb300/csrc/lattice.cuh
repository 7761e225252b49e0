// Compile-time lattice constants of the color-gradient LBM (Sec. 3.1).
//
// D3Q19 for momentum (c_s^2 = 1/3, weights 1/3, 1/18, 1/36), its first seven
// directions as D3Q7 for the two component densities (c_s^2 = 2/9, weights
// 1/3, 1/9), and d'Humieres' orthogonal moment basis for the MRT collision.
// Every table is a constexpr function so that fully unrolled loops in the
// kernels fold each entry into an immediate.
#pragma once

namespace lbm {

constexpr int Q19 = 19;
constexpr int Q7 = 7;

// Eq. d3q19: rest; faces +-x, +-y, +-z; xy edges (++, --, +-, -+);
// xz edges (++, --, +-, -+); yz edges (++, --, +-, -+). Opposites are
// adjacent: (1,2), (3,4), ..., (17,18).
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[Q19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[Q19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[Q19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
// Offset of voxel x + xi_q from x in a padded grid with strides 1, px, pxpy
// (with a compile-time q the direction's components fold into the code).
__host__ __device__ constexpr int stencil_offset(int q, int px, int pxpy);
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr int stencil_offset(int q, int px, int pxpy) {
    return cx(q) + cy(q) * px + cz(q) * pxpy;
}
__host__ __device__ constexpr int c2(int q) { return cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q); }

// D3Q19 weight t_q and D3Q7 weight w_q
__host__ __device__ constexpr float t19(int q) {
    return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr float w7(int q) { return q == 0 ? 1.0f / 3.0f : 1.0f / 9.0f; }

// Color-gradient stencil weight: C = sum_q g_q xi_q phi(x + xi_q) with g = 1 on
// faces and 1/2 on edges (= 18 t_q), which is 6 grad(phi) for smooth phi; with
// the alpha|C|/2 stress terms this is the scaling that gives sigma_ab = 6 alpha.
__host__ __device__ constexpr float grad_w(int q) { return q == 0 ? 0.0f : (q <= 6 ? 1.0f : 0.5f); }

// d'Humieres moment basis, row k evaluated at velocity q (integers).
// Order: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww,
// pxy, pyz, pxz, mx, my, mz.
__host__ __device__ constexpr int mrow(int k, int q) {
    const int x = cx(q), y = cy(q), z = cz(q), s = c2(q);
    return k == 0 ? 1
         : k == 1 ? 19 * s - 30
         : k == 2 ? (21 * s * s - 53 * s + 24) / 2
         : k == 3 ? x
         : k == 4 ? (5 * s - 9) * x
         : k == 5 ? y
         : k == 6 ? (5 * s - 9) * y
         : k == 7 ? z
         : k == 8 ? (5 * s - 9) * z
         : k == 9 ? 3 * x * x - s
         : k == 10 ? (3 * s - 5) * (3 * x * x - s)
         : k == 11 ? y * y - z * z
         : k == 12 ? (3 * s - 5) * (y * y - z * z)
         : k == 13 ? x * y
         : k == 14 ? y * z
         : k == 15 ? x * z
         : k == 16 ? (y * y - z * z) * x
         : k == 17 ? (z * z - x * x) * y
         : (x * x - y * y) * z;
}

// Rows 1 and 2 with their density part removed (e + 11 rho, eps - 3 rho):
// the collision works with these to avoid cancelling two O(10) numbers.
__host__ __device__ constexpr int mrow_shifted(int k, int q) {
    return k == 1 ? mrow(1, q) + 11 : (k == 2 ? mrow(2, q) - 3 : mrow(k, q));
}

__host__ __device__ constexpr int mnorm(int k) {
    int s = 0;
    for (int q = 0; q < Q19; ++q) s += mrow(k, q) * mrow(k, q);
    return s;
}

// Inverse basis: M^-1[q][k] = M[k][q] / |row k|^2 (rows are orthogonal).
__host__ __device__ constexpr float minv(int q, int k) {
    return static_cast<float>(mrow(k, q)) / static_cast<float>(mnorm(k));
}

}  // namespace lbm

#include <utility>

namespace lbm {

// Compile-time loop: f(std::integral_constant<int, I>{}) for I in [B, B+N).
template <int B, class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, B + Is>{}), ...);
}
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    static_for_impl<B>(f, std::make_integer_sequence<int, E - B>{});
}

}  // namespace lbm
