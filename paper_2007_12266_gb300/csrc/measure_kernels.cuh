// Per-site measures and block reductions shared by the single-domain and
// batched measure kernels (basic analysis of Sec. 4, integral measures of the
// table of integral measures in Sec. 3.4).
#pragma once

#include "step_kernels.cuh"

namespace lbm {

// Current-state populations of site n at AA parity PAR (the values the next
// step collides), in canonical order.
template <int PAR, class S>
__device__ __forceinline__ void load_site(const DomainView& d, int n, float (&f)[Q19], float (&a)[Q7],
                                          float (&b)[Q7]) {
    const int v = d.site_vox[n];
    int nb[Q19];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
        });
    }
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        f[q] = S::template ld_f<q>(d.f, read_slot<PAR, q>(d, n, nb));
        if constexpr (S::kRef) f[q] = fmaf(t19(q), d.drho[f_ref_read<PAR, q>(n, nb)], f[q]);
    });
    load_components<PAR, S>(d, n, v, nb, a, b);
}

// Per-thread accumulator of per-site fp32 quantities: compensated fp32
// (TwoSum: the exact rounding error of every addition is carried in lo, whose
// own rounding bounds the error at about k^2 2^-48 of the sum of magnitudes for
// k sites). The measure grid keeps k <= 64 (at most 1.5e-11), far below the
// fp32 state's own rounding; the block and global reductions are fp64.
// Accumulating in fp64 directly gives the same results but takes 3.3 times
// longer on this GPU, whose fp64 pipe is slow (460 against 140 us per analysis
// at 256^3).
struct AccF64 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (x - bp);
        hi = s;
        lo += err;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Add site n's contributions to the NSUM compensated accumulators.
// Sum layout (NSUM = 27):
//  0 Na, 1 Nb, 2 rho, 3 #(phi > 0), 4-6 u, 7-9 (Na/N) u, 10-12 (Nb/N) u,
//  13 M_a, 14 M_b, 15-17 P_a, 18-20 P_b, 21 K_a, 22 K_b, 23 p over A,
//  24 p over B, 25 #non-finite, 26 #sites with a component density below -1e-2
//  or a non-positive total density (small negative densities are legitimate
//  next to interfaces and are not counted)
template <int PAR, class S>
__device__ __forceinline__ void measure_site(const DomainView& d, int n, AccF64 (&acc)[NSUM]) {
    const float hfx = 0.5f * d.fx, hfy = 0.5f * d.fy, hfz = 0.5f * d.fz;
    float f[Q19], a[Q7], b[Q7];
    load_site<PAR, S>(d, n, f, a, b);
    // per-site quantities in fp32, accumulated in fp64
    float Na = 0.0f, Nb = 0.0f, rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    bool finite = true;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        finite = finite && isfinite(f[q]);
        rho += f[q];
        if constexpr (cx(q) != 0) jx += cx(q) * f[q];
        if constexpr (cy(q) != 0) jy += cy(q) * f[q];
        if constexpr (cz(q) != 0) jz += cz(q) * f[q];
        if constexpr (q < Q7) {
            Na += a[q];
            Nb += b[q];
        }
    });
    finite = finite && isfinite(Na) && isfinite(Nb);
    const float Nt = Na + Nb;
    const float phi = Nt > 0.0f ? (Na - Nb) / Nt : 0.0f;
    const float ux = jx + hfx, uy = jy + hfy, uz = jz + hfz;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float p = rho * (1.0f / 3.0f);
    const float xa = Nt > 0.0f ? Na / Nt : 0.0f, xb = Nt > 0.0f ? Nb / Nt : 0.0f;
    acc[0].add(Na);
    acc[1].add(Nb);
    acc[2].add(rho);
    acc[4].add(ux);
    acc[5].add(uy);
    acc[6].add(uz);
    acc[7].add(xa * ux);
    acc[8].add(xa * uy);
    acc[9].add(xa * uz);
    acc[10].add(xb * ux);
    acc[11].add(xb * uy);
    acc[12].add(xb * uz);
    if (phi > 0.0f) {
        acc[3].add(1.0);
        acc[13].add(rho);
        acc[15].add(rho * ux);
        acc[16].add(rho * uy);
        acc[17].add(rho * uz);
        acc[21].add(rho * uu);
        acc[23].add(p);
    } else {
        acc[14].add(rho);
        acc[18].add(rho * ux);
        acc[19].add(rho * uy);
        acc[20].add(rho * uz);
        acc[22].add(rho * uu);
        acc[24].add(p);
    }
    if (!finite) acc[25].add(1.0);
    if (Na < -1e-2f || Nb < -1e-2f || Nt <= 0.0f || rho <= 0.0f) acc[26].add(1.0);
}

// Block-wide fp64 reduction of the accumulators into out[0..NSUM) (thread 0..NSUM-1 write).
template <int BT>
__device__ __forceinline__ void block_reduce_sums(AccF64 (&acc)[NSUM], double* out) {
    __shared__ double red[BT / 32][NSUM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NSUM; ++i) {
        const double s = warp_sum(acc[i].value());
        if (lane == 0) red[w][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        double s = 0.0;
        for (int k = 0; k < BT / 32; ++k) s += red[k][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

}  // namespace lbm
