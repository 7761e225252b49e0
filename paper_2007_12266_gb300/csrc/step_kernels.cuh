// Device code of one color-gradient LBM timestep (Sec. 3.1), shared by the
// single-domain launchers and the batched launcher.
//
// State layout (structure of arrays, population-major, in place):
//   F[q*N + n], A[q*N + n], B[q*N + n]
// AA streaming: at an even step site n reads its own slots F[q][n] and writes
// the post-collision value of direction q to F[opp(q)][n]. At an odd step it
// reads direction q from F[opp(q)][m] where m is the upstream neighbour
// (x - xi_q) or, if that voxel is solid, from F[q][n] (bounce-back), and it
// writes direction q to F[q][m'] with m' = x + xi_q, or to F[opp(q)][n] when
// x + xi_q is solid (halfway bounce-back). Each site reads and writes the same
// slots within a step, so one array suffices and no two sites collide.
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// storage of the distributions
// ---------------------------------------------------------------------------

// Plain fp32 storage. ld_fdev / st_fdev exchange deviations f_q - t_q from
// the rest state, which the collision works with.
struct StoreF32 {
    template <int Q>
    static __device__ __forceinline__ float ld_fdev(const void* p, size_t i) {
        return static_cast<const float*>(p)[i] - t19(Q);
    }
    template <int Q>
    static __device__ __forceinline__ void st_fdev(void* p, size_t i, float dev) {
        static_cast<float*>(p)[i] = t19(Q) + dev;
    }
    template <int Q>
    static __device__ __forceinline__ float ld_f(const void* p, size_t i) {
        return static_cast<const float*>(p)[i];
    }
    template <int Q>
    static __device__ __forceinline__ void st_f(void* p, size_t i, float v) {
        static_cast<float*>(p)[i] = v;
    }
    template <int Q>
    static __device__ __forceinline__ float ld_c(const void* p, size_t i) {
        return static_cast<const float*>(p)[i];
    }
    template <int Q>
    static __device__ __forceinline__ void st_c(void* p, size_t i, float v) {
        static_cast<float*>(p)[i] = v;
    }
};

// fp16 storage: momentum populations as deviations from the rest state
// (f_q - t_q, rho = 1), component populations as plain fp16 values (their
// rest state depends on the local composition, and a plain fp16 keeps full
// relative precision near zero in the pure phases). The arithmetic stays fp32.
struct StoreF16 {
    template <int Q>
    static __device__ __forceinline__ float ld_fdev(const void* p, size_t i) {
        return __half2float(static_cast<const __half*>(p)[i]);
    }
    template <int Q>
    static __device__ __forceinline__ void st_fdev(void* p, size_t i, float dev) {
        static_cast<__half*>(p)[i] = __float2half_rn(dev);
    }
    template <int Q>
    static __device__ __forceinline__ float ld_f(const void* p, size_t i) {
        return t19(Q) + __half2float(static_cast<const __half*>(p)[i]);
    }
    template <int Q>
    static __device__ __forceinline__ void st_f(void* p, size_t i, float v) {
        static_cast<__half*>(p)[i] = __float2half_rn(v - t19(Q));
    }
    template <int Q>
    static __device__ __forceinline__ float ld_c(const void* p, size_t i) {
        return __half2float(static_cast<const __half*>(p)[i]);
    }
    template <int Q>
    static __device__ __forceinline__ void st_c(void* p, size_t i, float v) {
        static_cast<__half*>(p)[i] = __float2half_rn(v);
    }
};

// Read-only load that the compiler may not merge with an earlier load of the
// same address: re-reading a neighbour id from L1 is cheaper than keeping 18
// of them live in registers across the collision.
__device__ __forceinline__ int ld_fresh(const int* p) {
    int v;
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// ---------------------------------------------------------------------------
// AA read map: where the value of direction Q of site n lives at a step of
// parity PAR (the same slot the step writes direction opp(Q) to).
// ---------------------------------------------------------------------------
template <int PAR, int Q>
__device__ __forceinline__ size_t read_slot(const DomainView& d, int n, const int* nb) {
    const size_t N = static_cast<size_t>(d.n_sites);
    if constexpr (Q == 0 || PAR == 0) {
        return static_cast<size_t>(Q) * N + n;
    } else {
        // upstream site x - xi_Q = x + xi_opp(Q), or -1 (bounce-back)
        const int up = nb[opp(Q)];
        return up >= 0 ? static_cast<size_t>(opp(Q)) * N + up : static_cast<size_t>(Q) * N + n;
    }
}

template <int PAR, int Q>
__device__ __forceinline__ size_t write_slot(const DomainView& d, int n, const int* nb) {
    (void)nb;
    const size_t N = static_cast<size_t>(d.n_sites);
    if constexpr (Q == 0) {
        return static_cast<size_t>(n);
    } else if constexpr (PAR == 0) {
        return static_cast<size_t>(opp(Q)) * N + n;
    } else {
        // downstream site x + xi_Q, or -1 (halfway bounce-back)
        const int down = nb[Q];
        return down >= 0 ? static_cast<size_t>(Q) * N + down : static_cast<size_t>(opp(Q)) * N + n;
    }
}

// write slot with the downstream neighbour re-read from the padded site grid
template <int PAR, int Q>
__device__ __forceinline__ size_t write_slot_v(const DomainView& d, int n, int v) {
    const size_t N = static_cast<size_t>(d.n_sites);
    if constexpr (Q == 0) {
        return static_cast<size_t>(n);
    } else if constexpr (PAR == 0) {
        return static_cast<size_t>(opp(Q)) * N + n;
    } else {
        const int down = ld_fresh(d.vsite + v + d.off[Q]);
        return down >= 0 ? static_cast<size_t>(Q) * N + down : static_cast<size_t>(opp(Q)) * N + n;
    }
}

// ---------------------------------------------------------------------------
// phase pass: Na, Nb -> phi (dense grid) and N (per site)          Sec. 3.1
// ---------------------------------------------------------------------------
template <int PAR, class S>
__device__ __forceinline__ void phase_site(const DomainView& d, int n, int& v, float& Na, float& Nb) {
    v = d.site_vox[n];
    int nb[7];
    if constexpr (PAR == 1) {
        static_for<1, 7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + d.off[q]);
        });
    }
    Na = 0.0f;
    Nb = 0.0f;
    static_for<0, 7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const size_t i = read_slot<PAR, q>(d, n, nb);
        Na += S::template ld_c<q>(d.a, i);
        Nb += S::template ld_c<q>(d.b, i);
    });
}

__device__ __forceinline__ float phase_of(float Na, float Nb) {
    const float Nt = Na + Nb;
    return Nt > 0.0f ? (Na - Nb) / Nt : 0.0f;
}

template <int PAR, class S>
__device__ __forceinline__ void phase_thread(const DomainView& d, int t) {
    if (t < d.n_sites) {
        int v;
        float Na, Nb;
        phase_site<PAR, S>(d, t, v, Na, Nb);
        d.phi[v] = phase_of(Na, Nb);
        d.nsum[t] = Na + Nb;
    } else if (t < d.n_sites + d.n_halo) {
        // halo voxel of a periodic face: mirror the phase of its source site
        const int e = t - d.n_sites;
        int v;
        float Na, Nb;
        phase_site<PAR, S>(d, __ldg(d.halo_site + e), v, Na, Nb);
        d.phi[__ldg(d.halo_dst + e)] = phase_of(Na, Nb);
    }
}

// ---------------------------------------------------------------------------
// fused collide + stream                                            Sec. 3.1
// ---------------------------------------------------------------------------
template <int PAR, class S>
__device__ __forceinline__ void collide_thread(const DomainView& d, int n) {
    const int v = __ldg(d.site_vox + n);

    // neighbour sites for the odd-step gather / scatter
    int nb[Q19];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + d.off[q]);
        });
    }

    // incoming distributions, as deviations d_q = f_q - t_q from the rest
    // state (exact in fp32 near rest), so that density and momentum are sums of
    // small numbers and the relaxation acts on small quantities
    float f[Q19];
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        f[q] = S::template ld_fdev<q>(d.f, read_slot<PAR, q>(d, n, nb));
    });

    // phase field: own value and the 18 neighbours (solids hold phi_s)
    const float phi_c = __ldg(d.phi + v);
    const float Nt = __ldg(d.nsum + n);
    float p[Q19];
    static_for<1, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        p[q] = __ldg(d.phi + v + d.off[q]);
    });

    // color gradient C = sum_q g_q xi_q phi(x + xi_q)
    float Cx = 0.0f, Cy = 0.0f, Cz = 0.0f;
    static_for<1, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr float g = grad_w(q);
        if constexpr (cx(q) != 0) Cx = fmaf(g * cx(q), p[q], Cx);
        if constexpr (cy(q) != 0) Cy = fmaf(g * cy(q), p[q], Cy);
        if constexpr (cz(q) != 0) Cz = fmaf(g * cz(q), p[q], Cz);
    });
    const float Cmag = sqrtf(Cx * Cx + Cy * Cy + Cz * Cz);
    float nx = 0.0f, ny = 0.0f, nz = 0.0f;
    if (Cmag > 0.0f) {
        const float inv = 1.0f / Cmag;
        nx = Cx * inv;
        ny = Cy * inv;
        nz = Cz * inv;
    }

    // macroscopic moments: drho = rho - 1 and j from the deviations
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        drho += f[q];
        if constexpr (cx(q) > 0) jx += f[q];
        if constexpr (cx(q) < 0) jx -= f[q];
        if constexpr (cy(q) > 0) jy += f[q];
        if constexpr (cy(q) < 0) jy -= f[q];
        if constexpr (cz(q) > 0) jz += f[q];
        if constexpr (cz(q) < 0) jz -= f[q];
    });

    // relaxation rates from the viscosity (tau mixed linearly in phi)
    float s_nu = d.s_nu, s_m = d.s_m;
    if (!d.uniform_tau) {
        const float tau = d.tau_b + (d.tau_a - d.tau_b) * 0.5f * (1.0f + phi_c);
        s_nu = 1.0f / tau;
        s_m = 8.0f * (2.0f - s_nu) / (8.0f - s_nu);
    }

    // MRT collision, evaluated in its equivalent two-relaxation-time form.
    // With S from the viscosity, every non-conserved even moment (m1, m2,
    // m9..m15) relaxes with s_nu and every non-conserved odd moment (m4, m6,
    // m8, m16..m18) with s_m; the conserved ones equal their equilibria. So
    //   f* = f - s_nu (f+ - feq+) - s_m (f- - feq-) + 3 t_q xi_q . F
    // with f+- the even/odd parts over opposite pairs and feq the velocity-
    // space equilibrium whose moments are m^eq:
    //   feq+ = t_q (rho + 4.5 (xi.j)^2 - 1.5 j.j) + M^-1 dm_alpha
    //   feq- = 3 t_q xi.j
    // where dm_alpha holds the interfacial-tension terms of m1, m9, m11,
    // m13, m14, m15 (rho0 = 1). Everything below is relative to the rest
    // state t_q (rho = 1), i.e. in deviations.
    const float jj = jx * jx + jy * jy + jz * jz;
    const float ac = d.alpha * Cmag;
    const float hac = 0.5f * ac;
    float dma[Q19];
    dma[1] = -ac;
    dma[9] = hac * (2.0f * nx * nx - ny * ny - nz * nz);
    dma[11] = hac * (ny * ny - nz * nz);
    dma[13] = hac * nx * ny;
    dma[14] = hac * ny * nz;
    dma[15] = hac * nx * nz;
    const float drho_iso = drho - 1.5f * jj;

    // recoloring inputs: Na = N (1 + phi)/2, Nb = N (1 - phi)/2, so the
    // weights Nb/N and Na/N are (1 - phi)/2 and (1 + phi)/2
    const float Na = 0.5f * Nt * (1.0f + phi_c);
    const float Nb = 0.5f * Nt * (1.0f - phi_c);
    const float bxa = d.beta * 0.5f * (1.0f - phi_c);
    const float bxb = d.beta * 0.5f * (1.0f + phi_c);

    // The increments of the moving populations sum to minus the rest
    // increment in exact arithmetic; taking the rest increment as that sum
    // keeps fp32 mass exact up to unbiased rounding.
    float dsum = 0.0f;
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;   // q odd, opp(q) = q + 1
        constexpr int o = q + 1;
        constexpr float t = t19(q);
        float cu = 0.0f, xf = 0.0f;
        if constexpr (cx(q) != 0) { cu += cx(q) * jx; xf += cx(q) * d.fx; }
        if constexpr (cy(q) != 0) { cu += cy(q) * jy; xf += cy(q) * d.fy; }
        if constexpr (cz(q) != 0) { cu += cz(q) * jz; xf += cz(q) * d.fz; }
        float eqp = t * fmaf(4.5f * cu, cu, drho_iso);
        static_for<1, 16>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            if constexpr (k == 1 || k == 9 || k == 11 || k == 13 || k == 14 || k == 15) {
                if constexpr (mrow(k, q) != 0) eqp = fmaf(minv(q, k), dma[k], eqp);
            }
        });
        const float eqm = 3.0f * t * cu;
        const float fp = 0.5f * (f[q] + f[o]);
        const float fm = 0.5f * (f[q] - f[o]);
        const float dp = -s_nu * (fp - eqp);
        const float dmi = fmaf(3.0f * t, xf, -s_m * (fm - eqm));
        const float inc_q = dp + dmi, inc_o = dp - dmi;
        dsum += inc_q + inc_o;
        S::template st_fdev<q>(d.f, write_slot_v<PAR, q>(d, n, v), f[q] + inc_q);
        S::template st_fdev<o>(d.f, write_slot_v<PAR, o>(d, n, v), f[o] + inc_o);
    });
    S::template st_fdev<0>(d.f, write_slot_v<PAR, 0>(d, n, v), f[0] - dsum);

    // recolored component distributions (Eqs. LBE-mass-a/b), streamed on the
    // fly; the rest populations take the remainder of Na and Nb so that the
    // fp32 weights (whose sum is not exactly 1) create no mass
    float asum = 0.0f, bsum = 0.0f;
    static_for<1, Q7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        float ux = 0.0f, nn = 0.0f;
        if constexpr (cx(q) != 0) { ux = cx(q) * jx; nn = cx(q) * nx; }
        if constexpr (cy(q) != 0) { ux = cy(q) * jy; nn = cy(q) * ny; }
        if constexpr (cz(q) != 0) { ux = cz(q) * jz; nn = cz(q) * nz; }
        const float base = 1.0f + 4.5f * ux;
        const float av = w7(q) * Na * (base + bxa * nn);
        const float bv = w7(q) * Nb * (base - bxb * nn);
        asum += av;
        bsum += bv;
        const size_t i = write_slot_v<PAR, q>(d, n, v);
        S::template st_c<q>(d.a, i, av);
        S::template st_c<q>(d.b, i, bv);
    });
    const size_t i0 = write_slot_v<PAR, 0>(d, n, v);
    S::template st_c<0>(d.a, i0, Na - asum);
    S::template st_c<0>(d.b, i0, Nb - bsum);
}

// ---------------------------------------------------------------------------
// reservoir reset (unsteady protocol, Sec. 4.1): write the rest state into
// the slots the NEXT step (parity PAR) reads.
// ---------------------------------------------------------------------------
template <int PAR, class S>
__device__ __forceinline__ void reservoir_thread(const DomainView& d, int n, int side, float rho_in,
                                                 float rho_out) {
    const int v = d.site_vox[n];
    int nb[Q19];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + d.off[q]);
        });
    }
    const float rho = side == 1 ? rho_in : rho_out;
    const float na = side == 1 ? 1.0f : 0.0f;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const size_t i = read_slot<PAR, q>(d, n, nb);
        S::template st_f<q>(d.f, i, t19(q) * rho);
        if constexpr (q < Q7) {
            S::template st_c<q>(d.a, i, w7(q) * na);
            S::template st_c<q>(d.b, i, w7(q) * (1.0f - na));
        }
    });
}

}  // namespace lbm
