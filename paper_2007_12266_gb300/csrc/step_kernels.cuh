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
    using T = float;
    static constexpr bool kRef = false;   // component values stored as they are
    // Hot-path forms: p points at the slot itself and values are in the
    // collision's working units, deviations times kK (here 1).
    static constexpr float kK = 1.0f;
    template <int Q>
    static __device__ __forceinline__ float ld_fs(const T* p) { return *p - t19(Q); }
    template <int Q>
    static __device__ __forceinline__ void st_fs(T* p, float dev) { *p = t19(Q) + dev; }
    static __device__ __forceinline__ void st_cs(T* p, float v) { *p = v; }
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

// fp16 storage of deviations from a local rest-state equilibrium, arithmetic
// in fp32. Momentum: f_q - t_q rho(s), with rho of a reference site s kept in
// fp32 per site (DomainView::drho): the writing site for values written at an
// even step (read at the next odd step through the neighbour table) and the
// destination site, with its density of the last even step, for values
// written at an odd step (read at the next even step by that destination with
// one coalesced load); drho is written only at even steps.
// Components: A_q - w_q (1 + phi_w)/2 and B_q - w_q (1 - phi_w)/2, with phi_w
// the phase of the site w that wrote the value, at that step. The writer uses
// its own phase; the reader finds phi_w in the previous step's phase grid
// (DomainView::phi is double-buffered by step parity) at the upstream voxel
// x - xi_q, or at its own voxel when that link bounced back (DomainView::wall6),
// so no neighbour id is looked up for it. The phase pass needs only the sum
// of the references over the seven directions, Na = sum_q s_q + (1 + S)/2
// with S = sum_q w_q phi_w(q) (likewise Nb with -S; the writers' rest values
// absorb the fp32 weights' excess over 1); the collision, which holds those
// phases for its colour gradient, stores S per site (DomainView::rsum), so the
// phase pass reads one coalesced number instead of six phases. Against the
// writer's own (Na, Nb) the stored number gains w_q (N - 1)(1 +- phi_w)/2;
// N = Na + Nb follows the density, within a few 1e-2 of 1.
// Storing A, B themselves let every site of a pure phase round the same value
// the same way on the fp16 grid, a biased error that leaked 3e-3 of the
// component mass per 1,000 steps; storing f - t_q left the local density
// excursion (up to a few 1e-2 under a body force and capillary pressure) in
// the stored number and cost the velocity its precision. Referencing the
// components to the phase of the reading site instead (known to the reader
// without any lookup) left (phi_w - phi_r)/2, up to w_q at a sharp interface,
// in the stored numbers and raised the flux error against the oracle tenfold.
// ld_fdev / st_fdev below exchange the stored number; the kernels add the
// reference.
// Values are scaled by 2^14 (an exact power of two) to keep small deviations
// out of fp16's subnormal range; |deviation| up to 4 stays representable.
struct StoreF16 {
    using T = __half;
    static constexpr bool kRef = true;
    static constexpr float kScale = 16384.0f;
    static constexpr float kInv = 1.0f / 16384.0f;
    // Hot-path forms: the collision works in units of 2^-14 (kK = 2^14 times
    // the deviations), so the stored number is used as it is and the scale
    // costs no multiplication per value.
    static constexpr float kK = kScale;
    template <int Q>
    static __device__ __forceinline__ float ld_fs(const T* p) { return __half2float(*p); }
    template <int Q>
    static __device__ __forceinline__ void st_fs(T* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void st_cs(T* p, float v) { *p = __float2half_rn(v); }
    template <int Q>
    static __device__ __forceinline__ float ld_fdev(const void* p, size_t i) {
        return __half2float(static_cast<const __half*>(p)[i]) * kInv;
    }
    template <int Q>
    static __device__ __forceinline__ void st_fdev(void* p, size_t i, float dev) {
        static_cast<__half*>(p)[i] = __float2half_rn(dev * kScale);
    }
    template <int Q>
    static __device__ __forceinline__ float ld_f(const void* p, size_t i) {
        return t19(Q) + ld_fdev<Q>(p, i);
    }
    template <int Q>
    static __device__ __forceinline__ void st_f(void* p, size_t i, float v) {
        st_fdev<Q>(p, i, v - t19(Q));
    }
    template <int Q>
    static __device__ __forceinline__ float ld_c(const void* p, size_t i) {
        return __half2float(static_cast<const __half*>(p)[i]) * kInv;
    }
    template <int Q>
    static __device__ __forceinline__ void st_c(void* p, size_t i, float v) {
        static_cast<__half*>(p)[i] = __float2half_rn(v * kScale);
    }
};

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic
// stream serialization may start while the previous kernel in the stream is
// still running. wait_prior_grid() blocks until that kernel has completed and
// its writes are visible; allow_next_grid() lets the next kernel start its
// blocks. Without the launch attribute both are no-ops.
// Data written by an earlier kernel of the step chain (phi, nsum, the
// fp16 reference densities, the populations) is read with plain coherent
// loads only: a read-only (__ldg / .nc) load may legally be hoisted by the
// compiler above wait_prior_grid(), which would read the previous step's
// values. __ldg is kept for the static index arrays.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// sum form: component densities carried as per-site fixed-point sums
// ---------------------------------------------------------------------------
// The recolored populations of Eqs. LBE-mass-a/b are a function of the
// writing site's Na, Nb, velocity and colour normal, and the next step uses
// the populations a site receives only through their sums Na, Nb. In the sum
// form the collision adds each recolored value A*_q, B*_q straight into the
// sums of the site that receives it (x + xi_q, or x itself on a bounce-back
// link). A site's (Na, Nb) is one 64-bit word: Na in the high and Nb in the
// low 32 bits, each in units of 2^-28 (|N| < 8). Adding packed words adds both
// halves exactly as long as the low sum stays within 32 bits, and integer sums
// do not depend on the order of the additions, so the result is deterministic
// and each component's mass is conserved exactly.
constexpr float kSumOne = 268435456.0f;          // 2^28
constexpr float kSumInv = 1.0f / 268435456.0f;

__device__ __forceinline__ unsigned long long pack_sums(int a, int b) {
    return (static_cast<unsigned long long>(static_cast<unsigned>(a)) << 32) +
           static_cast<unsigned long long>(static_cast<long long>(b));
}
__device__ __forceinline__ void unpack_sums(unsigned long long s, int& a, int& b) {
    b = static_cast<int>(static_cast<unsigned>(s));
    a = static_cast<int>((static_cast<long long>(s) - static_cast<long long>(b)) >> 32);
}
// N = Na + Nb and phi = (Na - Nb)/(Na + Nb) of a site from its sums, in fp32
// (32-bit integer to float conversions: a 64-bit conversion runs on the fp64
// pipe, which is slow on this GPU); the phase pass and the collision both use
// this function, so they agree bit for bit.
__device__ __forceinline__ void sums_phase(int a, int b, float& Nt, float& phi) {
    const float fa = static_cast<float>(a), fb = static_cast<float>(b);
    const float nt = fa + fb;
    Nt = nt * kSumInv;
    phi = nt > 0.0f ? (fa - fb) / nt : 0.0f;
}
// The sums and the site -> voxel map (8 + 4 bytes per site, read by the phase
// pass and again by the collision) are accessed with an L2 evict-last policy,
// so that they stay in L2 between the two kernels while the populations
// stream through it.
__device__ __forceinline__ unsigned long long l2_keep() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void red_add(unsigned long long* p, unsigned long long v, unsigned long long pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ unsigned long long ld_keep(const unsigned long long* p, unsigned long long pol) {
    unsigned long long v;
    asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ void st_keep(unsigned long long* p, unsigned long long v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ int ldg_keep(const int* p, unsigned long long pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
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

// ---------------------------------------------------------------------------
// component populations (D3Q7, Eqs. LBE-mass-a/b)
// ---------------------------------------------------------------------------
// The site that wrote slot read_slot<PAR, Q>(n) during the previous step: the
// upstream neighbour x - xi_Q if it is a pore, else n itself (bounce-back).
template <int Q>
__device__ __forceinline__ int writer_of(int n, const int* nb) {
    if constexpr (Q == 0) {
        return n;
    } else {
        const int up = nb[opp(Q)];
        return up >= 0 ? up : n;
    }
}

// Site whose density is the reference of the momentum population read as
// direction Q by site n at a step of parity PAR (see StoreF16).
template <int PAR, int Q>
__device__ __forceinline__ int f_ref_read(int n, const int* nb) {
    if constexpr (PAR == 0) return n;
    else return writer_of<Q>(n, nb);
}

// Phase of the site that wrote the component value read as direction Q by the
// site at voxel v at a step of parity PAR (fp16 storage, see StoreF16): from
// the previous step's phase grid, at the upstream voxel x - xi_Q, or at v when
// x - xi_Q is solid (bit opp(Q) - 1 of the site's wall mask).
template <int PAR, int Q>
__device__ __forceinline__ float writer_phase(const DomainView& d, int v, unsigned wall) {
    const float* prev = d.phi[PAR ^ 1];
    if constexpr (Q == 0) {
        return prev[v];
    } else {
        constexpr int o = opp(Q);
        return prev[((wall >> (o - 1)) & 1u) ? v : v + stencil_off(d, o)];
    }
}

// A_q, B_q of site n (voxel v) at a step of parity PAR (nb[1..6]: face
// neighbours at odd steps).
template <int PAR, class S>
__device__ __forceinline__ void load_components(const DomainView& d, int n, int v, const int* nb, float (&a)[Q7],
                                                float (&b)[Q7]) {
    unsigned wall = 0;
    if constexpr (S::kRef) wall = __ldg(d.wall6 + n);
    static_for<0, Q7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const size_t i = read_slot<PAR, q>(d, n, nb);
        a[q] = S::template ld_c<q>(d.a, i);
        b[q] = S::template ld_c<q>(d.b, i);
        if constexpr (S::kRef) {
            const float pw = writer_phase<PAR, q>(d, v, wall);
            a[q] = fmaf(w7(q) * 0.5f, 1.0f + pw, a[q]);
            b[q] = fmaf(w7(q) * 0.5f, 1.0f - pw, b[q]);
        }
    });
}

// fp16 storage: S = sum_q w_q phi_w(q) over the seven component values that
// site n (voxel v) reads at a step of parity PAR (see writer_phase).
template <int PAR>
__device__ __forceinline__ float reference_phase_sum(const DomainView& d, int n, int v) {
    const unsigned wall = __ldg(d.wall6 + n);
    float S = 0.0f;
    static_for<0, Q7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        S = fmaf(w7(q), writer_phase<PAR, q>(d, v, wall), S);
    });
    return S;
}

// Whether the face-neighbour ids are needed to read the components.
template <int PAR>
constexpr bool need_face_nb() { return PAR == 1; }

// ---------------------------------------------------------------------------
// phase pass: Na, Nb -> phi (dense grid) and N (per site)          Sec. 3.1
// ---------------------------------------------------------------------------
// Phase pass of one site (or one periodic halo voxel mirroring a site).
// Ordering with the neighbouring kernels under programmatic launch: only the
// static index (site_vox, vsite) is read before wait_prior_grid(); A and B
// (written by the previous collision) are read, and phi / nsum (read by the
// previous collision) are written, only after it. Dependents are released
// after the wait, so the next collision never starts before the previous
// one has completed.
template <int PAR, class S>
__device__ __forceinline__ void phase_thread(const DomainView& d, int t) {
    int n = -1, dst = -1;
    if (t < d.n_sites) {
        n = t;
    } else if (t < d.n_sites + d.n_halo) {
        n = __ldg(d.halo_site + (t - d.n_sites));
        dst = __ldg(d.halo_dst + (t - d.n_sites));
    }
    int v = 0;
    int nb[7];
    if (n >= 0) {
        v = __ldg(d.site_vox + n);
        if constexpr (need_face_nb<PAR>()) {
            static_for<1, 7>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
            });
        }
    }
    wait_prior_grid();
    allow_next_grid();
    if (n < 0) return;
    float Na = 0.0f, Nb = 0.0f;
    if constexpr (S::kRef) {
        // stored deviations plus the references' sum, (1 +- rsum)/2 (the
        // writers' rest values absorb the fp32 weights' excess over 1)
        static_for<0, Q7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            const size_t i = read_slot<PAR, q>(d, n, nb);
            Na += S::template ld_c<q>(d.a, i);
            Nb += S::template ld_c<q>(d.b, i);
        });
        const float Sr = d.rsum[n];
        Na = fmaf(0.5f, 1.0f + Sr, Na);
        Nb = fmaf(0.5f, 1.0f - Sr, Nb);
    } else {
        float a[Q7], b[Q7];
        load_components<PAR, S>(d, n, v, nb, a, b);
        static_for<0, Q7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            Na += a[q];
            Nb += b[q];
        });
    }
    const float Nt = Na + Nb;
    const float phi = Nt > 0.0f ? (Na - Nb) / Nt : 0.0f;
    if (dst < 0) {
        d.phi[PAR][v] = phi;
        d.nsum[n] = Nt;
    } else {
        d.phi[PAR][dst] = phi;    // halo voxel of a periodic face
    }
}

// Phase pass of the sum form: phi (and, for a population-form collision
// next, N) from the site's component sums, for PER entries per thread
// (entries t0 + k * stride: sites, then periodic halo voxels). Ordering as in
// phase_thread: the sums were completed by the collision before the previous
// phase pass.
template <int PAR, bool WRITE_N, int PER>
__device__ __forceinline__ void phase_sum_thread(const DomainView& d, int t0, int stride) {
    const unsigned long long pol = l2_keep();
    int n[PER], dst[PER], v[PER];
    #pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int t = t0 + k * stride;
        n[k] = -1;
        dst[k] = -1;
        v[k] = 0;
        if (t < d.n_sites) {
            n[k] = t;
            v[k] = ldg_keep(d.site_vox + t, pol);
        } else if (t < d.n_sites + d.n_halo) {
            n[k] = __ldg(d.halo_site + (t - d.n_sites));
            dst[k] = __ldg(d.halo_dst + (t - d.n_sites));
        }
    }
    wait_prior_grid();
    allow_next_grid();
    unsigned long long s[PER];
    #pragma unroll
    for (int k = 0; k < PER; ++k) s[k] = n[k] >= 0 ? ld_keep(d.acc[PAR] + n[k], pol) : 0ull;
    #pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (n[k] < 0) continue;
        int a, b;
        unpack_sums(s[k], a, b);
        float Nt, phi;
        sums_phase(a, b, Nt, phi);
        if (dst[k] < 0) {
            d.phi[PAR][v[k]] = phi;
            if constexpr (WRITE_N) d.nsum[n[k]] = Nt;
        } else {
            d.phi[PAR][dst[k]] = phi;    // halo voxel of a periodic face
        }
    }
}

// ---------------------------------------------------------------------------
// fused collide + stream                                            Sec. 3.1
// ---------------------------------------------------------------------------
// Component forms of the collision (CF): 0 stores the recolored populations
// (AA slots); 1 and 2 add them into the receivers' sums (sum form), with the
// site's own Na, Nb taken from the phase pass (1, first step of a run) or
// from its own sums (2).
// At an odd step site n reads direction opp(q) from, and writes direction q
// to, the same slot: row q at the downstream neighbour x + xi_q, or row
// opp(q) at n itself when that voxel is solid. With fp16 storage both also
// use the same density reference (that neighbour's density of the last even
// step, which odd steps do not change). SlotCache keeps the slot (relative to
// row q, a signed 32-bit offset) and the reference of each direction between
// the gather and the scatter, in shared memory laid out [q - 1][thread] so
// that a warp's accesses fall in distinct banks.
struct SlotCache {
    int* slot;      // entry of direction 1 of this thread; direction q at slot[(q - 1) * stride]
                    // (even steps of the sum form: the face neighbour's site id, -1 if solid)
    float* ref;     // same layout (fp16 storage only)
    int stride;     // threads per block
};

// Incoming distributions of site n (voxel v), as deviations d_q = f_q - t_q
// from the rest state (exact in fp32 near rest), so that density and
// momentum are sums of small numbers and the relaxation acts on small
// quantities; in working units, i.e. times S::kK. Odd steps also fill the
// slot cache.
template <int PAR, class S>
__device__ __forceinline__ void load_f(const DomainView& d, int n, int v, float (&f)[Q19], SlotCache sc) {
    const int Ni = d.n_sites;
    const size_t N = static_cast<size_t>(Ni);
    const typename S::T* const F = static_cast<const typename S::T*>(d.f);
    constexpr float K = S::kK;
    if constexpr (PAR == 0) {
        // even step: own slots, row q; fp16 references are all this site's
        float r = 0.0f;
        if constexpr (S::kRef) r = d.drho[n];
        static_for<0, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            f[q] = S::template ld_fs<q>(F + q * N + n);
            if constexpr (S::kRef) f[q] = fmaf(t19(q) * K, r, f[q]);
        });
    } else {
        f[0] = S::template ld_fs<0>(F + n);
        if constexpr (S::kRef) f[0] = fmaf(t19(0) * K, d.drho[n], f[0]);
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;   // direction of the downstream slot
            constexpr int o = opp(q);                // direction read from it
            const int m = __ldg(d.vsite + v + stencil_off(d, q));
            const int s = m >= 0 ? m : n + (o - q) * Ni;
            sc.slot[(q - 1) * sc.stride] = s;
            f[o] = S::template ld_fs<o>(F + q * N + s);
            if constexpr (S::kRef) {
                const float r = d.drho[m >= 0 ? m : n];
                sc.ref[(q - 1) * sc.stride] = r;
                f[o] = fmaf(t19(o) * K, r, f[o]);
            }
        });
    }
}


// colour gradient C = sum_q g_q xi_q phi(x + xi_q); phi_at(q) gives the
// neighbour's phase (solids hold phi_s)
template <class PhiAt>
__device__ __forceinline__ void color_gradient(PhiAt&& phi_at, float& Cx, float& Cy, float& Cz) {
    Cx = 0.0f;
    Cy = 0.0f;
    Cz = 0.0f;
    static_for<1, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr float g = grad_w(q);
        const float p = phi_at(qc);
        if constexpr (cx(q) != 0) Cx = fmaf(g * cx(q), p, Cx);
        if constexpr (cy(q) != 0) Cy = fmaf(g * cy(q), p, Cy);
        if constexpr (cz(q) != 0) Cz = fmaf(g * cz(q), p, Cz);
    });
}

// macroscopic moments: drho = rho - 1 and j from the deviations
struct Moments {
    float drho, jx, jy, jz;
};
__device__ __forceinline__ Moments moments(const float (&f)[Q19]) {
    Moments m{0.0f, 0.0f, 0.0f, 0.0f};
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        m.drho += f[q];
        if constexpr (cx(q) > 0) m.jx += f[q];
        if constexpr (cx(q) < 0) m.jx -= f[q];
        if constexpr (cy(q) > 0) m.jy += f[q];
        if constexpr (cy(q) < 0) m.jy -= f[q];
        if constexpr (cz(q) > 0) m.jz += f[q];
        if constexpr (cz(q) < 0) m.jz -= f[q];
    });
    return m;
}

// Collision, recoloring and streaming of site n, given its incoming
// deviations f and their moments, its phase phi_c, Na, Nb and the colour
// gradient.
// Nt: Na + Nb from the phase pass (Na = Nt (1 + phi_c)/2, Nb = Nt (1 - phi_c)/2).
// a_own, b_own (CF == 2): the site's component sums in fixed point.
template <int PAR, class S, int CF = 0>
__device__ __forceinline__ void collide_site(const DomainView& d, int n, const float (&f)[Q19], Moments mo,
                                             float phi_c, float Nt, int a_own, int b_own, float Cx, float Cy,
                                             float Cz, SlotCache sc) {
    using T = typename S::T;
    const size_t N = static_cast<size_t>(d.n_sites);
    T* const F = static_cast<T*>(d.f);
    // f, drho and j are in working units (times K); the equilibrium's
    // quadratic terms take one factor 1/K, the interfacial terms and the
    // forcing (d.fterm is stored in working units) one factor K
    constexpr float K = S::kK;
    constexpr float iK = 1.0f / K;
    const float drho = mo.drho, jx = mo.jx, jy = mo.jy, jz = mo.jz;

    const float C2 = Cx * Cx + Cy * Cy + Cz * Cz;
    float nx = 0.0f, ny = 0.0f, nz = 0.0f, Cmag = 0.0f;
    if (C2 > 0.0f) {
        const float inv = rsqrtf(C2);
        Cmag = C2 * inv;
        nx = Cx * inv;
        ny = Cy * inv;
        nz = Cz * inv;
    }

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
    const float ac = (d.alpha * K) * Cmag;
    const float hac = 0.5f * ac;
    float dma[Q19];
    dma[1] = -ac;
    dma[9] = hac * (2.0f * nx * nx - ny * ny - nz * nz);
    dma[11] = hac * (ny * ny - nz * nz);
    dma[13] = hac * nx * ny;
    dma[14] = hac * ny * nz;
    dma[15] = hac * nx * nz;
    const float drho_iso = fmaf(-1.5f * iK, jj, drho);

    // recoloring weights Nb/N and Na/N are (1 - phi)/2 and (1 + phi)/2
    const float bxa = d.beta * 0.5f * (1.0f - phi_c);
    const float bxb = d.beta * 0.5f * (1.0f + phi_c);

    // destination of direction q (q >= 1): row opp(q) at n (even step) or
    // the cached slot of row q (odd step)
    auto dst = [&](auto qc, auto* base) {
        constexpr int q = decltype(qc)::value;
        if constexpr (PAR == 0) return base + opp(q) * N + n;
        else return base + q * N + sc.slot[(q - 1) * sc.stride];
    };

    // The increments of the moving populations sum to minus the rest
    // increment in exact arithmetic; taking the rest increment as that sum
    // keeps fp32 mass exact up to unbiased rounding.
    float dsum = 0.0f;
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;   // q odd, opp(q) = q + 1
        constexpr int o = q + 1;
        constexpr float t = t19(q);
        float cu = 0.0f;
        if constexpr (cx(q) != 0) cu += cx(q) * jx;
        if constexpr (cy(q) != 0) cu += cy(q) * jy;
        if constexpr (cz(q) != 0) cu += cz(q) * jz;
        float eqp = t * fmaf((4.5f * iK) * cu, cu, drho_iso);
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
        const float dmi = fmaf(-s_m, fm - eqm, d.fterm[q >> 1]);
        const float inc_q = dp + dmi, inc_o = dp - dmi;
        dsum += inc_q + inc_o;
        float vq = f[q] + inc_q, vo = f[o] + inc_o;
        if constexpr (S::kRef) {
            // even step: relative to this site's rest state t_q rho; odd step:
            // relative to the destination's density of the last even step
            if constexpr (PAR == 0) {
                vq = fmaf(-t, drho, vq);
                vo = fmaf(-t, drho, vo);
            } else {
                vq = fmaf(-t * K, sc.ref[(q - 1) * sc.stride], vq);
                vo = fmaf(-t * K, sc.ref[(o - 1) * sc.stride], vo);
            }
        }
        S::template st_fs<q>(dst(std::integral_constant<int, q>{}, F), vq);
        S::template st_fs<o>(dst(std::integral_constant<int, o>{}, F), vo);
    });
    if constexpr (S::kRef) {
        if constexpr (PAR == 0) {
            S::template st_fs<0>(F + n, fmaf(-t19(0), drho, f[0] - dsum));
            d.drho[n] = drho * iK;
        } else {
            S::template st_fs<0>(F + n, fmaf(-t19(0) * K, d.drho[n], f[0] - dsum));
        }
    } else {
        S::template st_fs<0>(F + n, f[0] - dsum);
    }

    // recolored component distributions (Eqs. LBE-mass-a/b), streamed on the
    // fly; the rest populations take the remainder of Na and Nb so that the
    // fp32 weights (whose sum is not exactly 1) create no mass. With fp16
    // storage the stored quantity is the deviation from w_q (1 +- phi_c)/2: the
    // deviation from w_q Na (w_q Nb), which the formula gives directly as
    // w_q Na (4.5 u.xi + beta Nb/N n.xi), plus w_q times
    //   Na - (1 + phi_c)/2 = (N - 1)(1 + phi_c)/2   (likewise for Nb).
    // (working units: Na, Nb times K, j divided by K back to u)
    const float NaK = (0.5f * K) * Nt * (1.0f + phi_c), NbK = (0.5f * K) * Nt * (1.0f - phi_c);
    if constexpr (CF != 0) {
        // Sum form: A*_q = w_q Na [1 + 4.5 u.xi_q + beta (Nb/N) n.xi_q] (likewise B*_q)
        // in fixed point, added into the sums of the site that receives it; the
        // rest value takes the remainder of the site's own Na (Nb), so the seven
        // values add up to it exactly.
        constexpr float kFix = kSumOne / K;   // working units -> fixed point
        int ra = a_own, rb = b_own;
        if constexpr (CF == 1) {
            ra = __float2int_rn(NaK * kFix);
            rb = __float2int_rn(NbK * kFix);
        }
        unsigned long long* const acc = d.acc[PAR ^ 1];
        const unsigned long long pol = l2_keep();
        static_for<1, Q7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            float ux = 0.0f, nn = 0.0f;
            if constexpr (cx(q) != 0) { ux = cx(q) * jx; nn = cx(q) * nx; }
            if constexpr (cy(q) != 0) { ux = cy(q) * jy; nn = cy(q) * ny; }
            if constexpr (cz(q) != 0) { ux = cz(q) * jz; nn = cz(q) * nz; }
            const float base = fmaf(4.5f * iK, ux, 1.0f);
            const int ia = __float2int_rn(w7(q) * NaK * (base + bxa * nn) * kFix);
            const int ib = __float2int_rn(w7(q) * NbK * (base - bxb * nn) * kFix);
            ra -= ia;
            rb -= ib;
            // receiver: x + xi_q if it is a pore site, else x itself (bounce-back)
            int m;
            if constexpr (PAR == 0) {
                m = sc.slot[(q - 1) * sc.stride];
            } else {
                const int sl = sc.slot[(q - 1) * sc.stride];
                m = static_cast<unsigned>(sl) < static_cast<unsigned>(d.n_sites) ? sl : -1;
            }
            if (m >= 0) {
                red_add(acc + m, pack_sums(ia, ib), pol);
            } else {
                ra += ia;
                rb += ib;
            }
        });
        red_add(acc + n, pack_sums(ra, rb), pol);
        // this step's sums of the site are consumed (the phase pass before this
        // collision was their last other reader): they receive the step after next
        st_keep(d.acc[PAR] + n, 0ull, pol);
        return;
    }
    T* const A = static_cast<T*>(d.a);
    T* const B = static_cast<T*>(d.b);
    // fp16 only: K (N - 1)(1 +- phi_c)/2, the offsets of the references
    const float hN = (0.5f * K) * (Nt - 1.0f);
    const float eA = hN * (1.0f + phi_c), eB = hN * (1.0f - phi_c);
    float asum = 0.0f, bsum = 0.0f;
    static_for<1, Q7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        float ux = 0.0f, nn = 0.0f;
        if constexpr (cx(q) != 0) { ux = cx(q) * jx; nn = cx(q) * nx; }
        if constexpr (cy(q) != 0) { ux = cy(q) * jy; nn = cy(q) * ny; }
        if constexpr (cz(q) != 0) { ux = cz(q) * jz; nn = cz(q) * nz; }
        float av, bv;
        if constexpr (S::kRef) {
            const float du = (4.5f * iK) * ux;
            av = w7(q) * NaK * (du + bxa * nn);
            bv = w7(q) * NbK * (du - bxb * nn);
            asum += av;
            bsum += bv;
            av = fmaf(w7(q), eA, av);
            bv = fmaf(w7(q), eB, bv);
        } else {
            const float base = fmaf(4.5f * iK, ux, 1.0f);
            av = w7(q) * NaK * (base + bxa * nn);
            bv = w7(q) * NbK * (base - bxb * nn);
            asum += av;
            bsum += bv;
        }
        S::st_cs(dst(qc, A), av);
        S::st_cs(dst(qc, B), bv);
    });
    if constexpr (S::kRef) {
        // The phase pass adds (1 + S)/2 to the seven values a site reads, S
        // holding w_q phi_c for this site's value of direction q; the seven
        // stored values above sum to Wsum (Na - (1 + phi_c)/2) with Wsum the
        // fp32 weights' sum 1 + 2^-26. The rest value takes the difference,
        // K (1 - Wsum)(Na - 1/2), so that its readers rebuild exactly Na (and
        // Nb) and the fp32 weights create no mass.
        constexpr double kWsum = static_cast<double>(w7(0)) + 6.0 * static_cast<double>(w7(1));
        constexpr float kWerr = static_cast<float>(1.0 - kWsum);
        S::st_cs(A + n, fmaf(kWerr, fmaf(-0.5f, K, NaK), fmaf(w7(0), eA, -asum)));
        S::st_cs(B + n, fmaf(kWerr, fmaf(-0.5f, K, NbK), fmaf(w7(0), eB, -bsum)));
    } else {
        S::st_cs(A + n, NaK - asum);
        S::st_cs(B + n, NbK - bsum);
    }
}

// One site per thread, direct loads.
template <int PAR, class S, int CF = 0>
__device__ __forceinline__ void collide_thread(const DomainView& d, int n, SlotCache sc) {
    const int v = CF != 0 ? ldg_keep(d.site_vox + n, l2_keep()) : __ldg(d.site_vox + n);
    float f[Q19];
    load_f<PAR, S>(d, n, v, f, sc);
    if constexpr (CF != 0 && PAR == 0) {
        // sum form, even step: the face neighbours that receive the component values
        static_for<1, Q7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            sc.slot[(q - 1) * sc.stride] = __ldg(d.vsite + v + stencil_off(d, q));
        });
    }
    // sum form from the sums: the site's own Na, Nb (complete before the
    // previous phase pass, like f)
    int a_own = 0, b_own = 0;
    if constexpr (CF == 2) unpack_sums(ld_keep(d.acc[PAR] + n, l2_keep()), a_own, b_own);

    // Everything above (site and neighbour ids, f and the sums from the
    // previous collision) is safe to read before the phase pass of this step
    // completes; phi and nsum are its outputs, and the A/B slots written below
    // are its inputs.
    allow_next_grid();
    wait_prior_grid();

    const float* pv = d.phi[PAR] + v;
    float phi_c, Nt;
    if constexpr (CF == 2) {
        sums_phase(a_own, b_own, Nt, phi_c);
    } else {
        phi_c = *pv;
        Nt = d.nsum[n];
    }
    float Cx, Cy, Cz;
    color_gradient([&](auto qc) { return pv[stencil_off(d, decltype(qc)::value)]; }, Cx, Cy, Cz);
    if constexpr (S::kRef && CF == 0) {
        // references of the values the next phase pass reads at this site: the
        // phase of x - xi_q, which this step writes, or this site's own on a
        // bounce-back link; every face direction has the same weight
        const unsigned wall = __ldg(d.wall6 + n);
        float Sf = 0.0f;
        static_for<1, Q7>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            Sf += (wall >> (q - 1)) & 1u ? phi_c : pv[stencil_off(d, q)];
        });
        d.rsum[n] = fmaf(w7(1), Sf, w7(0) * phi_c);
    }
    collide_site<PAR, S, CF>(d, n, f, moments(f), phi_c, Nt, a_own, b_own, Cx, Cy, Cz, sc);
}

// ---------------------------------------------------------------------------
// reservoir reset (unsteady protocol, Sec. 4.1): write the rest state into
// the slots the NEXT step (parity PAR) reads.
// ---------------------------------------------------------------------------
// SUMS: the sum form, where the next step reads the component sums (set to
// the reset state Na = 1, Nb = 0 at the inlet, 0 and 1 at the outlet) instead
// of the D3Q7 populations.
template <int PAR, class S, bool SUMS = false>
__device__ __forceinline__ void reservoir_thread(const DomainView& d, int n, int side, float rho_in,
                                                 float rho_out) {
    const int v = d.site_vox[n];
    int nb[Q19];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
        });
    }
    // fp16: the component references of the next step's reads (see StoreF16)
    const unsigned wall = S::kRef ? __ldg(d.wall6 + n) : 0u;
    const float rho = side == 1 ? rho_in : rho_out;
    const float na = side == 1 ? 1.0f : 0.0f;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const size_t i = read_slot<PAR, q>(d, n, nb);
        if constexpr (S::kRef) {
            const float dw = d.drho[f_ref_read<PAR, q>(n, nb)];
            S::template st_fdev<q>(d.f, i, t19(q) * (rho - 1.0f - dw));
        } else {
            S::template st_f<q>(d.f, i, t19(q) * rho);
        }
        if constexpr (q < Q7 && !SUMS) {
            float av = w7(q) * na, bv = w7(q) * (1.0f - na);
            if constexpr (S::kRef) {
                const float pw = writer_phase<PAR, q>(d, v, wall);
                av -= w7(q) * 0.5f * (1.0f + pw);
                bv -= w7(q) * 0.5f * (1.0f - pw);
            }
            S::template st_c<q>(d.a, i, av);
            S::template st_c<q>(d.b, i, bv);
        }
    });
    if constexpr (SUMS) {
        constexpr int one = 1 << 28;   // kSumOne
        d.acc[PAR][n] = side == 1 ? pack_sums(one, 0) : pack_sums(0, one);
    }
}

// ---------------------------------------------------------------------------
// pressure boundary at the z faces (Sec. 4.1: constant inlet and outlet
// pressures; Zou and He's non-equilibrium bounce-back): after streaming, the
// five populations that enter a face site from outside the domain (c_z = +1
// at the inlet z = 0, c_z = -1 at the outlet z = nz - 1) are set so that the
// site's density is the face density and its tangential velocity is zero:
//   u_z = +-(1 - (S_0 + 2 S_out) / rho)      S_0: c_z = 0, S_out: leaving
//   f_in(normal) = f_out(normal) +- rho u_z / 3
//   f_in(edge)   = f_out(opposite edge) +- rho u_z / 6 -+ N_t,
//   N_t = (1/2) sum_{c_z = 0} c_t f   (t = x, y, the tangential momentum)
// The one entering D3Q7 population of each component is the reservoir
// fluid's equilibrium at the face velocity: inlet A = w rho_in (1 + 4.5 u_z),
// B = 0; outlet B = w rho_out (1 - 4.5 u_z), A = 0. The values go into the
// slots the NEXT step (parity PAR) reads.
// ---------------------------------------------------------------------------
// Incoming populations of the next step at face site n as deviations
// d_q = f_q - t_q, and D = S_0 + 2 S_out - 1 in deviations (the weights of
// S_0 + 2 S_out add up to one): u_n is then formed from small numbers and
// rho - 1 instead of cancelling O(1) sums. nb: neighbour ids (filled here).
template <int PAR, class S>
__device__ __forceinline__ float face_deviations(const DomainView& d, int n, float sgn, int (&nb)[Q19],
                                                 float (&dv)[Q19], float& nx, float& ny) {
    const int v = d.site_vox[n];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
        });
    }
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        dv[q] = S::template ld_fdev<q>(d.f, read_slot<PAR, q>(d, n, nb));
        if constexpr (S::kRef) dv[q] = fmaf(t19(q), d.drho[f_ref_read<PAR, q>(n, nb)], dv[q]);
    });
    float D = 0.0f;
    nx = 0.0f;
    ny = 0.0f;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (cz(q) == 0) {
            D += dv[q];
            if constexpr (cx(q) != 0) nx += cx(q) * dv[q];
            if constexpr (cy(q) != 0) ny += cy(q) * dv[q];
        } else {
            if (cz(q) * sgn < 0.0f) D += 2.0f * dv[q];   // leaving the domain through this face
        }
    });
    return D;
}

// face: (rho, rho - 1) of the inlet computed on the device (flux inlet), or
// nullptr to take rho_in, drho_in
template <int PAR, class S>
__device__ __forceinline__ void pressure_face_thread(const DomainView& d, int n, int side, float rho_in,
                                                     float rho_out, float drho_in, float drho_out,
                                                     const float* face) {
    if (face && side == 1) {
        rho_in = face[0];
        drho_in = face[1];
    }
    int nb[Q19];
    float dv[Q19];
    const float sgn = side == 1 ? 1.0f : -1.0f;       // face normal into the domain
    const float rho = side == 1 ? rho_in : rho_out;
    const float drho = side == 1 ? drho_in : drho_out;
    float nx, ny;
    const float D = face_deviations<PAR, S>(d, n, sgn, nb, dv, nx, ny);
    nx *= 0.5f;
    ny *= 0.5f;
    const float un = (drho - D) / rho;                // velocity along the inward normal
    const float j3 = rho * un * (1.0f / 3.0f), j6 = rho * un * (1.0f / 6.0f);
    static_for<1, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (cz(q) != 0) {
            if (cz(q) * sgn > 0.0f) {
                float dev = dv[opp(q)] + (cx(q) == 0 && cy(q) == 0 ? j3 : j6);
                if constexpr (cx(q) != 0) dev -= cx(q) * nx;
                if constexpr (cy(q) != 0) dev -= cy(q) * ny;
                const size_t i = read_slot<PAR, q>(d, n, nb);
                if constexpr (S::kRef) dev = fmaf(-t19(q), d.drho[f_ref_read<PAR, q>(n, nb)], dev);
                S::template st_fdev<q>(d.f, i, dev);
            }
        }
    });
    // the entering component population
    const float uz = sgn * un;
    static_for<5, 7>([&](auto qc) {
        constexpr int q = decltype(qc)::value;   // 5: +z, 6: -z
        if (cz(q) * sgn > 0.0f) {
            const float eq = w7(q) * rho * (1.0f + 4.5f * cz(q) * uz);
            float av = side == 1 ? eq : 0.0f, bv = side == 1 ? 0.0f : eq;
            if constexpr (S::kRef) {
                // the reference the next step reads it with (see StoreF16)
                const float pw = writer_phase<PAR, q>(d, d.site_vox[n], __ldg(d.wall6 + n));
                av -= w7(q) * 0.5f * (1.0f + pw);
                bv -= w7(q) * 0.5f * (1.0f - pw);
            }
            const size_t i = read_slot<PAR, q>(d, n, nb);
            S::template st_c<q>(d.a, i, av);
            S::template st_c<q>(d.b, i, bv);
        }
    });
}

}  // namespace lbm
