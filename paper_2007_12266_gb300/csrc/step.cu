// Single-domain launchers of the timestep kernels (Sec. 3.1) and fluid
// initialisation.
#include "step_kernels.cuh"

namespace lbm {

namespace {

constexpr int kBlock = 256;

// Launch with programmatic stream serialization (see wait_prior_grid()).
template <class... KArgs, class... Args>
cudaError_t launch_pdl_bt(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
    return launch_pdl_bt(kernel, grid, kBlock, s, args...);
}

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_phase(DomainView d) {
    const int t = blockIdx.x * kBlock + threadIdx.x;
    phase_thread<PAR, S>(d, t);
}

constexpr int kPhaseSumPer = 2;   // entries per thread of the sum-form phase pass (1, 2, 4, 8 measured; 2 fastest)

template <int PAR, bool WRITE_N>
__global__ void __launch_bounds__(kBlock) k_phase_sum(DomainView d) {
    phase_sum_thread<PAR, WRITE_N, kPhaseSumPer>(d, blockIdx.x * kBlock * kPhaseSumPer + threadIdx.x, kBlock);
}

// Launch shape of the collision: 56 registers and 36 resident warps per SM
// (six blocks of 192 threads in FP32, nine of 128 in FP16) measured 4-5 %
// faster on the 256^3 workload than 64 registers and 32 warps (four blocks of
// 256), which leaves fewer warps to cover the memory latency.
template <class S>
struct CollideShape {
    static constexpr int kThreads = S::kRef ? 128 : 192;
    static constexpr int kBlocksPerSm = S::kRef ? 9 : 6;
};

// CF: component form of the collision (see collide_site)
template <int PAR, class S, int CF>
__global__ void __launch_bounds__(CollideShape<S>::kThreads, CollideShape<S>::kBlocksPerSm) k_collide(DomainView d) {
    constexpr int BT = CollideShape<S>::kThreads;
    // odd steps: slot (and fp16 reference) cache, see SlotCache; even steps of
    // the sum form: the six face neighbours
    constexpr int kSlots = PAR == 1 ? (Q19 - 1) * BT : (CF != 0 ? (Q7 - 1) * BT : 1);
    constexpr int kRefs = PAR == 1 && S::kRef ? (Q19 - 1) * BT : 1;
    __shared__ int slot[kSlots];
    __shared__ float ref[kRefs];
    const int n = blockIdx.x * BT + threadIdx.x;
    if (n < d.n_sites) collide_thread<PAR, S, CF>(d, n, SlotCache{slot + threadIdx.x, ref + threadIdx.x, BT});
}

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_pressure_faces(DomainView d, const int* sites,
                                                           const signed char* side, int n_face,
                                                           float rho_in, float rho_out, float drho_in,
                                                           float drho_out, const float* face) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n_face) pressure_face_thread<PAR, S>(d, sites[i], side[i], rho_in, rho_out, drho_in, drho_out, face);
}

// Flux inlet, first half: per-block sums (fixed grid, fixed order: the result
// does not depend on scheduling) of D_s over the inlet sites and their count.
template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_face_sum(DomainView d, const int* sites, const signed char* side,
                                                     int n_face, double* part) {
    __shared__ double sd[kBlock];
    __shared__ double sc[kBlock];
    double acc = 0.0, cnt = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n_face; i += kFaceBlocks * kBlock) {
        if (side[i] != 1) continue;
        int nb[Q19];
        float dv[Q19], nx, ny;
        acc += face_deviations<PAR, S>(d, sites[i], 1.0f, nb, dv, nx, ny);
        cnt += 1.0;
    }
    sd[threadIdx.x] = acc;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sd[0];
        part[2 * blockIdx.x + 1] = sc[0];
    }
}

// Second half: rho_in - 1 = (sum D + Q) / (n_in - Q), from sum_s (1 + D_s) / (n_in - Q).
__global__ void k_face_rho(const double* part, double flux, float* face) {
    if (threadIdx.x != 0) return;
    double D = 0.0, n = 0.0;
    for (int b = 0; b < kFaceBlocks; ++b) {
        D += part[2 * b];
        n += part[2 * b + 1];
    }
    const double drho = n > flux ? (D + flux) / (n - flux) : 0.0;
    face[0] = static_cast<float>(1.0 + drho);
    face[1] = static_cast<float>(drho);
}

template <int PAR, class S, bool SUMS>
__global__ void __launch_bounds__(kBlock) k_reservoir(DomainView d, const int* sites,
                                                      const signed char* side, int n_slab,
                                                      float rho_in, float rho_out) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n_slab) reservoir_thread<PAR, S, SUMS>(d, sites[i], side[i], rho_in, rho_out);
}

__device__ __forceinline__ float phi0_of_site(const DomainView& d, int n, const float* phi0, int nx, int ny,
                                              int px, int pxpy) {
    const int v = d.site_vox[n];
    const int z = v / pxpy - 1;
    const int r = v - (z + 1) * pxpy;
    const int y = r / px - 1;
    const int x = r - (y + 1) * px - 1;
    const float p = phi0[static_cast<size_t>(x) + static_cast<size_t>(nx) * (y + static_cast<size_t>(ny) * z)];
    return fminf(1.0f, fmaxf(-1.0f, p));
}

// The phase grid that step 0 reads as the previous step's: phi0 (fp16
// storage: the references of the initial component values).
__global__ void __launch_bounds__(kBlock) k_init_phase(DomainView d, const float* phi0, int nx, int ny, int px,
                                                       int pxpy) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    d.phi[1][d.site_vox[n]] = phi0_of_site(d, n, phi0, nx, ny, px, pxpy);
}

// fp16 storage: the references' phase sum of every site for a step of parity
// PAR (what the collision stores in rsum), after an initialisation or an import.
template <int PAR>
__global__ void __launch_bounds__(kBlock) k_ref_sum(DomainView d) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    d.rsum[n] = reference_phase_sum<PAR>(d, n, d.site_vox[n]);
}

// Initial state consistent with phi0 (rho = 1, u = 0), written in the even
// (natural) layout: Na = (1 + phi0)/2, Nb = (1 - phi0)/2. With fp16 storage the
// density reference is rho = 1 and the component references come from the
// phase grid that k_init_phase wrote (periodic mirrors included).
template <class S>
__global__ void __launch_bounds__(kBlock) k_init(DomainView d, const float* phi0, int nx, int ny,
                                                 int px, int pxpy) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    const float p = phi0_of_site(d, n, phi0, nx, ny, px, pxpy);
    const float na = 0.5f * (1.0f + p), nb = 0.5f * (1.0f - p);
    const int v = d.site_vox[n];
    unsigned wall = 0;
    if constexpr (S::kRef) {
        d.drho[n] = 0.0f;
        wall = __ldg(d.wall6 + n);
    }
    const size_t N = d.n_sites;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        S::template st_f<q>(d.f, q * N + n, t19(q));
        if constexpr (q < Q7) {
            float av = w7(q) * na, bv = w7(q) * nb;
            if constexpr (S::kRef) {
                const float pw = writer_phase<0, q>(d, v, wall);
                av -= w7(q) * 0.5f * (1.0f + pw);
                bv -= w7(q) * 0.5f * (1.0f - pw);
            }
            S::template st_c<q>(d.a, q * N + n, av);
            S::template st_c<q>(d.b, q * N + n, bv);
        }
    });
}

inline unsigned blocks_for(long long n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

}  // namespace

DomainView make_view(const lbpm_ctx* c) {
    DomainView d{};
    d.n_sites = static_cast<int>(c->N);
    d.n_halo = static_cast<int>(c->H);
    d.px = static_cast<int>(c->px);
    d.pxpy = static_cast<int>(c->px * c->py);
    d.site_vox = c->d_site_vox;
    d.vsite = c->d_vsite;
    d.phi[0] = c->d_phi;
    d.phi[1] = c->d_phi_alt ? c->d_phi_alt : c->d_phi;
    d.halo_dst = c->d_halo_dst;
    d.halo_site = c->d_halo_site;
    d.wall6 = c->d_wall6;
    d.nsum = c->d_nsum;
    d.drho = c->d_drho;
    d.rsum = c->d_rsum;
    d.f = c->d_f;
    d.a = c->d_a;
    d.b = c->d_b;
    d.acc[0] = c->d_acc;
    d.acc[1] = c->d_acc ? c->d_acc + c->N : nullptr;
    const lbpm_params& p = c->params;
    d.tau_a = static_cast<float>(p.tau_a);
    d.tau_b = static_cast<float>(p.tau_b);
    d.alpha = static_cast<float>(p.alpha);
    d.beta = static_cast<float>(p.beta);
    d.fx = static_cast<float>(p.force[0]);
    d.fy = static_cast<float>(p.force[1]);
    d.fz = static_cast<float>(p.force[2]);
    const float K = p.precision == LBPM_FP16 ? StoreF16::kK : StoreF32::kK;
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        d.fterm[k] = K * (3.0f * t19(q) * (cx(q) * d.fx + cy(q) * d.fy + cz(q) * d.fz));
    }
    d.uniform_tau = p.tau_a == p.tau_b;
    const float s_nu = 1.0f / static_cast<float>(p.tau_a);
    d.s_nu = s_nu;
    d.s_m = 8.0f * (2.0f - s_nu) / (8.0f - s_nu);
    return d;
}

cudaError_t launch_init_fluids(const lbpm_ctx* c, const float* phi0, cudaStream_t s) {
    DomainView d = make_view(c);
    if (c->N == 0) return cudaSuccess;
    const bool h = c->params.precision == LBPM_FP16;
    if (h) {
        k_init_phase<<<blocks_for(c->N), kBlock, 0, s>>>(d, phi0, c->nx, c->ny, c->px, c->px * c->py);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_fill_halo(c, s);   // periodic mirrors of the initial phase
        if (e != cudaSuccess) return e;
        k_init<StoreF16><<<blocks_for(c->N), kBlock, 0, s>>>(d, phi0, c->nx, c->ny, c->px, c->px * c->py);
        k_ref_sum<0><<<blocks_for(c->N), kBlock, 0, s>>>(d);
    } else {
        k_init<StoreF32><<<blocks_for(c->N), kBlock, 0, s>>>(d, phi0, c->nx, c->ny, c->px, c->px * c->py);
    }
    return cudaGetLastError();
}

cudaError_t launch_ref_sum(const lbpm_ctx* c, int parity, cudaStream_t s) {
    if (c->params.precision != LBPM_FP16 || c->N == 0) return cudaSuccess;
    if (parity == 0) k_ref_sum<0><<<blocks_for(c->N), kBlock, 0, s>>>(make_view(c));
    else k_ref_sum<1><<<blocks_for(c->N), kBlock, 0, s>>>(make_view(c));
    return cudaGetLastError();
}

cudaError_t launch_phase(const lbpm_ctx* c, int parity, cudaStream_t s) {
    DomainView d = make_view(c);
    const unsigned g = blocks_for(c->N + c->H);
    if (g == 0) return cudaSuccess;
    const bool h = c->params.precision == LBPM_FP16;
    if (parity == 0) return h ? launch_pdl(k_phase<0, StoreF16>, g, s, d) : launch_pdl(k_phase<0, StoreF32>, g, s, d);
    return h ? launch_pdl(k_phase<1, StoreF16>, g, s, d) : launch_pdl(k_phase<1, StoreF32>, g, s, d);
}

// one collision launch of the given parity, storage and component form
template <int PAR, int CF>
cudaError_t launch_collide_form(const lbpm_ctx* c, cudaStream_t s) {
    if (c->N == 0) return cudaSuccess;
    DomainView d = make_view(c);
    if (c->params.precision == LBPM_FP16) {
        constexpr int bt = CollideShape<StoreF16>::kThreads;
        return launch_pdl_bt(k_collide<PAR, StoreF16, CF>, static_cast<unsigned>((c->N + bt - 1) / bt), bt, s, d);
    }
    constexpr int bt = CollideShape<StoreF32>::kThreads;
    return launch_pdl_bt(k_collide<PAR, StoreF32, CF>, static_cast<unsigned>((c->N + bt - 1) / bt), bt, s, d);
}

cudaError_t launch_collide(const lbpm_ctx* c, int parity, cudaStream_t s) {
    return parity == 0 ? launch_collide_form<0, 0>(c, s) : launch_collide_form<1, 0>(c, s);
}

cudaError_t launch_phase_sum(const lbpm_ctx* c, int parity, bool write_nsum, cudaStream_t s) {
    DomainView d = make_view(c);
    const unsigned g = blocks_for((c->N + c->H + kPhaseSumPer - 1) / kPhaseSumPer);
    if (g == 0) return cudaSuccess;
    if (parity == 0) return write_nsum ? launch_pdl(k_phase_sum<0, true>, g, s, d) : launch_pdl(k_phase_sum<0, false>, g, s, d);
    return write_nsum ? launch_pdl(k_phase_sum<1, true>, g, s, d) : launch_pdl(k_phase_sum<1, false>, g, s, d);
}

cudaError_t launch_collide_sum(const lbpm_ctx* c, int parity, bool from_sums, cudaStream_t s) {
    if (from_sums) return parity == 0 ? launch_collide_form<0, 2>(c, s) : launch_collide_form<1, 2>(c, s);
    return parity == 0 ? launch_collide_form<0, 1>(c, s) : launch_collide_form<1, 1>(c, s);
}

// parity = parity of the step that will READ the reset values; reservoir slabs
// (reservoir_z = 1) or the pressure boundary at the z faces (reservoir_z = 2)
cudaError_t launch_reservoir(const lbpm_ctx* c, int parity, cudaStream_t s) {
    if (c->n_slab == 0) return cudaSuccess;
    DomainView d = make_view(c);
    const unsigned g = blocks_for(c->n_slab);
    const int ns = static_cast<int>(c->n_slab);
    const float ri = static_cast<float>(c->params.rho_in), ro = static_cast<float>(c->params.rho_out);
    const bool h = c->params.precision == LBPM_FP16;
    if (c->params.reservoir_z >= 2) {   // pressure faces; flux inlet (3)
        // rho - 1 formed in double, so the small difference keeps full fp32 precision
        const float di = static_cast<float>(c->params.rho_in - 1.0), dout = static_cast<float>(c->params.rho_out - 1.0);
        const int* st = c->d_slab_site;
        const signed char* sd = c->d_slab_side;
        float* face = nullptr;
        if (c->params.reservoir_z == 3) {
            face = c->d_face_rho;
            double* part = c->d_face_part;
            if (parity == 0) {
                if (h) k_face_sum<0, StoreF16><<<kFaceBlocks, kBlock, 0, s>>>(d, st, sd, ns, part);
                else k_face_sum<0, StoreF32><<<kFaceBlocks, kBlock, 0, s>>>(d, st, sd, ns, part);
            } else {
                if (h) k_face_sum<1, StoreF16><<<kFaceBlocks, kBlock, 0, s>>>(d, st, sd, ns, part);
                else k_face_sum<1, StoreF32><<<kFaceBlocks, kBlock, 0, s>>>(d, st, sd, ns, part);
            }
            k_face_rho<<<1, 32, 0, s>>>(part, c->params.flux_in, face);
        }
        if (parity == 0) {
            if (h) k_pressure_faces<0, StoreF16><<<g, kBlock, 0, s>>>(d, st, sd, ns, ri, ro, di, dout, face);
            else k_pressure_faces<0, StoreF32><<<g, kBlock, 0, s>>>(d, st, sd, ns, ri, ro, di, dout, face);
        } else {
            if (h) k_pressure_faces<1, StoreF16><<<g, kBlock, 0, s>>>(d, st, sd, ns, ri, ro, di, dout, face);
            else k_pressure_faces<1, StoreF32><<<g, kBlock, 0, s>>>(d, st, sd, ns, ri, ro, di, dout, face);
        }
        return cudaGetLastError();
    }
    if (parity == 0) {
        if (h) k_reservoir<0, StoreF16, false><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
        else k_reservoir<0, StoreF32, false><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
    } else {
        if (h) k_reservoir<1, StoreF16, false><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
        else k_reservoir<1, StoreF32, false><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
    }
    return cudaGetLastError();
}

cudaError_t launch_reservoir_sum(const lbpm_ctx* c, int parity, cudaStream_t s) {
    if (c->n_slab == 0 || c->params.reservoir_z != 1) return cudaSuccess;
    DomainView d = make_view(c);
    const unsigned g = blocks_for(c->n_slab);
    const int ns = static_cast<int>(c->n_slab);
    const float ri = static_cast<float>(c->params.rho_in), ro = static_cast<float>(c->params.rho_out);
    const bool h = c->params.precision == LBPM_FP16;
    if (parity == 0) {
        if (h) k_reservoir<0, StoreF16, true><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
        else k_reservoir<0, StoreF32, true><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
    } else {
        if (h) k_reservoir<1, StoreF16, true><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
        else k_reservoir<1, StoreF32, true><<<g, kBlock, 0, s>>>(d, c->d_slab_site, c->d_slab_side, ns, ri, ro);
    }
    return cudaGetLastError();
}

}  // namespace lbm
