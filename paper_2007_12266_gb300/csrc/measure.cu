// Basic analysis and integral measures (Sec. 3.4 table of integral measures;
// Sec. 4 basic analysis: saturation, velocity and pressure per fluid, and the
// instability check), field export and distribution import/export.
//
// The reductions run in a fixed order: each thread walks a fixed strided set
// of sites (compensated fp32, fp64 accuracy, see AccF64), blocks reduce in
// fp64 with warp shuffles and shared memory, and one block reduces the
// per-block partials in fp64. The result depends
// only on the domain, never on timing.
#include <algorithm>
#include <limits>

#include "measure_kernels.cuh"

namespace lbm {

namespace {

constexpr int kBlock = 256;
constexpr int kMeasureBlocks = 152 * 4;     // at least this many blocks (when there are sites for them)
constexpr long long kMeasureSitesPerThread = 64;   // at most this many sites per thread (accuracy, see AccF64)

inline unsigned blocks_for(long long n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_measure(DomainView d, double* partials) {
    AccF64 acc[NSUM];
    for (int n = blockIdx.x * kBlock + threadIdx.x; n < d.n_sites; n += gridDim.x * kBlock)
        measure_site<PAR, S>(d, n, acc);
    block_reduce_sums<kBlock>(acc, partials + static_cast<size_t>(blockIdx.x) * NSUM);
}

__global__ void k_reduce_partials(const double* partials, int nblocks, double* out) {
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (i >= NSUM) return;
    double s = 0.0;
    for (int k = lane; k < nblocks; k += 32) s += partials[static_cast<size_t>(k) * NSUM + i];
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
}

__global__ void k_fill(float* p, long long n, float v) {
    const long long i = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (i < n) p[i] = v;
}

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_field(DomainView d, int which, int nx, int ny, int px,
                                                  int py, float* dense) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    float f[Q19], a[Q7], b[Q7];
    load_site<PAR, S>(d, n, f, a, b);
    float Na = 0.0f, Nb = 0.0f, rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        rho += f[q];
        if constexpr (cx(q) != 0) jx += cx(q) * f[q];
        if constexpr (cy(q) != 0) jy += cy(q) * f[q];
        if constexpr (cz(q) != 0) jz += cz(q) * f[q];
        if constexpr (q < Q7) {
            Na += a[q];
            Nb += b[q];
        }
    });
    float val;
    switch (which) {
    case LBPM_FIELD_PHI: {
        const float Nt = Na + Nb;
        val = Nt > 0.0f ? (Na - Nb) / Nt : 0.0f;
        break;
    }
    case LBPM_FIELD_PRESSURE: val = rho / 3.0f; break;
    case LBPM_FIELD_UX: val = jx + 0.5f * d.fx; break;
    case LBPM_FIELD_UY: val = jy + 0.5f * d.fy; break;
    case LBPM_FIELD_UZ: val = jz + 0.5f * d.fz; break;
    case LBPM_FIELD_NA: val = Na; break;
    case LBPM_FIELD_NB: val = Nb; break;
    default: val = rho; break;
    }
    const int pv = d.site_vox[n];
    const long long X = pv % px, r = pv / px, Y = r % py, Z = r / py;
    dense[(X - 1) + static_cast<long long>(nx) * ((Y - 1) + static_cast<long long>(ny) * (Z - 1))] = val;
}

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_export(DomainView d, int which, float* out) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    float f[Q19], a[Q7], b[Q7];
    load_site<PAR, S>(d, n, f, a, b);
    const size_t N = d.n_sites;
    if (which == LBPM_DIST_F) {
#pragma unroll
        for (int q = 0; q < Q19; ++q) out[q * N + n] = f[q];
    } else {
#pragma unroll
        for (int q = 0; q < Q7; ++q) out[q * N + n] = which == LBPM_DIST_A ? a[q] : b[q];
    }
}

// Canonical distributions of the voxels of a sub-box [lo, hi) of the image,
// one thread per box voxel, out[q][box voxel] (x fastest); solids NaN.
template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_box(DomainView d, int which, int3 lo, int3 ext, float* out) {
    const long long nbox = static_cast<long long>(ext.x) * ext.y * ext.z;
    const long long i = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (i >= nbox) return;
    const int x = static_cast<int>(i % ext.x), r = static_cast<int>(i / ext.x);
    const int y = r % ext.y, z = r / ext.y;
    const int pv = (lo.x + x + 1) + d.px * (lo.y + y + 1) + d.pxpy * (lo.z + z + 1);
    const int n = d.vsite[pv];
    const int Q = which == LBPM_DIST_F ? Q19 : Q7;
    if (n < 0) {
        for (int q = 0; q < Q; ++q) out[q * nbox + i] = __int_as_float(0x7fc00000);   // NaN
        return;
    }
    float f[Q19], a[Q7], b[Q7];
    load_site<PAR, S>(d, n, f, a, b);
    const float* v = which == LBPM_DIST_F ? f : (which == LBPM_DIST_A ? a : b);
    for (int q = 0; q < Q; ++q) out[q * nbox + i] = v[q];
}

// fp16 store: the reference density of imported momentum populations is the
// sum of the imported values at each site (any reference works as long as the
// reader uses the same one); imported component values are stored relative to
// the references the next step reads them with (the previous phase grid).
__global__ void __launch_bounds__(kBlock) k_import_ref(DomainView d, const float* in) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    const size_t N = d.n_sites;
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < Q19; ++q) s += in[q * N + n];
    d.drho[n] = s - 1.0f;
}

template <int PAR, class S>
__global__ void __launch_bounds__(kBlock) k_import(DomainView d, int which, const float* in) {
    const int n = blockIdx.x * kBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    const int v = d.site_vox[n];
    int nb[Q19];
    if constexpr (PAR == 1) {
        static_for<1, Q19>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
        });
    }
    const unsigned wall = S::kRef ? __ldg(d.wall6 + n) : 0u;
    const size_t N = d.n_sites;
    static_for<0, Q19>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const size_t i = read_slot<PAR, q>(d, n, nb);
        if (which == LBPM_DIST_F) {
            float val = in[q * N + n];
            if constexpr (S::kRef) val -= t19(q) * d.drho[f_ref_read<PAR, q>(n, nb)];
            S::template st_f<q>(d.f, i, val);
        }
        if constexpr (q < Q7) {
            if (which != LBPM_DIST_F) {
                float val = in[q * N + n];
                if constexpr (S::kRef) {
                    const float pw = writer_phase<PAR, q>(d, v, wall);
                    val -= w7(q) * 0.5f * (which == LBPM_DIST_A ? 1.0f + pw : 1.0f - pw);
                }
                if (which == LBPM_DIST_A) S::template st_c<q>(d.a, i, val);
                else S::template st_c<q>(d.b, i, val);
            }
        }
    });
}

template <template <int, class> class K, class... Args>
cudaError_t dispatch(const lbpm_ctx* c, int parity, unsigned grid, cudaStream_t s, Args... args) {
    if (grid == 0) return cudaSuccess;
    const bool h = c->params.precision == LBPM_FP16;
    (void)h;
    if (parity == 0) {
        if (h) K<0, StoreF16>::launch(grid, s, args...);
        else K<0, StoreF32>::launch(grid, s, args...);
    } else {
        if (h) K<1, StoreF16>::launch(grid, s, args...);
        else K<1, StoreF32>::launch(grid, s, args...);
    }
    return cudaGetLastError();
}

template <int PAR, class S>
struct MeasureK {
    static void launch(unsigned g, cudaStream_t s, DomainView d, double* p) {
        k_measure<PAR, S><<<g, kBlock, 0, s>>>(d, p);
    }
};
template <int PAR, class S>
struct FieldK {
    static void launch(unsigned g, cudaStream_t s, DomainView d, int w, int nx, int ny, int px, int py,
                       float* o) {
        k_field<PAR, S><<<g, kBlock, 0, s>>>(d, w, nx, ny, px, py, o);
    }
};
template <int PAR, class S>
struct ExportK {
    static void launch(unsigned g, cudaStream_t s, DomainView d, int w, float* o) {
        k_export<PAR, S><<<g, kBlock, 0, s>>>(d, w, o);
    }
};
template <int PAR, class S>
struct BoxK {
    static void launch(unsigned g, cudaStream_t s, DomainView d, int w, int3 lo, int3 ext, float* o) {
        k_box<PAR, S><<<g, kBlock, 0, s>>>(d, w, lo, ext, o);
    }
};
template <int PAR, class S>
struct ImportK {
    static void launch(unsigned g, cudaStream_t s, DomainView d, int w, const float* i) {
        k_import<PAR, S><<<g, kBlock, 0, s>>>(d, w, i);
    }
};

}  // namespace

// d_out receives NSUM doubles. Uses c->d_partials (allocated on demand).
cudaError_t launch_measure(lbpm_ctx* c, int parity, double* d_out, cudaStream_t s) {
    // enough blocks that no thread sums more than kMeasureSitesPerThread sites
    long long nb = (c->N + kBlock - 1) / kBlock;
    const long long need = (c->N + kBlock * kMeasureSitesPerThread - 1) / (kBlock * kMeasureSitesPerThread);
    nb = std::min(nb, std::max<long long>(kMeasureBlocks, need));
    if (nb < 1) nb = 1;
    if (c->n_partials < nb) {
        dfree(c, c->d_partials);
        c->d_partials = static_cast<double*>(dalloc(c, sizeof(double) * NSUM * nb));
        if (!c->d_partials) return cudaErrorMemoryAllocation;
        c->n_partials = nb;
    }
    cudaError_t e = dispatch<MeasureK>(c, parity, static_cast<unsigned>(nb), s, make_view(c), c->d_partials);
    if (e != cudaSuccess) return e;
    k_reduce_partials<<<1, 32 * NSUM, 0, s>>>(c->d_partials, static_cast<int>(nb), d_out);
    return cudaGetLastError();
}

cudaError_t launch_field(const lbpm_ctx* c, int parity, int which, float* dense, cudaStream_t s) {
    k_fill<<<blocks_for(c->V), kBlock, 0, s>>>(dense, c->V, std::numeric_limits<float>::quiet_NaN());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return dispatch<FieldK>(c, parity, blocks_for(c->N), s, make_view(c), which, c->nx, c->ny, c->px,
                            c->py, dense);
}

cudaError_t launch_export_dist(const lbpm_ctx* c, int parity, int which, float* out, cudaStream_t s) {
    return dispatch<ExportK>(c, parity, blocks_for(c->N), s, make_view(c), which, out);
}

cudaError_t launch_read_box(const lbpm_ctx* c, int parity, int which, const int* lo, const int* hi, float* out,
                            cudaStream_t s) {
    const int3 l = make_int3(lo[0], lo[1], lo[2]);
    const int3 ext = make_int3(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]);
    const long long nbox = static_cast<long long>(ext.x) * ext.y * ext.z;
    return dispatch<BoxK>(c, parity, blocks_for(nbox), s, make_view(c), which, l, ext, out);
}

cudaError_t launch_import_dist(const lbpm_ctx* c, int parity, int which, const float* in, cudaStream_t s) {
    if (c->params.precision == LBPM_FP16 && c->N > 0 && which == LBPM_DIST_F) {
        k_import_ref<<<blocks_for(c->N), kBlock, 0, s>>>(make_view(c), in);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = dispatch<ImportK>(c, parity, blocks_for(c->N), s, make_view(c), which, in);
    if (e != cudaSuccess) return e;
    return launch_ref_sum(c, parity, s);   // fp16: the phase pass's references of the imported state
}

}  // namespace lbm
