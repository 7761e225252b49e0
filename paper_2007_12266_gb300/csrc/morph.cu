// Shell aggregation (Sec. 3.3, shell aggregation protocol): move the
// fluid-fluid interface of fluid a by a signed distance delta (dilation > 0,
// erosion < 0) through its distance map, then re-initialise the component
// densities consistently with the new phase field.
//
//   Phi_a   signed distance to the interface, < 0 inside fluid a (phi > 0).
//           Near the interface it is Eq. lb-dist solved for the distance,
//           Phi = -atanh(phi) / beta, used where |phi| < tanh(3 beta) (the
//           equilibrium profile gives it to about three voxels); further out
//           it is min over those band voxels y within R of |x - y| + |Phi(y)|
//           (the far-field rule); voxels with no band voxel within R keep
//           their phase.
//   Phi'    = Phi - delta (the dilated set {Phi < delta} has its boundary at
//           Phi' = 0).
//   phi'    = -tanh(beta Phi'), Eq. lb-dist-to-phase.
//   A_q, B_q = w_q N (1 +- phi') / 2 at the changed sites, N = Na + Nb kept.
//
// Two kernels: the first writes phi and the band distance |Phi| of every site
// onto dense voxel grids (solid NaN / +inf), the second forms phi' from them,
// counts the sites of fluid a before and after, and (apply) rewrites A and B
// in the slots the next step reads.
#include <cmath>
#include <vector>

#include "measure_kernels.cuh"

namespace lbm {

namespace {

constexpr int kMorphBlock = 256;

struct MorphGrid {
    int nx, ny, nz;
    int per[3];
    float* phi;      // [V] phase of the site at each voxel, NaN on solid
    float* dist;     // [V] |Phi| for band voxels, +inf otherwise
    float* ntot;     // [N] Na + Nb per site
};

__device__ __forceinline__ void site_xyz(const DomainView& d, int v, int& x, int& y, int& z) {
    z = v / d.pxpy - 1;
    const int r = v - (z + 1) * d.pxpy;
    y = r / d.px - 1;
    x = r - (y + 1) * d.px - 1;
}

template <int PAR, class S>
__global__ void __launch_bounds__(kMorphBlock) k_morph_phase(DomainView d, MorphGrid g, float phi_band, float inv_beta) {
    const int n = blockIdx.x * kMorphBlock + threadIdx.x;
    if (n >= d.n_sites) return;
    float f[Q19], a[Q7], b[Q7];
    load_site<PAR, S>(d, n, f, a, b);
    float Na = 0.0f, Nb = 0.0f;
#pragma unroll
    for (int q = 0; q < Q7; ++q) {
        Na += a[q];
        Nb += b[q];
    }
    const float Nt = Na + Nb;
    const float phi = Nt > 0.0f ? (Na - Nb) / Nt : 0.0f;
    int x, y, z;
    site_xyz(d, d.site_vox[n], x, y, z);
    const long long u = x + static_cast<long long>(g.nx) * (y + static_cast<long long>(g.ny) * z);
    g.phi[u] = phi;
    g.dist[u] = fabsf(phi) < phi_band ? fabsf(atanhf(phi)) * inv_beta : INFINITY;
    g.ntot[n] = Nt;
}

template <int PAR, class S>
__global__ void __launch_bounds__(kMorphBlock) k_morph_apply(DomainView d, MorphGrid g, const int3* off,
                                                             const long long* off_lin, const float* off_len,
                                                             int n_off, int R, float beta, float delta, int apply,
                                                             unsigned long long* counts) {
    const int n = blockIdx.x * kMorphBlock + threadIdx.x;
    int before = 0, after = 0;
    if (n < d.n_sites) {
        const int v = d.site_vox[n];
        int c[3];
        site_xyz(d, v, c[0], c[1], c[2]);
        const long long u = c[0] + static_cast<long long>(g.nx) * (c[1] + static_cast<long long>(g.ny) * c[2]);
        const float phi = g.phi[u];
        float Phi = NAN;
        const float own = g.dist[u];
        if (own < INFINITY) {
            Phi = phi > 0.0f ? -own : own;     // band: Eq. lb-dist
        } else {
            // far field: nearest band voxel within R, through its own distance;
            // voxels at least R from every face use linear offsets
            const int dims[3] = {g.nx, g.ny, g.nz};
            float best = INFINITY;
            const bool interior = c[0] >= R && c[0] < g.nx - R && c[1] >= R && c[1] < g.ny - R && c[2] >= R &&
                                  c[2] < g.nz - R;
            if (interior) {
                for (int i = 0; i < n_off; ++i) best = fminf(best, off_len[i] + g.dist[u + off_lin[i]]);
            }
            for (int i = 0; i < (interior ? 0 : n_off); ++i) {
                long long w = 0;
                bool inside = true;
                const int o[3] = {off[i].x, off[i].y, off[i].z};
                long long stride = 1;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int xx = c[a] + o[a];
                    if (xx < 0 || xx >= dims[a]) {
                        if (!g.per[a]) {
                            inside = false;
                            break;
                        }
                        xx = ((xx % dims[a]) + dims[a]) % dims[a];
                    }
                    w += xx * stride;
                    stride *= dims[a];
                }
                if (inside) best = fminf(best, off_len[i] + g.dist[w]);
            }
            if (best < INFINITY) Phi = phi > 0.0f ? -best : best;
        }
        before = phi > 0.0f;
        after = before;
        if (Phi == Phi) {   // not far from the interface
            const float phin = -tanhf(beta * (Phi - delta));   // Eq. lb-dist-to-phase
            after = phin > 0.0f;
            if (apply) {
                const float N = g.ntot[n];
                int nb[Q19];
                if constexpr (PAR == 1) {
                    static_for<1, Q19>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        nb[q] = __ldg(d.vsite + v + stencil_off(d, q));
                    });
                }
                const float na = 0.5f * N * (1.0f + phin), nbb = 0.5f * N * (1.0f - phin);
                const unsigned wall = S::kRef ? __ldg(d.wall6 + n) : 0u;
                static_for<0, Q7>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    float av = w7(q) * na, bv = w7(q) * nbb;
                    if constexpr (S::kRef) {
                        // the reference the next step reads it with
                        const float pw = writer_phase<PAR, q>(d, v, wall);
                        av -= w7(q) * 0.5f * (1.0f + pw);
                        bv -= w7(q) * 0.5f * (1.0f - pw);
                    }
                    const size_t i = read_slot<PAR, q>(d, n, nb);
                    S::template st_c<q>(d.a, i, av);
                    S::template st_c<q>(d.b, i, bv);
                });
            }
        }
    }
    // exact integer counts: warp sums, one atomic per warp
    const unsigned full = 0xffffffffu;
    const int sb = __popc(__ballot_sync(full, before != 0));
    const int sa = __popc(__ballot_sync(full, after != 0));
    if ((threadIdx.x & 31) == 0) {
        if (sb) atomicAdd(counts, static_cast<unsigned long long>(sb));
        if (sa) atomicAdd(counts + 1, static_cast<unsigned long long>(sa));
    }
}

unsigned blocks_of(long long n) { return static_cast<unsigned>((n + kMorphBlock - 1) / kMorphBlock); }

}  // namespace

cudaError_t launch_morph(const lbpm_ctx* c, int parity, float delta, int R, int apply, float* phi_grid,
                         float* dist_grid, float* ntot, int3* off, long long* off_lin, float* off_len, int n_off,
                         unsigned long long* counts, cudaStream_t s) {
    DomainView d = make_view(c);
    MorphGrid g{c->nx, c->ny, c->nz, {c->params.periodic[0], c->params.periodic[1], c->params.periodic[2]},
                phi_grid, dist_grid, ntot};
    const float beta = static_cast<float>(c->params.beta);
    const float phi_band = std::tanh(3.0f * beta);
    const bool h = c->params.precision == LBPM_FP16;
    const unsigned gN = blocks_of(c->N);
    if (gN == 0) return cudaSuccess;
    if (parity == 0) {
        if (h) k_morph_phase<0, StoreF16><<<gN, kMorphBlock, 0, s>>>(d, g, phi_band, 1.0f / beta);
        else k_morph_phase<0, StoreF32><<<gN, kMorphBlock, 0, s>>>(d, g, phi_band, 1.0f / beta);
    } else {
        if (h) k_morph_phase<1, StoreF16><<<gN, kMorphBlock, 0, s>>>(d, g, phi_band, 1.0f / beta);
        else k_morph_phase<1, StoreF32><<<gN, kMorphBlock, 0, s>>>(d, g, phi_band, 1.0f / beta);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (parity == 0) {
        if (h) k_morph_apply<0, StoreF16><<<gN, kMorphBlock, 0, s>>>(d, g, off, off_lin, off_len, n_off, R, beta, delta, apply, counts);
        else k_morph_apply<0, StoreF32><<<gN, kMorphBlock, 0, s>>>(d, g, off, off_lin, off_len, n_off, R, beta, delta, apply, counts);
    } else {
        if (h) k_morph_apply<1, StoreF16><<<gN, kMorphBlock, 0, s>>>(d, g, off, off_lin, off_len, n_off, R, beta, delta, apply, counts);
        else k_morph_apply<1, StoreF32><<<gN, kMorphBlock, 0, s>>>(d, g, off, off_lin, off_len, n_off, R, beta, delta, apply, counts);
    }
    return cudaGetLastError();
}

}  // namespace lbm
