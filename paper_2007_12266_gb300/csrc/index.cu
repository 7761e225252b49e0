// Sparse pore-site indexer on the device.
//
// Pore voxels (label 0, Sec. 3.3) are numbered in x-fastest lexicographic
// order by an exclusive prefix sum over the pore flags, which makes the site
// numbering identical to a sequential scan of the image. Two padded grids
// (one halo voxel per face) then resolve neighbours without branches:
// vsite[pv] is the site id of padded voxel pv (-1: solid or wall) and
// phi[pv] holds the phase field, with phi_s (Sec. 3.2, Eq. phi_s) at solids and
// 0 outside non-periodic faces. Halo voxels of periodic axes copy the voxel
// they wrap to; those that mirror pores are listed so the phase pass can
// refresh them every step.
#include "internal.h"
#include "lattice.cuh"

namespace lbm {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;
constexpr int kBlock = 256;

inline unsigned blocks_for(long long n, int b = kBlock) { return static_cast<unsigned>((n + b - 1) / b); }

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive block scan of one value per thread; returns the block total
__device__ int block_excl_scan(int v, int& total) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const int before = w > 0 ? warp_tot[w - 1] : 0;
    total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int* in, long long n, int* sums) {
    const long long base = static_cast<long long>(blockIdx.x) * kTile;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + static_cast<long long>(i) * kScanThreads + threadIdx.x;
        if (j < n) s += in[j];
    }
    int total;
    block_excl_scan(s, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const int* in, long long n, int* out,
                                                            const int* offsets) {
    const long long base = static_cast<long long>(blockIdx.x) * kTile + static_cast<long long>(threadIdx.x) * kScanItems;
    int vals[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + i;
        vals[i] = j < n ? in[j] : 0;
        s += vals[i];
    }
    int total;
    int run = block_excl_scan(s, total) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long j = base + i;
        if (j < n) out[j] = run;
        run += vals[i];
    }
}

__device__ __forceinline__ long long padded_of(long long v, int nx, int ny, int px, int py) {
    const long long x = v % nx;
    const long long r = v / nx;
    const long long y = r % ny;
    const long long z = r / ny;
    return (x + 1) + static_cast<long long>(px) * ((y + 1) + static_cast<long long>(py) * (z + 1));
}

__global__ void k_flag_pore(const uint16_t* labels, long long V, int* flags) {
    const long long v = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (v < V) flags[v] = labels[v] == 0 ? 1 : 0;
}

__global__ void k_scatter_sites(const uint16_t* labels, const int* scan, long long V, int nx, int ny,
                                int px, int py, int* site_vox, int* vsite, float* phi) {
    const long long v = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (v >= V) return;
    const long long pv = padded_of(v, nx, ny, px, py);
    if (labels[v] == 0) {
        const int s = scan[v];
        site_vox[s] = static_cast<int>(pv);
        vsite[pv] = s;
    } else {
        vsite[pv] = -1;
    }
    phi[pv] = 0.0f;
}

// Resolve a padded voxel: returns 0 for interior voxels, 1 for a halo voxel
// that wraps to padded voxel *src, 2 for a wall (outside a non-periodic face).
__device__ __forceinline__ int halo_kind(long long pv, int nx, int ny, int nz, int px, int py,
                                         int perx, int pery, int perz, long long* src) {
    long long X = pv % px;
    const long long r = pv / px;
    long long Y = r % py;
    long long Z = r / py;
    const bool interior = X >= 1 && X <= nx && Y >= 1 && Y <= ny && Z >= 1 && Z <= nz;
    if (interior) return 0;
    bool wall = false;
    if (X == 0) { if (perx) X = nx; else wall = true; }
    else if (X == nx + 1) { if (perx) X = 1; else wall = true; }
    if (Y == 0) { if (pery) Y = ny; else wall = true; }
    else if (Y == ny + 1) { if (pery) Y = 1; else wall = true; }
    if (Z == 0) { if (perz) Z = nz; else wall = true; }
    else if (Z == nz + 1) { if (perz) Z = 1; else wall = true; }
    if (wall) return 2;
    *src = X + static_cast<long long>(px) * (Y + static_cast<long long>(py) * Z);
    return 1;
}

struct Geo {
    int nx, ny, nz, px, py, perx, pery, perz;
    long long Vp;
};

Geo geo_of(const lbpm_ctx* c) {
    return Geo{c->nx, c->ny, c->nz, c->px, c->py, c->params.periodic[0], c->params.periodic[1],
               c->params.periodic[2], c->Vp};
}

// phi2: the second phase grid (fp16 storage), or nullptr
__global__ void k_fill_halo(Geo g, int* vsite, float* phi, float* phi2) {
    const long long pv = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (pv >= g.Vp) return;
    long long src = 0;
    const int k = halo_kind(pv, g.nx, g.ny, g.nz, g.px, g.py, g.perx, g.pery, g.perz, &src);
    if (k == 1) {
        vsite[pv] = vsite[src];
        phi[pv] = phi[src];
        if (phi2) phi2[pv] = phi2[src];
    } else if (k == 2) {
        vsite[pv] = -1;
        phi[pv] = 0.0f;
        if (phi2) phi2[pv] = 0.0f;
    }
}

__global__ void k_halo_flags(Geo g, const int* vsite, int* flags) {
    const long long pv = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (pv >= g.Vp) return;
    long long src = 0;
    const int k = halo_kind(pv, g.nx, g.ny, g.nz, g.px, g.py, g.perx, g.pery, g.perz, &src);
    flags[pv] = (k == 1 && vsite[pv] >= 0) ? 1 : 0;
}

__global__ void k_halo_scatter(long long Vp, const int* flags, const int* scan, const int* vsite,
                               int* halo_dst, int* halo_site) {
    const long long pv = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (pv >= Vp || !flags[pv]) return;
    const int e = scan[pv];
    halo_dst[e] = static_cast<int>(pv);
    halo_site[e] = vsite[pv];
}

__global__ void k_affinity_table(const uint16_t* labels, long long V, int nx, int ny, int px, int py,
                                 const float* table, int n_labels, float* phi, float* phi2) {
    const long long v = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (v >= V) return;
    const int lab = labels[v];
    if (lab == 0) return;
    const float a = lab < n_labels ? table[lab] : 0.0f;
    const long long pv = padded_of(v, nx, ny, px, py);
    phi[pv] = a;
    if (phi2) phi2[pv] = a;
}

__global__ void k_affinity_map(const uint16_t* labels, long long V, int nx, int ny, int px, int py,
                               const float* map, float* phi, float* phi2) {
    const long long v = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (v >= V) return;
    if (labels[v] == 0) return;
    const long long pv = padded_of(v, nx, ny, px, py);
    phi[pv] = map[v];
    if (phi2) phi2[pv] = map[v];
}

// 1: inlet (the first `depth` z layers), 2: outlet (the last ones), 0: neither
__device__ __forceinline__ int slab_side(int pv, int pxpy, int nz, int depth) {
    const int z = pv / pxpy - 1;
    if (z < depth) return 1;
    if (z >= nz - depth) return 2;
    return 0;
}

__global__ void k_slab_flags(const int* site_vox, long long N, int pxpy, int nz, int depth, int* flags) {
    const long long n = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (n >= N) return;
    flags[n] = slab_side(site_vox[n], pxpy, nz, depth) != 0 ? 1 : 0;
}

__global__ void k_slab_scatter(const int* site_vox, long long N, int pxpy, int nz, int depth,
                               const int* flags, const int* scan, int* sites, signed char* side) {
    const long long n = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (n >= N || !flags[n]) return;
    const int e = scan[n];
    sites[e] = static_cast<int>(n);
    side[e] = static_cast<signed char>(slab_side(site_vox[n], pxpy, nz, depth));
}

__global__ void k_export_index(const int* site_vox, const int* vsite, long long N, int nx, int ny,
                               int px, int py, DomainView d, long long* site2vox, int* nbr) {
    const long long n = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (n >= N) return;
    const int pv = site_vox[n];
    if (site2vox) {
        const long long X = pv % px, r = pv / px, Y = r % py, Z = r / py;
        site2vox[n] = (X - 1) + static_cast<long long>(nx) * ((Y - 1) + static_cast<long long>(ny) * (Z - 1));
    }
    if (nbr) {
        for (int q = 1; q < Q19; ++q) nbr[static_cast<long long>(q - 1) * N + n] = vsite[pv + stencil_off(d, q)];
    }
}

// Which face links of each site bounce back: bit q - 1 for x + xi_q solid or
// wall (q = 1..6). Read by the fp16 collision to pick the site whose phase is
// the reference of each stored component value.
__global__ void k_wall_mask(const int* site_vox, const int* vsite, long long N, int px, int pxpy,
                            unsigned char* wall6) {
    const long long n = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (n >= N) return;
    const int pv = site_vox[n];
    unsigned m = 0;
    for (int q = 1; q < Q7; ++q)
        if (vsite[pv + stencil_offset(q, px, pxpy)] < 0) m |= 1u << (q - 1);
    wall6[n] = static_cast<unsigned char>(m);
}

}  // namespace

cudaError_t launch_flag_pore(const uint16_t* labels, long long V, int* flags, cudaStream_t s) {
    k_flag_pore<<<blocks_for(V), kBlock, 0, s>>>(labels, V, flags);
    return cudaGetLastError();
}

// Device-wide exclusive scan of n ints (n < 2^31), reduce-then-scan by tiles.
cudaError_t exclusive_scan(lbpm_ctx* c, const int* in, int* out, long long n) {
    if (n <= 0) return cudaSuccess;
    const long long tiles = (n + kTile - 1) / kTile;
    if (tiles == 1) {
        k_tile_scan<<<1, kScanThreads, 0, c->stream>>>(in, n, out, nullptr);
        return cudaGetLastError();
    }
    int* sums = static_cast<int*>(dalloc(c, sizeof(int) * tiles));
    int* offs = static_cast<int*>(dalloc(c, sizeof(int) * tiles));
    if (!sums || !offs) {
        dfree(c, sums);
        dfree(c, offs);
        return cudaErrorMemoryAllocation;
    }
    k_tile_sums<<<static_cast<unsigned>(tiles), kScanThreads, 0, c->stream>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan(c, sums, offs, tiles);
    if (e == cudaSuccess) {
        k_tile_scan<<<static_cast<unsigned>(tiles), kScanThreads, 0, c->stream>>>(in, n, out, offs);
        e = cudaGetLastError();
    }
    dfree(c, sums);
    dfree(c, offs);
    return e;
}

cudaError_t launch_scatter_sites(const lbpm_ctx* c, const int* scan, cudaStream_t s) {
    k_scatter_sites<<<blocks_for(c->V), kBlock, 0, s>>>(c->d_labels, scan, c->V, c->nx, c->ny, c->px,
                                                        c->py, c->d_site_vox, c->d_vsite, c->d_phi);
    return cudaGetLastError();
}

cudaError_t launch_fill_halo(const lbpm_ctx* c, cudaStream_t s) {
    k_fill_halo<<<blocks_for(c->Vp), kBlock, 0, s>>>(geo_of(c), c->d_vsite, c->d_phi, c->d_phi_alt);
    return cudaGetLastError();
}

cudaError_t launch_halo_flags(const lbpm_ctx* c, int* flags, cudaStream_t s) {
    k_halo_flags<<<blocks_for(c->Vp), kBlock, 0, s>>>(geo_of(c), c->d_vsite, flags);
    return cudaGetLastError();
}

cudaError_t launch_halo_scatter(const lbpm_ctx* c, const int* flags, const int* scan, cudaStream_t s) {
    k_halo_scatter<<<blocks_for(c->Vp), kBlock, 0, s>>>(c->Vp, flags, scan, c->d_vsite, c->d_halo_dst,
                                                       c->d_halo_site);
    return cudaGetLastError();
}

cudaError_t launch_affinity_table(const lbpm_ctx* c, const float* table, int n_labels, cudaStream_t s) {
    k_affinity_table<<<blocks_for(c->V), kBlock, 0, s>>>(c->d_labels, c->V, c->nx, c->ny, c->px, c->py,
                                                         table, n_labels, c->d_phi, c->d_phi_alt);
    return cudaGetLastError();
}

cudaError_t launch_affinity_map(const lbpm_ctx* c, const float* map, cudaStream_t s) {
    k_affinity_map<<<blocks_for(c->V), kBlock, 0, s>>>(c->d_labels, c->V, c->nx, c->ny, c->px, c->py,
                                                       map, c->d_phi, c->d_phi_alt);
    return cudaGetLastError();
}

// reservoir slabs are four layers deep; the pressure and flux boundaries act on the face layer
int slab_depth(const lbpm_ctx* c) { return c->params.reservoir_z >= 2 ? 1 : 4; }

cudaError_t launch_slab_flags(const lbpm_ctx* c, int* flags, cudaStream_t s) {
    k_slab_flags<<<blocks_for(c->N), kBlock, 0, s>>>(c->d_site_vox, c->N, c->px * c->py, c->nz, slab_depth(c),
                                                     flags);
    return cudaGetLastError();
}

cudaError_t launch_slab_scatter(const lbpm_ctx* c, const int* flags, const int* scan, cudaStream_t s) {
    k_slab_scatter<<<blocks_for(c->N), kBlock, 0, s>>>(c->d_site_vox, c->N, c->px * c->py, c->nz, slab_depth(c),
                                                       flags, scan, c->d_slab_site, c->d_slab_side);
    return cudaGetLastError();
}

cudaError_t launch_export_index(const lbpm_ctx* c, long long* site2vox, int* nbr, cudaStream_t s) {
    if (c->N == 0) return cudaSuccess;
    k_export_index<<<blocks_for(c->N), kBlock, 0, s>>>(c->d_site_vox, c->d_vsite, c->N, c->nx, c->ny,
                                                       c->px, c->py, make_view(c), site2vox, nbr);
    return cudaGetLastError();
}

cudaError_t launch_wall_mask(const lbpm_ctx* c, cudaStream_t s) {
    if (c->N == 0) return cudaSuccess;
    k_wall_mask<<<blocks_for(c->N), kBlock, 0, s>>>(c->d_site_vox, c->d_vsite, c->N, c->px,
                                                    c->px * c->py, c->d_wall6);
    return cudaGetLastError();
}

}  // namespace lbm
