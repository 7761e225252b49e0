// Batched form: many independent domains (jobs) advanced together.
//
// Each job keeps its own context and device arrays. A batch builds a table of
// the jobs' views and of the first tile of each job (passed by value in the
// kernel's parameter space), and advances every job with ONE launch per pass:
// the phase kernel, then the fused collide-stream kernel, over the tiles of
// all jobs, either one block per tile (the default) or a persistent grid whose
// blocks walk the tile list round-robin. Step bundles are captured into a CUDA
// graph. Bundles hold an even number of steps, so every job is at an even
// step at a bundle boundary and the AA parity of each launch is a
// compile-time constant for the whole batch. (The alternative of one
// cooperative kernel for every pass of a bundle is in batch_fused.cu.)
//
// The launch shape (threads per block, resident blocks per SM or one block
// per tile, or the fused kernel) is picked by a small autotuner that times
// candidates on real steps (every candidate computes identical results, so
// tuning advances the simulation normally) and caches the winner per GPU,
// precision and size class.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "batch.h"
#include "measure_kernels.cuh"

namespace lbm {


namespace {

constexpr int kMaxBlocksPerSm = 16;

// Blocks take tiles blockIdx.x, + gridDim.x, ... (one tile per block when the
// grid covers them all), so the tiles in flight at any moment are neighbours
// in the numbering and their phi stencils and neighbour ids share L2 lines.
static_assert(sizeof(BatchLaunch) <= 32000, "job table must fit the kernel parameter space");

// job owning tile t: the last j with tile_begin[j] <= t (uniform search)
__device__ __forceinline__ int job_of_tile(const BatchLaunch& p, int t) {
    int lo = 0, hi = p.n_jobs;   // tile_begin[lo] <= t < tile_begin[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p.tile_begin[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int PAR, class S, int BT>
__global__ void __launch_bounds__(BT) k_batch_phase(const __grid_constant__ BatchLaunch p) {
    const int nt = p.tile_begin[p.n_jobs];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int j = job_of_tile(p, t);
        const int i0 = (t - p.tile_begin[j]) * BT * kBatchPhasePer + static_cast<int>(threadIdx.x);
#pragma unroll
        for (int k = 0; k < kBatchPhasePer; ++k) phase_thread<PAR, S>(p.v[j], i0 + k * BT);
    }
}

// Phase pass of the sum form (see phase_sum_thread), kBatchPhasePer entries
// per thread.
template <int PAR, bool WRITE_N, int BT>
__global__ void __launch_bounds__(BT) k_batch_phase_sum(const __grid_constant__ BatchLaunch p) {
    const int nt = p.tile_begin[p.n_jobs];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int j = job_of_tile(p, t);
        phase_sum_thread<PAR, WRITE_N, kBatchPhasePer>(
            p.v[j], (t - p.tile_begin[j]) * BT * kBatchPhasePer + static_cast<int>(threadIdx.x), BT);
    }
}

// CF: component form of the collision (see collide_site).
// 36 resident warps per SM where the block size allows (56 registers at 128
// threads), as for the single-domain collision.
template <int PAR, class S, int CF, int BT>
__global__ void __launch_bounds__(BT, 1152 / BT) k_batch_collide(const __grid_constant__ BatchLaunch p) {
    constexpr int kSlots = PAR == 1 ? (Q19 - 1) * BT : (CF != 0 ? (Q7 - 1) * BT : 1);
    constexpr int kRefs = PAR == 1 && S::kRef ? (Q19 - 1) * BT : 1;
    __shared__ int slot[kSlots];
    __shared__ float ref[kRefs];
    const int nt = p.tile_begin[p.n_jobs];
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int j = job_of_tile(p, t);
        const DomainView& d = p.v[j];
        const int n = (t - p.tile_begin[j]) * BT + threadIdx.x;
        if (n < d.n_sites) collide_thread<PAR, S, CF>(d, n, SlotCache{slot + threadIdx.x, ref + threadIdx.x, BT});
    }
}

template <int BT>
struct Launch {
    template <class K>
    static cudaError_t go(K kernel, unsigned grid, cudaStream_t s, const BatchLaunch& p) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(BT);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, p);
    }
};

// phase pass: form 0 = populations, 1 = sums, 2 = sums writing N (last step of a run)
template <int BT, int PAR>
cudaError_t batch_phase_par(int form, bool fp16, unsigned grid, cudaStream_t s, const BatchLaunch& p) {
    if (form == 1) return Launch<BT>::go(k_batch_phase_sum<PAR, false, BT>, grid, s, p);
    if (form == 2) return Launch<BT>::go(k_batch_phase_sum<PAR, true, BT>, grid, s, p);
    return fp16 ? Launch<BT>::go(k_batch_phase<PAR, StoreF16, BT>, grid, s, p)
                : Launch<BT>::go(k_batch_phase<PAR, StoreF32, BT>, grid, s, p);
}

// collision: form = component form CF (0 populations, 1 / 2 sums)
template <int BT, int PAR, int CF>
cudaError_t batch_collide_cf(bool fp16, unsigned grid, cudaStream_t s, const BatchLaunch& p) {
    return fp16 ? Launch<BT>::go(k_batch_collide<PAR, StoreF16, CF, BT>, grid, s, p)
                : Launch<BT>::go(k_batch_collide<PAR, StoreF32, CF, BT>, grid, s, p);
}
template <int BT, int PAR>
cudaError_t batch_collide_par(int form, bool fp16, unsigned grid, cudaStream_t s, const BatchLaunch& p) {
    if (form == 1) return batch_collide_cf<BT, PAR, 1>(fp16, grid, s, p);
    if (form == 2) return batch_collide_cf<BT, PAR, 2>(fp16, grid, s, p);
    return batch_collide_cf<BT, PAR, 0>(fp16, grid, s, p);
}

template <int BT>
cudaError_t batch_bt(int kernel, int form, int par, bool fp16, unsigned grid, cudaStream_t s, const BatchLaunch& p) {
    if (kernel == 0)
        return par == 0 ? batch_phase_par<BT, 0>(form, fp16, grid, s, p) : batch_phase_par<BT, 1>(form, fp16, grid, s, p);
    return par == 0 ? batch_collide_par<BT, 0>(form, fp16, grid, s, p) : batch_collide_par<BT, 1>(form, fp16, grid, s, p);
}

}  // namespace

// Launch one phase (0 = phase pass, 1 = collide-stream) over the jobs of p,
// in the given form (see batch_phase_par / batch_collide_par).
cudaError_t launch_batch(int kernel, int form, int par, bool fp16, int bt, unsigned grid, cudaStream_t s,
                         const BatchLaunch& p) {
    if (p.n_jobs == 0 || p.tile_begin[p.n_jobs] == 0) return cudaSuccess;
    switch (bt) {
    case 128: return batch_bt<128>(kernel, form, par, fp16, grid, s, p);
    case 192: return batch_bt<192>(kernel, form, par, fp16, grid, s, p);
    case 512: return batch_bt<512>(kernel, form, par, fp16, grid, s, p);
    default: return batch_bt<256>(kernel, form, par, fp16, grid, s, p);
    }
}

namespace {

static_assert(sizeof(DomainView) % sizeof(int) == 0, "view copied as ints");

// Per-tile fp64 partial sums of the measures (kBatchMeasureTile sites per
// tile, kBatchMeasureTile / BT per thread, strided by BT so that loads
// coalesce); each job's parity is read per tile.
template <class S, int BT>
__global__ void __launch_bounds__(BT) k_batch_measure(const DomainView* views, const int* parity,
                                                      const BatchTile* tiles, int n_tiles, double* partials) {
    __shared__ DomainView sv;
    __shared__ int par;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x < static_cast<int>(sizeof(DomainView) / sizeof(int)))
            reinterpret_cast<int*>(&sv)[threadIdx.x] = reinterpret_cast<const int*>(views + tl.job)[threadIdx.x];
        if (threadIdx.x == 0) par = parity[tl.job];
        __syncthreads();
        AccF64 acc[NSUM];
        for (int k = 0; k < kBatchMeasureTile / BT; ++k) {
            const int n = tl.first + k * BT + static_cast<int>(threadIdx.x);
            if (n >= sv.n_sites) break;
            if (par) measure_site<1, S>(sv, n, acc);
            else measure_site<0, S>(sv, n, acc);
        }
        block_reduce_sums<BT>(acc, partials + static_cast<size_t>(t) * NSUM);
    }
}

// One block per job, one warp per quantity: fixed-order sum of the job's tiles.
__global__ void k_batch_job_reduce(const double* partials, const int* tile_begin, int n_jobs, double* out) {
    const int j = blockIdx.x;
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= n_jobs || i >= NSUM) return;
    double s = 0.0;
    for (int t = tile_begin[j] + lane; t < tile_begin[j + 1]; t += 32) s += partials[static_cast<size_t>(t) * NSUM + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[static_cast<size_t>(j) * NSUM + i] = s;
}

}  // namespace

cudaError_t launch_batch_measure(bool fp16, unsigned grid, cudaStream_t s, const DomainView* v, const int* parity,
                                 const BatchTile* t, int nt, double* partials, const int* tile_begin, int n_jobs,
                                 double* out) {
    if (nt > 0) {
        if (fp16) k_batch_measure<StoreF16, 256><<<grid, 256, 0, s>>>(v, parity, t, nt, partials);
        else k_batch_measure<StoreF32, 256><<<grid, 256, 0, s>>>(v, parity, t, nt, partials);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_jobs > 0) k_batch_job_reduce<<<n_jobs, 32 * NSUM, 0, s>>>(partials, tile_begin, n_jobs, out);
    return cudaGetLastError();
}

// Resident blocks per SM of a batch kernel at a block size (occupancy limit).
int batch_max_blocks(int kernel, bool fp16, int bt) {
    int nb = 0;
    const void* f = nullptr;
#define LBPM_PICK(BT)                                                                                        \
    f = kernel == 0 ? (fp16 ? (const void*)k_batch_phase<1, StoreF16, BT> : (const void*)k_batch_phase<1, StoreF32, BT>) \
                    : (fp16 ? (const void*)k_batch_collide<1, StoreF16, 2, BT>                                \
                            : (const void*)k_batch_collide<1, StoreF32, 2, BT>);
    if (bt == 128) { LBPM_PICK(128) } else if (bt == 192) { LBPM_PICK(192) } else if (bt == 512) { LBPM_PICK(512) } else { LBPM_PICK(256) }
#undef LBPM_PICK
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, bt, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, std::min(nb, kMaxBlocksPerSm));
}

}  // namespace lbm
