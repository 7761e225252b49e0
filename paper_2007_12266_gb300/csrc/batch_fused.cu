// Batched form, fused: one persistent kernel runs every pass of a bundle of
// timesteps (phase pass, collision, reservoir reset; Sec. 3.1 and Sec. 4.1)
// for all jobs of a batch.
//
// The grid is cooperative (every block resident at once). Within a pass the
// blocks take tiles from an atomic counter, so the uneven jobs balance
// dynamically; between passes every block meets at a grid-wide barrier,
// because a phase pass needs the whole previous collision and a collision
// needs the whole phase pass (the colour gradient reads the neighbours'
// phase). The barrier's wait is bounded: a block that waits longer than the
// launch's limit sets the error flag and returns, and so does every other
// block that sees the flag, so a lost arrival ends the kernel with an error
// instead of a hang (the host reports it as LBPM_E_TIMEOUT).
//
// Memory ordering across a barrier: each block's writes are released by a
// gpu-scope fence of its thread 0 after the block barrier, and acquired after
// the wait by an acquire load and a gpu-scope fence, followed by the block
// barrier. Everything a pass reads that an earlier pass of the same launch
// wrote (populations, sums, phase grid, N, density references) is read with
// coherent loads; only the static index goes through the read-only path.
#include "step_kernels.cuh"
#include "batch.h"

namespace lbm {

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Grid-wide barrier over `expected` blocks (ctl[0]: arrivals, ctl[1]:
// generation), bounded by limit_ns. Returns false (and sets *err) if the wait
// gave up or another block already did.
__device__ bool grid_barrier(unsigned* ctl, int* err, unsigned expected, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(ctl + 1);   // read before arriving
        __threadfence();                                // release this block's writes
        if (atomicAdd(ctl, 1u) + 1u == expected) {
            ctl[0] = 0u;                                // nobody arrives again before the release
            st_release_u32(ctl + 1, gen + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(ctl + 1) == gen) {
                if (ld_volatile_int(err) || global_ns() - t0 > limit_ns) {
                    atomicOr(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        if (ld_volatile_int(err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// first tile of each job for a pass, and the job owning tile t (uniform search)
__device__ __forceinline__ int fused_job_of(const int* tile_begin, int n_jobs, int t) {
    int lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_begin[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One pass: blocks take tiles from the pass's counter until the jobs' tiles
// run out; op(job, index of the tile within the job). (Tiles taken per warp,
// without the block barriers, measured slower: 16 % in FP32.)
template <class Op>
__device__ __forceinline__ void fused_pass(const FusedLaunch& p, int pass, const int* tile_begin, Op&& op) {
    __shared__ int s_tile;
    const int nt = tile_begin[p.n_jobs];
    for (;;) {
        if (threadIdx.x == 0) s_tile = static_cast<int>(atomicAdd(p.ctl + 2 + pass, 1u));
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= nt) break;
        const int j = fused_job_of(tile_begin, p.n_jobs, t);
        op(j, t - tile_begin[j]);
    }
}

// Forms of each pass by kind of step (as in the graph path): the phase pass
// 0 = populations, 1 = sums, 2 = sums writing N; the collision's component
// form CF; the reservoir reset writing sums or populations.
template <int KIND>
struct FusedKind {
    static constexpr int kPhase = KIND == kFusedSumMid ? 1 : (KIND == kFusedSumLast ? 2 : 0);
    static constexpr int kCollide = KIND == kFusedSumFirst ? 1 : (KIND == kFusedSumMid ? 2 : 0);
    static constexpr bool kClearTargets = KIND == kFusedSumFirst;
    static constexpr bool kResetSums = KIND == kFusedSumFirst || KIND == kFusedSumMid;
};

// NS timesteps of the given kind, the first at parity PAR0.
template <class S, int BT, int KIND, int PAR0, int NS>
__global__ void __launch_bounds__(BT, 1152 / BT) k_batch_fused(const __grid_constant__ FusedLaunch p) {
    using K = FusedKind<KIND>;
    __shared__ int slot[(Q19 - 1) * BT];
    __shared__ float ref[S::kRef ? (Q19 - 1) * BT : 1];
    const unsigned nblocks = gridDim.x;
    int pass = 0;
    bool go = true;
    static_for<0, NS>([&](auto kc) {
        constexpr int PAR = PAR0 ^ (decltype(kc)::value & 1);
        if (!go) return;
        // phase pass (and, at the first step of a sum-form run, clearing the
        // sums the collision accumulates into)
        // (fused_phase_per(BT) independent entries per thread: the pass is
        // latency-bound, and the fused kernel runs fewer warps than the
        // separate phase kernel because it holds the collision's registers)
        fused_pass(p, pass++, p.tiles[0], [&](int j, int tj) {
            const DomainView& d = p.v[j];
            constexpr int PER = fused_phase_per(BT);
            const int i0 = tj * BT * PER + static_cast<int>(threadIdx.x);
            if constexpr (K::kPhase == 0) {
                #pragma unroll
                for (int k = 0; k < PER; ++k) phase_thread<PAR, S>(d, i0 + k * BT);
            } else {
                phase_sum_thread<PAR, K::kPhase == 2, PER>(d, i0, BT);
            }
            if constexpr (K::kClearTargets) {
                #pragma unroll
                for (int k = 0; k < PER; ++k)
                    if (i0 + k * BT < d.n_sites) d.acc[PAR ^ 1][i0 + k * BT] = 0ull;
            }
        });
        go = grid_barrier(p.ctl, p.err, nblocks, p.limit_ns);
        if (!go) return;
        fused_pass(p, pass++, p.tiles[1], [&](int j, int tj) {
            const DomainView& d = p.v[j];
            const int n = tj * BT + static_cast<int>(threadIdx.x);
            if (n < d.n_sites) collide_thread<PAR, S, K::kCollide>(d, n, SlotCache{slot + threadIdx.x, ref + threadIdx.x, BT});
        });
        if (p.tiles[2][p.n_jobs] > 0) {
            go = grid_barrier(p.ctl, p.err, nblocks, p.limit_ns);
            if (!go) return;
            fused_pass(p, pass++, p.tiles[2], [&](int j, int tj) {
                const FusedSlab& sl = p.slab[j];
                const int i = tj * BT + static_cast<int>(threadIdx.x);
                if (i < sl.n) reservoir_thread<PAR ^ 1, S, K::kResetSums>(p.v[j], sl.site[i], sl.side[i], sl.rho_in, sl.rho_out);
            });
        }
        if constexpr (decltype(kc)::value + 1 < NS) go = grid_barrier(p.ctl, p.err, nblocks, p.limit_ns);
    });
}

// A lone barrier for the self-test (lbpm_batch_check_barrier): `expected`
// arrivals, which may exceed the grid on purpose so that the wait runs out.
__global__ void k_barrier_probe(unsigned* ctl, int* err, unsigned expected, unsigned long long limit_ns) {
    grid_barrier(ctl, err, expected, limit_ns);
}

template <class S, int BT, int KIND, int PAR0, int NS>
cudaError_t go_fused(unsigned grid, cudaStream_t s, const FusedLaunch& p) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_fused<S, BT, KIND, PAR0, NS>, p);
}

template <class S, int BT>
const void* fused_fn(int kind) {
    switch (kind) {
    case kFusedSumFirst: return reinterpret_cast<const void*>(k_batch_fused<S, BT, kFusedSumFirst, 0, 1>);
    case kFusedSumMid: return reinterpret_cast<const void*>(k_batch_fused<S, BT, kFusedSumMid, 1, 2>);
    case kFusedSumLast: return reinterpret_cast<const void*>(k_batch_fused<S, BT, kFusedSumLast, 1, 1>);
    default: return reinterpret_cast<const void*>(k_batch_fused<S, BT, kFusedPop, 0, 2>);
    }
}

template <class S, int BT>
cudaError_t launch_fused_bt(int kind, unsigned grid, cudaStream_t s, const FusedLaunch& p) {
    switch (kind) {
    case kFusedSumFirst: return go_fused<S, BT, kFusedSumFirst, 0, 1>(grid, s, p);
    case kFusedSumMid: return go_fused<S, BT, kFusedSumMid, 1, 2>(grid, s, p);
    case kFusedSumLast: return go_fused<S, BT, kFusedSumLast, 1, 1>(grid, s, p);
    default: return go_fused<S, BT, kFusedPop, 0, 2>(grid, s, p);
    }
}

}  // namespace

static_assert(sizeof(FusedLaunch) <= 32000, "fused job table must fit the kernel parameter space");

cudaError_t launch_batch_fused(int kind, bool fp16, int bt, unsigned grid, cudaStream_t s, const FusedLaunch& p) {
    if (bt == 128)
        return fp16 ? launch_fused_bt<StoreF16, 128>(kind, grid, s, p) : launch_fused_bt<StoreF32, 128>(kind, grid, s, p);
    if (bt == 192)
        return fp16 ? launch_fused_bt<StoreF16, 192>(kind, grid, s, p) : launch_fused_bt<StoreF32, 192>(kind, grid, s, p);
    return fp16 ? launch_fused_bt<StoreF16, 256>(kind, grid, s, p) : launch_fused_bt<StoreF32, 256>(kind, grid, s, p);
}

int batch_fused_blocks_per_sm(int kind, bool fp16, int bt) {
    const void* f = bt == 128   ? (fp16 ? fused_fn<StoreF16, 128>(kind) : fused_fn<StoreF32, 128>(kind))
                    : bt == 192 ? (fp16 ? fused_fn<StoreF16, 192>(kind) : fused_fn<StoreF32, 192>(kind))
                                : (fp16 ? fused_fn<StoreF16, 256>(kind) : fused_fn<StoreF32, 256>(kind));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, bt == 128 || bt == 192 ? bt : 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_barrier_probe(unsigned grid, unsigned expected, unsigned long long limit_ns, unsigned* ctl, int* err,
                                 cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_barrier_probe, ctl, err, expected, limit_ns);
}

}  // namespace lbm
