// Batched form: declarations shared by batch.cu, batch_fused.cu and
// batch_api.cu, apart from the step kernels' shared header (internal.h),
// which they only use.
#pragma once
#include "internal.h"

namespace lbm {

// Sites of one tile of the batched basic analysis: 32 per thread of a
// 256-thread block, each thread summing its sites in compensated fp32 before
// the block's one fp64 reduction (as the single-domain analysis does; within
// the accumulator's 64-site bound).
constexpr int kBatchMeasureTile = 256 * 32;

// Entries per thread of the batched phase pass (a phase tile holds this many
// times the threads of a block; two independent round trips in flight per
// thread, as in the single-domain pass; 2 is 2 % faster than 1 on the 64-job
// set, 4 the same as 2).
constexpr int kBatchPhasePer = 2;

// Fused batched form (batch_fused.cu): one cooperative persistent launch per
// bundle runs the phase pass, the collision and the reservoir reset of every
// job, with bounded grid barriers between the passes.

constexpr int kFusedJobs = 112;   // jobs per fused launch (the table lives in the parameter space)
enum FusedStepKind { kFusedPop = 0, kFusedSumFirst = 1, kFusedSumMid = 2, kFusedSumLast = 3 };
constexpr int kFusedCtl = 2 + 6;  // barrier arrivals and generation, then one tile counter per pass
// phase entries per thread in the fused kernel (a phase tile is that many x
// threads): 8 at 256 threads (64 registers; 16 spill), 4 at 128 and 192 (56
// registers; 8 spill)
constexpr int fused_phase_per(int bt) { return bt >= 256 ? 8 : 4; }
struct FusedSlab {
    const int* site;
    const signed char* side;
    int n;
    float rho_in, rho_out;
};
struct FusedLaunch {
    int n_jobs;
    int tiles[3][kFusedJobs + 1];    // first tile of each job: phase entries, sites, slab sites
    unsigned long long limit_ns;     // bound of a barrier wait
    unsigned* ctl;                   // [kFusedCtl] zeroed before each launch
    int* err;                        // set when a barrier wait gave up
    DomainView v[kFusedJobs];
    FusedSlab slab[kFusedJobs];
};
// kind: FusedStepKind (pop: two steps from an even one; sum first: one step
// from an even one; sum middle: two steps from an odd one; sum last: one step
// at an odd one); bt = 128, 192 or 256 threads per block.
cudaError_t launch_batch_fused(int kind, bool fp16, int bt, unsigned grid, cudaStream_t s, const FusedLaunch& p);
int batch_fused_blocks_per_sm(int kind, bool fp16, int bt);
// One lone barrier of `grid` blocks waiting for `expected` arrivals (self-test).
cudaError_t launch_barrier_probe(unsigned grid, unsigned expected, unsigned long long limit_ns, unsigned* ctl, int* err,
                                 cudaStream_t s);

}  // namespace lbm
