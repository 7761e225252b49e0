// C ABI of the batched form (declared in include/lbpm.h): a batch of job
// contexts advanced together by the batch kernels (batch.cu: one launch per
// pass) or the fused kernel (batch_fused.cu: one launch per bundle).
#include <algorithm>
#include <new>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "batch.h"

using namespace lbm;

struct lbpm_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    lbpm_alloc_fn alloc = nullptr;
    lbpm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::vector<lbpm_ctx*> jobs;
    int precision = -1;
    // device tables
    DomainView* d_views = nullptr;
    int* d_parity = nullptr;
    std::vector<BatchLaunch> launch[2];          // phase, collide job tables (tile = kBatchPhasePer x bt, bt entries)
    BatchTile* d_mtiles = nullptr;               // measure tiles (kBatchMeasureTile sites)
    int* d_mbegin = nullptr;                     // [J+1] first measure tile of each job
    double* d_partials = nullptr;
    double* d_out = nullptr;
    size_t cap_views = 0, cap_mtiles = 0;
    int n_mtiles = 0;
    bool dirty = true;
    // launch shape
    // resident blocks per SM of the persistent grids (0 = occupancy limit, -1 =
    // one block per tile). The default is the fastest shape measured on GB300
    // for mixed job sizes in both storages: one block per tile (the hardware
    // block scheduler balances uneven tiles better than a static round-robin
    // over persistent blocks) of 192 threads (six blocks, 36 warps per SM at 56
    // registers for the collision).
    int bt = 192;
    int bps[2] = {-1, -1};
    int n_sm = 0;
    // bundle graphs (2 timesteps): graph = population form; sum_graph = two
    // middle steps of the sum form starting at an odd step (see batch_advance_sum)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t sum_graph = nullptr;
    long long launches = 0;
    // fused persistent form (blocks per SM -2 for both passes, see batch_fused.cu):
    // the job table, the barrier and tile-counter words, the error flag, and the
    // graph of two steps (two middle steps in the sum form)
    bool fused_ready = false;
    FusedLaunch* fused = nullptr;
    unsigned* d_ctl = nullptr;
    int* d_err = nullptr;
    cudaGraphExec_t fused_graph = nullptr;
};

namespace {

lbpm_status bfail(lbpm_batch* b, lbpm_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}

lbpm_status bfail_cuda(lbpm_batch* b, const char* what, cudaError_t e) {
    return bfail(b, e == cudaErrorMemoryAllocation ? LBPM_E_OOM : LBPM_E_CUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define LBPM_BCK(b, call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bfail_cuda(b, #call, e_);    \
    } while (0)

void* balloc(lbpm_batch* b, size_t bytes) {
    void* p = nullptr;
    if (b->alloc) return b->alloc(bytes ? bytes : 16, b->stream, b->alloc_user);
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void bfree(lbpm_batch* b, void* p) {
    if (!p) return;
    if (b->free_fn) b->free_fn(p, b->alloc_user);
    else cudaFree(p);
}

template <class T>
bool ensure(lbpm_batch* b, T** p, size_t* cap, size_t n) {
    if (*p && *cap >= n) return true;
    bfree(b, *p);
    const size_t c = std::max<size_t>(n, 16) * 3 / 2;
    *p = static_cast<T*>(balloc(b, sizeof(T) * c));
    *cap = *p ? c : 0;
    return *p != nullptr;
}

void drop_graph(lbpm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->sum_graph) cudaGraphExecDestroy(b->sum_graph);
    b->sum_graph = nullptr;
    if (b->fused_graph) cudaGraphExecDestroy(b->fused_graph);
    b->fused_graph = nullptr;
}

lbpm_status enter(lbpm_batch* b) {
    if (!b) return LBPM_E_INVALID;
    b->err.clear();
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail_cuda(b, "cudaSetDevice", e);
    return LBPM_OK;
}

// (Re)build the device job table and tile lists.
lbpm_status rebuild(lbpm_batch* b) {
    drop_graph(b);
    const int J = static_cast<int>(b->jobs.size());
    std::vector<DomainView> views(J);
    std::vector<int> parity(J);
    std::vector<BatchTile> mtiles;
    std::vector<int> mbegin(J + 1, 0);
    for (int k = 0; k < 2; ++k) b->launch[k].clear();
    for (int j = 0; j < J; ++j) {
        const lbpm_ctx* c = b->jobs[j];
        views[j] = make_view(c);
        parity[j] = static_cast<int>(c->step & 1);
        const long long counts[2] = {c->N + c->H, c->N};
        for (int k = 0; k < 2; ++k) {
            if (j % kBatchLaunchJobs == 0) {
                b->launch[k].emplace_back();
                std::memset(&b->launch[k].back(), 0, sizeof(BatchLaunch));
            }
            BatchLaunch& L = b->launch[k].back();
            const long long per_tile = k == 0 ? static_cast<long long>(b->bt) * kBatchPhasePer : b->bt;
            const long long tiles = (counts[k] + per_tile - 1) / per_tile;
            if (L.tile_begin[L.n_jobs] + tiles > (1LL << 30))
                return bfail(b, LBPM_E_INVALID, "batch too large for one launch table");
            L.v[L.n_jobs] = views[j];
            L.tile_begin[L.n_jobs + 1] = L.tile_begin[L.n_jobs] + static_cast<int>(tiles);
            ++L.n_jobs;
        }
        mbegin[j] = static_cast<int>(mtiles.size());
        for (long long f = 0; f < c->N; f += kBatchMeasureTile) mtiles.push_back(BatchTile{j, static_cast<int>(f)});
    }
    mbegin[J] = static_cast<int>(mtiles.size());
    if (!ensure(b, &b->d_views, &b->cap_views, J)) return bfail(b, LBPM_E_OOM, "batch table allocation failed");
    // parity, measure-begin, partials and outputs are re-allocated to fit
    bfree(b, b->d_parity);
    bfree(b, b->d_mbegin);
    bfree(b, b->d_partials);
    bfree(b, b->d_out);
    b->d_parity = static_cast<int*>(balloc(b, sizeof(int) * std::max(J, 1)));
    b->d_mbegin = static_cast<int*>(balloc(b, sizeof(int) * (J + 1)));
    b->d_partials = static_cast<double*>(balloc(b, sizeof(double) * NSUM * std::max<size_t>(mtiles.size(), 1)));
    b->d_out = static_cast<double*>(balloc(b, sizeof(double) * NSUM * std::max(J, 1)));
    if (!b->d_parity || !b->d_mbegin || !b->d_partials || !b->d_out)
        return bfail(b, LBPM_E_OOM, "batch table allocation failed");
    if (!ensure(b, &b->d_mtiles, &b->cap_mtiles, mtiles.size()))
        return bfail(b, LBPM_E_OOM, "batch tile allocation failed");
    if (J) {
        LBPM_BCK(b, cudaMemcpyAsync(b->d_views, views.data(), sizeof(DomainView) * J, cudaMemcpyHostToDevice, b->stream));
        LBPM_BCK(b, cudaMemcpyAsync(b->d_parity, parity.data(), sizeof(int) * J, cudaMemcpyHostToDevice, b->stream));
    }
    LBPM_BCK(b, cudaMemcpyAsync(b->d_mbegin, mbegin.data(), sizeof(int) * (J + 1), cudaMemcpyHostToDevice, b->stream));
    b->n_mtiles = static_cast<int>(mtiles.size());
    if (b->n_mtiles)
        LBPM_BCK(b, cudaMemcpyAsync(b->d_mtiles, mtiles.data(), sizeof(BatchTile) * mtiles.size(),
                                    cudaMemcpyHostToDevice, b->stream));
    // fused table: up to kFusedJobs jobs, no pressure or flux faces
    b->fused_ready = false;
    bool fusable = J > 0 && J <= kFusedJobs && b->bt != 512;
    for (const lbpm_ctx* c : b->jobs) fusable = fusable && c->params.reservoir_z <= 1;
    if (fusable) {
        if (!b->fused) b->fused = new (std::nothrow) FusedLaunch;
        if (!b->d_ctl) b->d_ctl = static_cast<unsigned*>(balloc(b, sizeof(unsigned) * kFusedCtl));
        if (!b->d_err) {
            b->d_err = static_cast<int*>(balloc(b, sizeof(int)));
            if (b->d_err) LBPM_BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
        }
        if (!b->fused || !b->d_ctl || !b->d_err) return bfail(b, LBPM_E_OOM, "fused batch table allocation failed");
        FusedLaunch& F = *b->fused;
        std::memset(&F, 0, sizeof(FusedLaunch));
        F.n_jobs = J;
        F.limit_ns = 2000000000ull;   // 2 s: far above any pass of a batch that fits the GPU
        F.ctl = b->d_ctl;
        F.err = b->d_err;
        for (int j = 0; j < J; ++j) {
            const lbpm_ctx* c = b->jobs[j];
            const long long n_slab = c->params.reservoir_z == 1 ? c->n_slab : 0;
            const long long counts[3] = {c->N + c->H, c->N, n_slab};
            const long long per_tile[3] = {static_cast<long long>(b->bt) * fused_phase_per(b->bt), b->bt, b->bt};
            for (int k = 0; k < 3; ++k)
                F.tiles[k][j + 1] = F.tiles[k][j] + static_cast<int>((counts[k] + per_tile[k] - 1) / per_tile[k]);
            F.v[j] = views[j];
            F.slab[j] = FusedSlab{c->d_slab_site, c->d_slab_side, static_cast<int>(n_slab),
                                  static_cast<float>(c->params.rho_in), static_cast<float>(c->params.rho_out)};
        }
        b->fused_ready = true;
    }
    LBPM_BCK(b, cudaStreamSynchronize(b->stream));
    b->dirty = false;
    return LBPM_OK;
}

unsigned grid_for(const lbpm_batch* b, int k, const BatchLaunch& L) {
    const int n_tiles = L.tile_begin[L.n_jobs];
    if (b->bps[k] < 0) return static_cast<unsigned>(std::max(1, n_tiles));   // one block per tile
    const int occ = batch_max_blocks(k, b->precision == LBPM_FP16, b->bt);
    const int bps = b->bps[k] > 0 ? std::min(b->bps[k], occ) : occ;
    const long long persistent = static_cast<long long>(bps) * b->n_sm;
    return static_cast<unsigned>(std::max<long long>(1, std::min<long long>(persistent, n_tiles)));
}

// Kinds of batched timestep, as in lbpm_advance: the population form, and the
// first, middle and last step of a run of the sum form.
enum BatchStep { kBPop = 0, kBSumFirst = 1, kBSumMid = 2, kBSumLast = 3 };

cudaError_t enqueue_step(lbpm_batch* b, int kind, int par, cudaStream_t s) {
    const bool h = b->precision == LBPM_FP16;
    // kernel forms (see launch_batch) of each kind: phase pass, collision
    const int phase_form[4] = {0, 0, 1, 2};
    const int collide_form[4] = {0, 1, 2, 0};
    cudaError_t e = cudaSuccess;
    if (kind == kBSumFirst)
        for (lbpm_ctx* c : b->jobs)
            if (e == cudaSuccess) e = clear_sums(c, par ^ 1, s);
    for (size_t i = 0; i < b->launch[0].size() && e == cudaSuccess; ++i) {
        e = launch_batch(0, phase_form[kind], par, h, b->bt, grid_for(b, 0, b->launch[0][i]), s, b->launch[0][i]);
        if (e == cudaSuccess)
            e = launch_batch(1, collide_form[kind], par, h, b->bt, grid_for(b, 1, b->launch[1][i]), s,
                             b->launch[1][i]);
    }
    const bool sums_next = kind == kBSumFirst || kind == kBSumMid;
    for (lbpm_ctx* c : b->jobs)
        if (e == cudaSuccess && c->n_slab)
            e = sums_next ? launch_reservoir_sum(c, par ^ 1, s) : launch_reservoir(c, par ^ 1, s);
    return e;
}

// Capture two timesteps of the given kind starting at parity `par0` into *out.
lbpm_status capture(lbpm_batch* b, int kind, int par0, cudaGraphExec_t* out) {
    if (*out) cudaGraphExecDestroy(*out);
    *out = nullptr;
    if (!b->cap_stream) LBPM_BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    LBPM_BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t el = enqueue_step(b, kind, par0, b->cap_stream);
    if (el == cudaSuccess) el = enqueue_step(b, kind, par0 ^ 1, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail_cuda(b, "batch graph capture", e);
    return LBPM_OK;
}

// Whether every job of the batch can run the sum form.
bool batch_sum_form(const lbpm_batch* b) {
    for (const lbpm_ctx* c : b->jobs)
        if (!sum_form_capable(c)) return false;
    return true;
}

// Whether the batch runs the fused persistent kernel (chosen with blocks per
// SM -2, and possible for this batch).
bool use_fused(const lbpm_batch* b) { return b->bps[0] == -2 && b->bps[1] == -2 && b->fused_ready; }

// One fused launch: clear its barrier and tile counters, then the cooperative
// grid of as many blocks as fit the GPU at once.
cudaError_t fused_launch(lbpm_batch* b, int kind, cudaStream_t s) {
    const bool h = b->precision == LBPM_FP16;
    const int per_sm = batch_fused_blocks_per_sm(kind, h, b->bt);
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaError_t e = cudaMemsetAsync(b->d_ctl, 0, sizeof(unsigned) * kFusedCtl, s);
    if (e == cudaSuccess) e = launch_batch_fused(kind, h, b->bt, static_cast<unsigned>(per_sm * b->n_sm), s, *b->fused);
    return e;
}

lbpm_status capture_fused(lbpm_batch* b, int kind, cudaGraphExec_t* out) {
    if (*out) cudaGraphExecDestroy(*out);
    *out = nullptr;
    if (!b->cap_stream) LBPM_BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    LBPM_BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t el = fused_launch(b, kind, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail_cuda(b, "fused batch graph capture", e);
    return LBPM_OK;
}

// lbpm_batch_advance with the fused kernel: in the sum form one launch for the
// first step, a graph of two middle steps replayed, one launch for the last
// step; in the population form a graph of two steps replayed.
lbpm_status batch_advance_fused(lbpm_batch* b, long long nsteps) {
    if (batch_sum_form(b)) {
        LBPM_BCK(b, fused_launch(b, kFusedSumFirst, b->stream));
        if (nsteps > 2) {
            if (!b->fused_graph) {
                lbpm_status s = capture_fused(b, kFusedSumMid, &b->fused_graph);
                if (s) return s;
            }
            for (long long k = 2; k < nsteps; k += 2) LBPM_BCK(b, cudaGraphLaunch(b->fused_graph, b->stream));
        }
        LBPM_BCK(b, fused_launch(b, kFusedSumLast, b->stream));
        b->launches += 2 + (nsteps - 2) / 2;
    } else {
        if (!b->fused_graph) {
            lbpm_status s = capture_fused(b, kFusedPop, &b->fused_graph);
            if (s) return s;
        }
        for (long long k = 0; k < nsteps; k += 2) LBPM_BCK(b, cudaGraphLaunch(b->fused_graph, b->stream));
        b->launches += nsteps / 2;
    }
    for (lbpm_ctx* c : b->jobs) c->step += nsteps;
    return LBPM_OK;
}

int kernels_per_bundle(const lbpm_batch* b) {
    int k = 4 * static_cast<int>(b->launch[0].size());
    for (const lbpm_ctx* c : b->jobs) k += c->n_slab ? 2 : 0;
    return k;
}

// lbpm_batch_advance in the sum form (nsteps even, >= 2): the first step
// reads the populations, nsteps - 2 middle steps (pairs starting at an odd
// step, replayed from a graph) carry the components as sums, the last step
// writes the populations.
lbpm_status batch_advance_sum(lbpm_batch* b, long long nsteps) {
    LBPM_BCK(b, enqueue_step(b, kBSumFirst, 0, b->stream));
    if (nsteps > 2) {
        if (!b->sum_graph) {
            lbpm_status s = capture(b, kBSumMid, 1, &b->sum_graph);
            if (s) return s;
        }
        for (long long k = 2; k < nsteps; k += 2) LBPM_BCK(b, cudaGraphLaunch(b->sum_graph, b->stream));
    }
    LBPM_BCK(b, enqueue_step(b, kBSumLast, 1, b->stream));
    b->launches += (nsteps / 2) * kernels_per_bundle(b);
    for (lbpm_ctx* c : b->jobs) c->step += nsteps;
    return LBPM_OK;
}

// launch-shape cache: (gpu, precision, log2 of the site count) -> (bt, bps0, bps1)
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune_cache;

std::string tune_key(const lbpm_batch* b) {
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, b->device);
    long long n = 0;
    for (const lbpm_ctx* c : b->jobs) n += c->N;
    int lg = 0;
    while ((1LL << (lg + 1)) <= n) ++lg;
    return std::string(p.name) + "/" + std::to_string(b->precision) + "/" + std::to_string(lg);
}

}  // namespace

extern "C" {

lbpm_status lbpm_batch_create(lbpm_batch** out, int device, void* cuda_stream) {
    if (!out) return LBPM_E_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return LBPM_E_INVALID;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LBPM_E_CUDA;
    lbpm_batch* b = new (std::nothrow) lbpm_batch();
    if (!b) return LBPM_E_OOM;
    b->device = device;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, device);
    *out = b;
    return LBPM_OK;
}

lbpm_status lbpm_batch_destroy(lbpm_batch* b) {
    if (!b) return LBPM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    bfree(b, b->d_views);
    bfree(b, b->d_parity);
    bfree(b, b->d_mtiles);
    bfree(b, b->d_mbegin);
    bfree(b, b->d_partials);
    bfree(b, b->d_out);
    bfree(b, b->d_ctl);
    bfree(b, b->d_err);
    delete b->fused;
    delete b;
    return LBPM_OK;
}

lbpm_status lbpm_batch_set_allocator(lbpm_batch* b, lbpm_alloc_fn alloc, lbpm_free_fn free_fn, void* user) {
    if (!b) return LBPM_E_INVALID;
    if (b->d_views) return bfail(b, LBPM_E_STATE, "set the allocator before adding jobs");
    if (alloc && !free_fn) return bfail(b, LBPM_E_INVALID, "an allocator needs a free function");
    b->alloc = alloc;
    b->free_fn = alloc ? free_fn : nullptr;
    b->alloc_user = user;
    return LBPM_OK;
}

const char* lbpm_batch_last_error(const lbpm_batch* b) { return b ? b->err.c_str() : ""; }

lbpm_status lbpm_batch_add(lbpm_batch* b, lbpm_ctx* job) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (!job) return bfail(b, LBPM_E_INVALID, "job is NULL");
    if (job->device != b->device) return bfail(b, LBPM_E_INVALID, "job lives on another device");
    if (!job->have_fluids) return bfail(b, LBPM_E_STATE, "initialise the job's fluids first");
    if (job->step & 1) return bfail(b, LBPM_E_STATE, "a job joins a batch at an even step");
    if (std::find(b->jobs.begin(), b->jobs.end(), job) != b->jobs.end())
        return bfail(b, LBPM_E_INVALID, "job is already in the batch");
    if (b->precision >= 0 && job->params.precision != b->precision)
        return bfail(b, LBPM_E_INVALID, "all jobs of a batch share the storage precision");
    if (job->N + job->H >= (1LL << 31)) return bfail(b, LBPM_E_INVALID, "job too large");
    // the job's pending work (on its own stream) must be done before the batch uses it
    if (cudaStreamSynchronize(job->stream) != cudaSuccess) return bfail(b, LBPM_E_CUDA, "job stream failed");
    b->precision = job->params.precision;
    b->jobs.push_back(job);
    b->dirty = true;
    return LBPM_OK;
}

lbpm_status lbpm_batch_remove(lbpm_batch* b, lbpm_ctx* job) {
    lbpm_status s = enter(b);
    if (s) return s;
    auto it = std::find(b->jobs.begin(), b->jobs.end(), job);
    if (it == b->jobs.end()) return bfail(b, LBPM_E_INVALID, "job is not in the batch");
    LBPM_BCK(b, cudaStreamSynchronize(b->stream));
    b->jobs.erase(it);
    if (b->jobs.empty()) b->precision = -1;
    b->dirty = true;
    return LBPM_OK;
}

lbpm_status lbpm_batch_refresh(lbpm_batch* b) {
    lbpm_status s = enter(b);
    if (s) return s;
    LBPM_BCK(b, cudaStreamSynchronize(b->stream));
    b->dirty = true;
    return LBPM_OK;
}

lbpm_status lbpm_batch_size(const lbpm_batch* b, int* n_jobs, long long* n_sites) {
    if (!b) return LBPM_E_INVALID;
    if (n_jobs) *n_jobs = static_cast<int>(b->jobs.size());
    if (n_sites) {
        long long n = 0;
        for (const lbpm_ctx* c : b->jobs) n += c->N;
        *n_sites = n;
    }
    return LBPM_OK;
}

lbpm_status lbpm_batch_advance(lbpm_batch* b, long long nsteps) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (nsteps < 0 || (nsteps & 1)) return bfail(b, LBPM_E_INVALID, "nsteps must be even and >= 0");
    for (lbpm_ctx* c : b->jobs) {
        if (c->unstable) return bfail(b, LBPM_E_UNSTABLE, "a job was flagged unstable");
        if (c->step & 1) return bfail(b, LBPM_E_STATE, "a job was advanced to an odd step outside the batch");
    }
    if (b->jobs.empty() || nsteps == 0) return LBPM_OK;
    if (b->dirty && (s = rebuild(b))) return s;
    if (use_fused(b)) return batch_advance_fused(b, nsteps);
    if (batch_sum_form(b)) return batch_advance_sum(b, nsteps);
    if (!b->graph && (s = capture(b, kBPop, 0, &b->graph))) return s;
    for (long long k = 0; k < nsteps; k += 2) LBPM_BCK(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches += (nsteps / 2) * kernels_per_bundle(b);
    for (lbpm_ctx* c : b->jobs) c->step += nsteps;
    return LBPM_OK;
}

lbpm_status lbpm_batch_measure(lbpm_batch* b, lbpm_measures* out) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (!out) return bfail(b, LBPM_E_INVALID, "out is NULL");
    const int J = static_cast<int>(b->jobs.size());
    if (!J) return LBPM_OK;
    if (b->dirty && (s = rebuild(b))) return s;
    std::vector<int> parity(J);
    for (int j = 0; j < J; ++j) parity[j] = static_cast<int>(b->jobs[j]->step & 1);
    LBPM_BCK(b, cudaMemcpyAsync(b->d_parity, parity.data(), sizeof(int) * J, cudaMemcpyHostToDevice, b->stream));
    const unsigned grid = static_cast<unsigned>(std::max(1, std::min(b->n_mtiles, 4 * b->n_sm)));
    LBPM_BCK(b, launch_batch_measure(b->precision == LBPM_FP16, grid, b->stream, b->d_views, b->d_parity,
                                     b->d_mtiles, b->n_mtiles, b->d_partials, b->d_mbegin, J, b->d_out));
    std::vector<double> S(static_cast<size_t>(NSUM) * J);
    LBPM_BCK(b, cudaMemcpyAsync(S.data(), b->d_out, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, b->stream));
    int err = 0;
    if (b->d_err) LBPM_BCK(b, cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LBPM_BCK(b, cudaStreamSynchronize(b->stream));
    b->launches += 2;
    if (err) {
        LBPM_BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
        for (lbpm_ctx* c : b->jobs) c->unstable = true;
        return bfail(b, LBPM_E_TIMEOUT, "a grid barrier of the fused batch kernel gave up waiting; the jobs' states are "
                                        "incomplete (re-initialise or restore them)");
    }
    lbpm_status st = LBPM_OK;
    for (int j = 0; j < J; ++j) {
        fill_measures(b->jobs[j], S.data() + static_cast<size_t>(NSUM) * j, out + j);
        if (out[j].status) {
            b->jobs[j]->unstable = true;
            st = LBPM_E_UNSTABLE;
        }
    }
    if (st) return bfail(b, st, "a job has non-finite values or a blown-up density");
    return LBPM_OK;
}

lbpm_status lbpm_batch_set_launch(lbpm_batch* b, int threads, int bps_phase, int bps_collide) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (threads != 128 && threads != 192 && threads != 256 && threads != 512)
        return bfail(b, LBPM_E_INVALID, "threads per block must be 128, 192, 256 or 512");
    if (bps_phase < -2 || bps_collide < -2) return bfail(b, LBPM_E_INVALID, "blocks per SM must be >= -2");
    if ((bps_phase == -2) != (bps_collide == -2))
        return bfail(b, LBPM_E_INVALID, "the fused kernel (-2) covers both passes: give -2 for both");
    if (bps_phase == -2 && threads == 512) return bfail(b, LBPM_E_INVALID, "the fused kernel runs 128, 192 or 256 threads");
    LBPM_BCK(b, cudaStreamSynchronize(b->stream));
    if (threads != b->bt) b->dirty = true;
    b->bt = threads;
    b->bps[0] = bps_phase;
    b->bps[1] = bps_collide;
    drop_graph(b);
    return LBPM_OK;
}

lbpm_status lbpm_batch_tune(lbpm_batch* b, int steps_per_candidate, int* threads, int* bps_phase, int* bps_collide) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (b->jobs.empty()) return bfail(b, LBPM_E_STATE, "the batch has no job");
    if (steps_per_candidate < 2 || (steps_per_candidate & 1))
        return bfail(b, LBPM_E_INVALID, "steps_per_candidate must be even and >= 2");
    const std::string key = tune_key(b);
    std::vector<int> best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best.empty()) {
        cudaEvent_t e0, e1;
        LBPM_BCK(b, cudaEventCreate(&e0));
        LBPM_BCK(b, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        const bool h = b->precision == LBPM_FP16;
        for (int bt : {128, 192, 256, 512}) {
            const int occ = std::min(batch_max_blocks(0, h, bt), batch_max_blocks(1, h, bt));
            // the fused persistent kernel (where it applies), one block per tile,
            // then persistent grids at the occupancy limit, half of it, a quarter
            for (int frac : {-2, -1, 4, 2, 1}) {
                if (frac == -2) {
                    if (bt == 512 || b->jobs.size() > static_cast<size_t>(kFusedJobs)) continue;
                    bool ok = true;
                    for (const lbpm_ctx* c : b->jobs) ok = ok && c->params.reservoir_z <= 1;
                    if (!ok) continue;
                }
                const int bps = frac < 0 ? frac : std::max(1, occ * frac / 4);
                if ((s = lbpm_batch_set_launch(b, bt, bps, bps))) break;
                if ((s = lbpm_batch_advance(b, 2))) break;  // capture + warm up
                cudaEventRecord(e0, b->stream);
                if ((s = lbpm_batch_advance(b, steps_per_candidate))) break;
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = {bt, bps, bps};
                }
            }
            if (s) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s) return s;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if ((s = lbpm_batch_set_launch(b, best[0], best[1], best[2]))) return s;
    if (threads) *threads = best[0];
    if (bps_phase) *bps_phase = best[1];
    if (bps_collide) *bps_collide = best[2];
    return LBPM_OK;
}

lbpm_status lbpm_batch_check_barrier(lbpm_batch* b, int missing, double limit_s) {
    lbpm_status s = enter(b);
    if (s) return s;
    if (missing < 0 || !(limit_s > 0.0) || limit_s > 10.0)
        return bfail(b, LBPM_E_INVALID, "missing must be >= 0 and the limit in (0, 10] s");
    unsigned* ctl = static_cast<unsigned*>(balloc(b, sizeof(unsigned) * 2));
    int* err = static_cast<int*>(balloc(b, sizeof(int)));
    if (!ctl || !err) {
        bfree(b, ctl);
        bfree(b, err);
        return bfail(b, LBPM_E_OOM, "barrier self-test allocation failed");
    }
    int h_err = 0;
    const unsigned grid = static_cast<unsigned>(b->n_sm);
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(unsigned) * 2, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), b->stream);
    if (e == cudaSuccess)
        e = launch_barrier_probe(grid, grid + static_cast<unsigned>(missing),
                                 static_cast<unsigned long long>(limit_s * 1e9), ctl, err, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    bfree(b, ctl);
    bfree(b, err);
    if (e != cudaSuccess) return bfail_cuda(b, "barrier self-test", e);
    if (h_err) return bfail(b, LBPM_E_TIMEOUT, "the grid barrier's wait ran out");
    return LBPM_OK;
}

lbpm_status lbpm_batch_launch_count(const lbpm_batch* b, long long* launches) {
    if (!b || !launches) return LBPM_E_INVALID;
    *launches = b->launches;
    return LBPM_OK;
}

}  // extern "C"
