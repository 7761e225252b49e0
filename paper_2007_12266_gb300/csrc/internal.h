// Host-side context and the device view shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbpm.h"
#include "lattice.cuh"

namespace lbm {

// Everything a step kernel needs, passed by value as a kernel parameter.
// Grids are "padded": (nx+2)(ny+2)(nz+2) voxels, one halo layer per face, so
// neighbour voxel = v + off[q] never leaves the allocation. The halo of a
// periodic axis mirrors the opposite face; on a non-periodic axis it is wall.
struct DomainView {
    int n_sites;        // N: pore sites
    int n_halo;         // H: halo voxels that mirror a pore site
    int px, pxpy;       // padded-grid strides in y and z: xi_q is at offset cx + cy px + cz pxpy
    const int* site_vox;   // [N] padded voxel of each site
    const int* vsite;      // [Vp] site id, -1 for solid / wall
    float* phi[2];         // [Vp] phase field by step parity: the phase pass of a step of parity P
                           //     writes phi[P] and the collision reads it; with fp16 storage the
                           //     previous step's phi[P ^ 1] is the reference of the stored
                           //     components (with fp32 storage both point to one grid).
                           //     Solids hold phi_s, walls 0.
    const int* halo_dst;   // [H] padded halo voxel
    const int* halo_site;  // [H] site it mirrors
    const unsigned char* wall6;  // [N] bit q - 1 set when x + xi_q (q = 1..6) is solid or wall
    float* nsum;           // [N] Na + Nb of the current step (phase pass -> collision)
    float* rsum;           // [N] fp16 store: sum_q w_q phi_w(q) of the component references that the
                           //     next phase pass reads (collision -> phase pass, see StoreF16)
    float* drho;           // [N] rho - 1 of each site at the last even step, fp16 store: the
                           //     reference of the stored momentum deviations
    void* f;               // [19][N] momentum distributions (AA in place)
    void* a;               // [7][N]  component A
    void* b;               // [7][N]  component B
    unsigned long long* acc[2];  // [N] sum form: packed fixed-point (Na, Nb) of each site at the step of
                                 //     parity p, accumulated by the previous collision (see pack_sums)
    float tau_a, tau_b, alpha, beta;
    float fx, fy, fz;
    float fterm[9];        // 3 t_q xi_q . F of the odd directions q = 2k + 1 (forcing term per pair), in
                           // the collision's working units (times 2^14 with fp16 storage)
    float s_nu, s_m;       // rates when tau_a == tau_b
    int uniform_tau;
};

// offset of x + xi_q from x in the view's padded grids
__host__ __device__ __forceinline__ int stencil_off(const DomainView& d, int q) {
    return stencil_offset(q, d.px, d.pxpy);
}

struct Allocation {
    void* ptr;
    size_t bytes;
};

}  // namespace lbm

struct lbpm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // allocator
    lbpm_alloc_fn alloc = nullptr;
    lbpm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::vector<lbm::Allocation> allocs;
    // image
    int nx = 0, ny = 0, nz = 0;
    int px = 0, py = 0, pz = 0;
    long long V = 0, Vp = 0;
    long long N = 0, H = 0;
    bool have_image = false, have_fluids = false, unstable = false;
    uint16_t* d_labels = nullptr;   // [V]
    int* d_site_vox = nullptr;      // [N]
    int* d_vsite = nullptr;         // [Vp]
    float* d_phi = nullptr;         // [Vp]
    float* d_phi_alt = nullptr;     // [Vp] fp16 storage: the phase grid of odd steps
    int* d_halo_dst = nullptr;      // [H]
    int* d_halo_site = nullptr;     // [H]
    unsigned char* d_wall6 = nullptr;  // [N] face links that bounce back
    float* d_nsum = nullptr;        // [N]
    float* d_rsum = nullptr;        // [N] fp16 storage
    double* d_face_part = nullptr;          // flux inlet: per-block sums (2 * kFaceBlocks)
    float* d_face_rho = nullptr;            // flux inlet: (rho, rho - 1) of the inlet face
    float* d_drho = nullptr;                // [N] fp16 store
    void* d_f = nullptr;
    void* d_a = nullptr;
    void* d_b = nullptr;
    unsigned long long* d_acc = nullptr;   // [2N] sum form: packed component sums by step parity
    int step_form = LBPM_STEP_AUTO;        // lbpm_set_step_form
    int* d_slab_site = nullptr;     // reservoir sites
    signed char* d_slab_side = nullptr;
    long long n_slab = 0;
    double* d_partials = nullptr;   // measure partial sums
    long long n_partials = 0;
    // parameters and state
    lbpm_params params{};
    long long step = 0;
    long long launches = 0;
    int block = 256;
    // captured step bundles: graphs[0] = 2 timesteps, graphs[1] = 16 timesteps (population form);
    // sum_graphs[0] / [1]: 2 / 16 middle timesteps of the sum form
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graphs[2] = {nullptr, nullptr};
    cudaGraphExec_t sum_graphs[2] = {nullptr, nullptr};
    bool use_graphs = true;
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_collide, ev_phase;  // (start, end) indices
    size_t ev_next = 0;
};

namespace lbm {

// device memory through the ctx's allocator
void* dalloc(lbpm_ctx* c, size_t bytes);
void dfree(lbpm_ctx* c, void* p);

// launchers (return cudaError_t of the launch)
cudaError_t launch_flag_pore(const uint16_t* labels, long long V, int* flags, cudaStream_t s);
cudaError_t exclusive_scan(lbpm_ctx* c, const int* in, int* out, long long n);
cudaError_t launch_scatter_sites(const lbpm_ctx* c, const int* scan, cudaStream_t s);
cudaError_t launch_fill_halo(const lbpm_ctx* c, cudaStream_t s);
cudaError_t launch_halo_flags(const lbpm_ctx* c, int* flags, cudaStream_t s);
cudaError_t launch_halo_scatter(const lbpm_ctx* c, const int* flags, const int* scan, cudaStream_t s);
cudaError_t launch_affinity_table(const lbpm_ctx* c, const float* table, int n_labels, cudaStream_t s);
cudaError_t launch_affinity_map(const lbpm_ctx* c, const float* map, cudaStream_t s);
cudaError_t launch_slab_flags(const lbpm_ctx* c, int* flags, cudaStream_t s);
cudaError_t launch_slab_scatter(const lbpm_ctx* c, const int* flags, const int* scan, cudaStream_t s);
cudaError_t launch_export_index(const lbpm_ctx* c, long long* site2vox, int* nbr, cudaStream_t s);
cudaError_t launch_wall_mask(const lbpm_ctx* c, cudaStream_t s);

// Look up (once per device, with that device current) the device address of
// the static staging array of lbpm_read_field_noalloc; called by lbpm_create.
cudaError_t noalloc_setup(int device);

DomainView make_view(const lbpm_ctx* c);
cudaError_t launch_init_fluids(const lbpm_ctx* c, const float* phi0, cudaStream_t s);
cudaError_t launch_ref_sum(const lbpm_ctx* c, int parity, cudaStream_t s);
cudaError_t launch_phase(const lbpm_ctx* c, int parity, cudaStream_t s);
cudaError_t launch_collide(const lbpm_ctx* c, int parity, cudaStream_t s);
// Sum form of a timestep (components carried as per-site sums, see pack_sums):
// phase pass from the sums (write_nsum: also Na + Nb for a population-form
// collision), and the collision scattering its recolored values into the
// receivers' sums (from_sums: the site's own Na, Nb come from its sums,
// otherwise from the phase pass of the population form).
cudaError_t launch_phase_sum(const lbpm_ctx* c, int parity, bool write_nsum, cudaStream_t s);
cudaError_t launch_collide_sum(const lbpm_ctx* c, int parity, bool from_sums, cudaStream_t s);
// Reservoir slabs (reservoir_z = 1) in the sum form: the reset state goes into
// the sums the next step (parity `parity`) reads, and into its f slots.
cudaError_t launch_reservoir_sum(const lbpm_ctx* c, int parity, cudaStream_t s);
// Whether a context can run the sum form (no pressure or flux faces, the
// population form not forced).
bool sum_form_capable(const lbpm_ctx* c);
// Clear the sums that the first step of a sum-form run (parity `par`) accumulates into.
cudaError_t clear_sums(const lbpm_ctx* c, int par, cudaStream_t s);
cudaError_t launch_reservoir(const lbpm_ctx* c, int parity, cudaStream_t s);
// flux inlet: blocks of the fixed-order face reduction
constexpr int kFaceBlocks = 64;
cudaError_t launch_morph(const lbpm_ctx* c, int parity, float delta, int R, int apply, float* phi_grid,
                         float* dist_grid, float* ntot, int3* off, long long* off_lin, float* off_len, int n_off,
                         unsigned long long* counts, cudaStream_t s);

constexpr int NSUM = 27;  // per-site sums reduced by the measure kernel
void fill_measures(const lbpm_ctx* c, const double* S, lbpm_measures* out);

// One tile of a batched launch: `first` is the first thread index (site, or
// site/halo entry for the phase pass) of job `job` that the block handles.
struct BatchTile {
    int job;
    int first;
};
// Job table of one batched step launch, passed by value in the kernel's
// parameter space (at most kBatchLaunchJobs jobs per launch; larger batches
// take several launches per kernel). Tiles of bt threads are numbered job by
// job: job j owns tiles [tile_begin[j], tile_begin[j + 1]). Every thread of a
// block finds its job from blockIdx alone, so the job index and the view's
// fields are warp-uniform values read from the constant bank.
constexpr int kBatchLaunchJobs = 128;
struct BatchLaunch {
    int n_jobs;
    int tile_begin[kBatchLaunchJobs + 1];
    DomainView v[kBatchLaunchJobs];
};
// form: phase pass 0 = populations, 1 = sums, 2 = sums writing N; collision
// 0 = populations, 1 = sums from the phase pass, 2 = sums from the sums.
cudaError_t launch_batch(int kernel, int form, int par, bool fp16, int bt, unsigned grid, cudaStream_t s,
                         const BatchLaunch& p);
cudaError_t launch_batch_measure(bool fp16, unsigned grid, cudaStream_t s, const DomainView* v, const int* parity,
                                 const BatchTile* t, int nt, double* partials, const int* tile_begin, int n_jobs,
                                 double* out);
int batch_max_blocks(int kernel, bool fp16, int bt);
cudaError_t launch_measure(lbpm_ctx* c, int parity, double* d_out, cudaStream_t s);
cudaError_t launch_field(const lbpm_ctx* c, int parity, int which, float* dense, cudaStream_t s);
cudaError_t launch_export_dist(const lbpm_ctx* c, int parity, int which, float* out, cudaStream_t s);
cudaError_t launch_read_box(const lbpm_ctx* c, int parity, int which, const int* lo, const int* hi, float* out,
                            cudaStream_t s);
cudaError_t launch_import_dist(const lbpm_ctx* c, int parity, int which, const float* in, cudaStream_t s);

}  // namespace lbm
