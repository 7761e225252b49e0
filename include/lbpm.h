/*
 * lbpm.h - C ABI of the GB300 color-gradient lattice Boltzmann library.
 *
 * The library advances the two-fluid color-gradient LBM of the LBPM paper
 * (arXiv 2007.12266) on the pore sites of a segmented 3-D image, on one
 * NVIDIA GB300 (sm_103a). One context ("ctx") holds one simulated domain.
 *
 * Model (Sec. 3.1 "Color Lattice-Boltzmann Model"):
 *   - D3Q19 MRT momentum LBE with body force F; equilibrium moments carry the
 *     interfacial-tension terms alpha|C| (m1, m9, m11, m13, m14, m15),
 *     sigma_ab = 6 alpha;
 *   - two D3Q7 component distributions A, B recolored by the phase field
 *     phi = (Na - Nb)/(Na + Nb) with parameter beta (Eqs. LBE-mass-a/b);
 *   - wetting through a per-solid-voxel affinity phi_s that enters the
 *     color gradient C (Sec. 3.2, Eq. phi_s: cos(theta_eq) = phi_s);
 *   - streaming in place (AA pattern) with halfway bounce-back at solids.
 *
 * Conventions shared by every call:
 *   - Voxel arrays are x-fastest: voxel (x, y, z) is at x + nx*(y + ny*z).
 *   - Every host input buffer is owned by the caller and is copied before the
 *     call returns; the library keeps no host pointer.
 *   - Device memory is owned by the ctx. It comes from the allocator set with
 *     lbpm_set_allocator (the Python binding installs PyTorch's caching
 *     allocator), else from cudaMalloc.
 *   - Work is issued on the ctx's CUDA stream. Calls that return host data
 *     synchronize that stream; lbpm_advance does not.
 *   - No C++ exception crosses this ABI. Every call returns an lbpm_status;
 *     lbpm_last_error(ctx) gives a message for the last failure. Errors raised
 *     asynchronously by device work surface at the next lbpm_sync,
 *     lbpm_measure, lbpm_read_* or lbpm_advance call.
 *   - A ctx is not thread-safe: use it from one host thread at a time.
 */
#ifndef LBPM_H
#define LBPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbpm_ctx lbpm_ctx;

typedef enum {
    LBPM_OK = 0,
    LBPM_E_INVALID = 1,   /* bad argument, size or parameter */
    LBPM_E_OOM = 2,       /* device allocation failed */
    LBPM_E_CUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    LBPM_E_STATE = 4,     /* call out of order (e.g. advance before init) */
    LBPM_E_UNSTABLE = 5,  /* the last measure found non-finite values or a blown-up density */
    LBPM_E_TIMEOUT = 6    /* a bounded device-side wait gave up (the fused batch kernel's
                             grid barrier; see lbpm_batch_measure, lbpm_batch_check_barrier) */
} lbpm_status;

/* Storage precision of the distributions. */
enum { LBPM_FP32 = 0, LBPM_FP16 = 1 };

/* Step forms for lbpm_set_step_form. */
enum { LBPM_STEP_AUTO = 0, LBPM_STEP_POPULATIONS = 1 };

/* Field selectors for lbpm_read_field. */
enum { LBPM_FIELD_PHI = 0, LBPM_FIELD_PRESSURE = 1, LBPM_FIELD_UX = 2,
       LBPM_FIELD_UY = 3, LBPM_FIELD_UZ = 4, LBPM_FIELD_NA = 5, LBPM_FIELD_NB = 6,
       LBPM_FIELD_RHO = 7 };

/* Distribution selectors for lbpm_read_distributions / lbpm_write_distributions. */
enum { LBPM_DIST_F = 0, LBPM_DIST_A = 1, LBPM_DIST_B = 2 };

/*
 * Model parameters (Sec. 3.1): tau_a, tau_b set the kinematic viscosity of
 * each fluid, nu = (tau - 1/2)/3 (the relaxation matrix "is determined based
 * on the kinematic viscosity"); alpha sets the interfacial tension
 * sigma_ab = 6 alpha; beta sets the interface thickness; force is the
 * constant body force F. Unsteady-flow boundaries (Sec. 4.1), z axis
 * non-periodic: reservoir_z = 1, reservoir slabs - after each step the four
 * z-layers at z = 0 are reset to fluid A at rest at density rho_in and the
 * four at z = nz - 1 to fluid B at rho_out; reservoir_z = 2, constant
 * pressure at the faces (Zou and He's scheme, cited in Sec. 4.1) - after each
 * step the populations entering the face sites z = 0 and z = nz - 1 from
 * outside are rebuilt so that those sites have density rho_in (rho_out) and no
 * tangential velocity, and fluid A enters at the inlet, fluid B at the
 * outlet; reservoir_z = 3, constant flux at the inlet (the flux condition of
 * Sec. 4.1: a total volumetric flow rate, not a velocity at each point) and
 * constant pressure rho_out at the outlet - the inlet face is a pressure face
 * whose uniform density is chosen at every step so that the face velocities
 * sum to flux_in (lattice units: sum over the inlet sites of u_z), letting
 * the local inlet velocities follow the interior flow.
 * Valid ranges: tau > 0.5; alpha >= 0; beta >= 0 (0 disables recoloring);
 * finite force; precision LBPM_FP32 or LBPM_FP16; periodic[i] in {0, 1};
 * rho_in, rho_out > 0. Otherwise LBPM_E_INVALID.
 */
typedef struct {
    double tau_a, tau_b;
    double alpha, beta;
    double force[3];
    int precision;        /* storage of the distributions: LBPM_FP32, or LBPM_FP16 - each value kept in
                           * fp16 as its deviation from a local rest state (about half the memory and
                           * traffic), all arithmetic fp32, the measures fp64 */
    int periodic[3];      /* 1 = periodic axis; a non-periodic face is a solid wall (phi_s = 0) */
    int reservoir_z;      /* 0 none, 1 reservoir slabs, 2 pressure faces, 3 flux inlet + pressure outlet */
    double rho_in, rho_out;
    double flux_in;       /* reservoir_z = 3: total inlet flux, 0 <= flux_in < number of inlet sites */
} lbpm_params;

/*
 * Basic analysis and integral measures of the current state, all summed in
 * fp64 on the device in a fixed order (deterministic for a given domain):
 * basic analysis of Sec. 4 (saturation, average velocity and pressure per
 * fluid, instability detection) and the integral measures of Sec. 3.4 (table
 * of integral measures: M, P, K per fluid region, p_alpha = mean pressure;
 * regions: phi > 0 is fluid A, the rest is B). Velocities are the reported
 * velocity u = (j + F/2)/rho0, pressure p = rho/3.
 *   sat_mass   = sum Na / sum (Na + Nb)         (conserved saturation of A)
 *   sat_count  = #{phi > 0} / n_sites
 *   flux       = (1/V) sum_pore u  (Darcy flux; V counts all voxels)
 *   flux_a/b   = (1/V) sum_pore (Na/N) u, (Nb/N) u
 *   mom_a/b    = sum_region rho u; ke_a/b = sum_region rho u.u
 *   mass_a/b   = sum Na, sum Nb; mass_total = sum rho
 *   vol_a/b    = site counts of the regions; p_a/b = region mean of p
 *   ca         = total capillary number, Eq. capillary_number:
 *                (eps_a mu_a |<u>_a| + eps_b mu_b |<u>_b|)/sigma with
 *                <u>_alpha = P_alpha/M_alpha, eps_alpha = vol_alpha/V,
 *                mu = (tau - 1/2)/3, sigma = 6 alpha
 *   status     = 0 ok, bit 0 a non-finite value, bit 1 a component density
 *                below -1e-2 or a non-positive total density (instability)
 */
typedef struct {
    long long step;
    double sat_mass, sat_count;
    double mass_a, mass_b, mass_total;
    double mom_a[3], mom_b[3];
    double flux[3], flux_a[3], flux_b[3];
    double ke_a, ke_b;
    double p_a, p_b;
    double vol_a, vol_b;
    double ca;
    long long n_sites;
    int status;
} lbpm_measures;

/* Device allocator hooks: alloc returns a device pointer of at least `bytes`
 * usable on `stream`, or NULL; free releases it. `user` is passed back. */
typedef void* (*lbpm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*lbpm_free_fn)(void* ptr, void* user);

/* Library version string (static storage). */
const char* lbpm_version(void);

/* Create a ctx on CUDA `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream: the library has no notion of
 * a framework's "current" stream, so the Python binding passes PyTorch's
 * current stream explicitly). *out receives the ctx. Set-up done here, once
 * per device: the device address of lbpm_read_field_noalloc's static staging
 * array is looked up (which places that array on the GPU).
 * Errors: LBPM_E_INVALID (out NULL, bad device), LBPM_E_CUDA. */
lbpm_status lbpm_create(lbpm_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the ctx and the ctx itself. NULL is a no-op. */
lbpm_status lbpm_destroy(lbpm_ctx* ctx);

/* Route the ctx's device allocations through alloc/free. Must be called
 * before lbpm_load_image (LBPM_E_STATE otherwise). NULL alloc restores
 * cudaMalloc/cudaFree. */
lbpm_status lbpm_set_allocator(lbpm_ctx* ctx, lbpm_alloc_fn alloc, lbpm_free_fn free_fn,
                               void* user);

/* Message for the last failed call on ctx (or the last failed lbpm_create
 * when ctx is NULL). Valid until the next call on the ctx. */
const char* lbpm_last_error(const lbpm_ctx* ctx);

/*
 * Load the labelled image (Sec. 3.3, "Initial conditions and wetting maps":
 * one integer label per voxel). labels: uint16 [nz][ny][nx], x fastest;
 * label 0 = pore, label k >= 1 = solid of wetting class k. Builds the sparse
 * pore-site index on the device: pore voxels are numbered in x-fastest
 * lexicographic order, and each site's 18 neighbours are resolved with
 * periodic wrap on the axes params.periodic marks (call lbpm_set_params
 * first, or the default is periodic on all axes). Affinities default to 0
 * until lbpm_set_affinity_* is called. Replaces any previous image and
 * discards the fluid state.
 * Limits: nx, ny, nz >= 1; (nx+2)(ny+2)(nz+2) < 2^31; at least one pore.
 * Errors: LBPM_E_INVALID, LBPM_E_OOM, LBPM_E_CUDA.
 */
lbpm_status lbpm_load_image(lbpm_ctx* ctx, const uint16_t* labels, int nx, int ny, int nz);

/* Wetting map by label (Sec. 3.2: "the wetting map assigns a label to each
 * solid voxel, and the associated wetting affinity is specified for each
 * label"): affinity_by_label[k] is phi_s of label k, for k < n_labels
 * (entry 0 is ignored). Labels >= n_labels get 0. |phi_s| <= 1.
 * Requires a loaded image (LBPM_E_STATE). Takes effect from the next step. */
lbpm_status lbpm_set_affinity_table(lbpm_ctx* ctx, const float* affinity_by_label, int n_labels);

/* Per-voxel wetting map: affinity_per_voxel float [nz][ny][nx]; values at
 * solid voxels are used as phi_s, pore entries are ignored. |phi_s| <= 1. */
lbpm_status lbpm_set_affinity_map(lbpm_ctx* ctx, const float* affinity_per_voxel);

/* Set the model parameters (see lbpm_params). Periodicity and precision
 * changes after lbpm_load_image rebuild the index / storage and discard the
 * fluid state (LBPM_E_STATE is not raised; the state must be re-initialised). */
lbpm_status lbpm_set_params(lbpm_ctx* ctx, const lbpm_params* params);

/* Initialise the fluids from a phase field phi0 float [nz][ny][nx] (pore
 * entries read, clamped to [-1, 1]): Na = (1+phi0)/2, Nb = (1-phi0)/2,
 * A_q = w_q Na, B_q = w_q Nb, f_q = t_q (rho = 1, u = 0); step counter 0.
 * Reservoir layers, if enabled, are then set. Errors: LBPM_E_STATE (no image). */
lbpm_status lbpm_init_fluids(lbpm_ctx* ctx, const float* phi0_per_voxel);

/* Enqueue nsteps timesteps on the ctx stream (asynchronous). Each step: the
 * phase pass (phi and N from A, B), then the fused collide-stream pass
 * (color gradient, MRT collision with the alpha terms and the force,
 * recoloring, AA streaming with bounce-back), then the reservoir reset.
 * nsteps >= 0. Errors: LBPM_E_STATE (no fluids), LBPM_E_UNSTABLE (a previous
 * measure flagged the state), LBPM_E_CUDA. */
lbpm_status lbpm_advance(lbpm_ctx* ctx, long long nsteps);

/* Wait for the ctx stream and report any asynchronous device error. */
lbpm_status lbpm_sync(lbpm_ctx* ctx);

/* Compute the measures of the current state (synchronizes). Returns
 * LBPM_E_UNSTABLE, with *out filled, when out->status != 0. */
lbpm_status lbpm_measure(lbpm_ctx* ctx, lbpm_measures* out);

/* Dense field of the current state into out_dense float [nz][ny][nx]
 * (caller-allocated, nx*ny*nz floats); solid voxels get NaN. */
lbpm_status lbpm_read_field(lbpm_ctx* ctx, int which, float* out_dense);

/* Largest image (nx*ny*nz voxels) that lbpm_read_field_noalloc accepts. */
#define LBPM_NOALLOC_FIELD_MAX_VOXELS (1LL << 21)

/*
 * Allocation-free lbpm_read_field (the paper has no counterpart; this is a
 * library service). For callers that cannot let the library allocate device
 * memory after set-up - for example a loop that runs under a fixed device
 * memory budget handed out at start-up, or a host that must not enter the
 * allocator while other work owns it. lbpm_read_field allocates and frees a
 * temporary device buffer on every call; this variant stages the field in
 * one static device array of LBPM_NOALLOC_FIELD_MAX_VOXELS floats (8 MiB,
 * enough for a 128^3 image) that the library holds on every GPU where it is
 * loaded, until the process exits. It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * Same arguments, output and errors as lbpm_read_field, plus LBPM_E_INVALID
 * when the image has more than LBPM_NOALLOC_FIELD_MAX_VOXELS voxels.
 * lbpm_create looks up the array's device address (once per device, with
 * that device current), which also loads the array onto that GPU, so the
 * call itself neither loads code nor places memory. All calls on a device
 * share the array and it keeps the last call's contents: each call
 * overwrites every entry it returns (NaN at solids), but calls whose device
 * work overlaps (other streams or threads) race on it, so callers must
 * serialise them.
 */
lbpm_status lbpm_read_field_noalloc(lbpm_ctx* ctx, int which, float* out_dense);

/* Distributions of the current state in canonical order, population-major:
 * out[q*n_sites + n] = f_q (or A_q, B_q) at site n, the value the next step
 * will collide, whatever the AA parity. Q = 19 for F, 7 for A, B. */
lbpm_status lbpm_read_distributions(lbpm_ctx* ctx, int which, float* out_canonical);

/* Distributions of the current state at the voxels of a sub-box of the image
 * (a library service for probing a large domain without exporting it whole):
 * lo[3], hi[3] are voxel bounds (x, y, z) with 0 <= lo < hi <= (nx, ny, nz);
 * out (caller-allocated, Q*bx*by*bz floats, b = hi - lo) receives
 * out[q*bx*by*bz + (z*by + y)*bx + x] = f_q (A_q, B_q) of the voxel lo + (x, y, z)
 * in canonical order as lbpm_read_distributions gives it, NaN at solid voxels.
 * Errors: LBPM_E_INVALID (NULL pointer, unknown set, box empty or outside the
 * image), LBPM_E_STATE (no fluids), LBPM_E_OOM, LBPM_E_CUDA. */
lbpm_status lbpm_read_box(lbpm_ctx* ctx, int which, const int* lo, const int* hi, float* out);

/* Overwrite one distribution set from canonical order (same layout as
 * lbpm_read_distributions) at the current step parity. */
lbpm_status lbpm_write_distributions(lbpm_ctx* ctx, int which, const float* in_canonical);

/* Number of pore sites of the loaded image (0 before lbpm_load_image). */
lbpm_status lbpm_num_sites(const lbpm_ctx* ctx, long long* n_sites);

/* Completed timesteps since lbpm_init_fluids / lbpm_restore. */
lbpm_status lbpm_step_count(const lbpm_ctx* ctx, long long* step);

/* The sparse index: site2vox int64 [n_sites] (voxel index of each site) and
 * nbr int32 [18][n_sites]: nbr[(q-1)*n_sites + n] is the site reached from
 * site n along xi_q (q = 1..18, D3Q19 order of Eq. d3q19 with the sign order
 * (+,-) per axis pair and (++, --, +-, -+) per edge group), wrapped on
 * periodic axes, or -1 where that voxel is solid or outside the domain.
 * Either pointer may be NULL to skip it. */
lbpm_status lbpm_get_index(lbpm_ctx* ctx, int64_t* site2vox, int32_t* nbr);

/* Snapshot of the full fluid state (distributions in canonical fp32 order
 * plus the step counter) into host_buf. With host_buf NULL, *bytes receives
 * the size needed. lbpm_restore reloads such a snapshot into a ctx holding
 * the same image; the next steps are bit-identical to an uninterrupted run
 * in FP32 storage. Errors: LBPM_E_INVALID (size or header mismatch). */
lbpm_status lbpm_snapshot(lbpm_ctx* ctx, void* host_buf, size_t* bytes);
lbpm_status lbpm_restore(lbpm_ctx* ctx, const void* host_buf, size_t bytes);

/*
 * How lbpm_advance carries the two component distributions between the
 * timesteps of one call (a library choice; the paper's model, Eqs.
 * LBE-mass-a/b, is the same in both forms).
 *   LBPM_STEP_POPULATIONS: every timestep stores the 7 + 7 recolored D3Q7
 *     populations in place (AA pattern) and the next phase pass reads them.
 *   LBPM_STEP_AUTO (default): inside a call of two or more timesteps, each
 *     collision adds its recolored values straight into the component
 *     densities Na, Nb of the sites that receive them (the streaming
 *     destinations, or the site itself on a bounce-back link), kept per site
 *     as one 64-bit fixed-point pair (2^-28 units); the next phase pass and
 *     collision read those sums instead of 14 populations. This is exact
 *     algebra: the recolored populations depend only on the writer's Na, Nb,
 *     velocity and colour normal, and the next step uses only their sums.
 *     Integer sums are independent of the order of the additions (results
 *     are deterministic) and conserve each component's mass exactly. The
 *     first timestep of a call reads, and the last one writes, the
 *     populations, so between calls the state is the same as in the
 *     population form and every export, measure and snapshot applies
 *     unchanged. Reservoir slabs (reservoir_z = 1) reset the slab sites' sums;
 *     runs with pressure or flux faces (reservoir_z = 2, 3) always use the
 *     population form. The batched form (lbpm_batch_advance) and the serving
 *     loop use the sum form when every job of the batch can.
 * Errors: LBPM_E_INVALID (unknown form).
 */
lbpm_status lbpm_set_step_form(lbpm_ctx* ctx, int form);

/* Kernel timing for roofline reports: while enabled, lbpm_advance records CUDA
 * events around each launch of the fused collide-stream kernel on the ctx
 * stream. lbpm_kernel_timing returns (after synchronizing) the summed event
 * time in ms and the launch count since the last reset, and resets them. */
lbpm_status lbpm_enable_kernel_timing(lbpm_ctx* ctx, int enable);
lbpm_status lbpm_kernel_timing(lbpm_ctx* ctx, double* ms_collide, long long* n_collide,
                               double* ms_phase, long long* n_phase);

/*
 * Batched form: several jobs (independent contexts on one GPU, same storage
 * precision) advanced together. Every timestep of the whole batch is ONE
 * launch of the phase pass and ONE of the fused collide-stream kernel, both
 * over a list of tiles that covers all jobs' sites (or, with the fused launch
 * shape of lbpm_batch_set_launch, one kernel runs every pass of a bundle);
 * bundles of two steps are replayed from a CUDA graph. Inside a call of two or more steps the
 * components travel as per-site sums when every job allows it (see
 * lbpm_set_step_form). Each job's results agree with
 * advancing it alone to fp32 rounding (1e-5 relative per distribution after
 * 24 steps in the tests: the batched and single-domain kernels are compiled
 * separately and the compiler may contract multiply-adds differently); two
 * batched runs of the same jobs are bit-identical. Jobs keep their own state and every per-job call
 * (lbpm_measure, lbpm_read_field, ...) stays valid; a job joins at an even
 * step and must be removed before it is destroyed. After changing a job's
 * parameters, call lbpm_batch_refresh. Work runs on the batch's stream: use
 * the same stream for the jobs, or synchronise them.
 */
typedef struct lbpm_batch lbpm_batch;

/* Create an empty batch on CUDA `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). *out receives it.
 * Errors: LBPM_E_INVALID (out NULL, bad device), LBPM_E_OOM, LBPM_E_CUDA. */
lbpm_status lbpm_batch_create(lbpm_batch** out, int device, void* cuda_stream);
/* Wait for the batch's stream and free its tables; the jobs are not touched
 * (they stay valid and belong to the caller). NULL is a no-op. */
lbpm_status lbpm_batch_destroy(lbpm_batch* batch);
/* Allocator hooks for the batch's own tables (see lbpm_set_allocator). */
lbpm_status lbpm_batch_set_allocator(lbpm_batch* batch, lbpm_alloc_fn alloc, lbpm_free_fn free_fn, void* user);
const char* lbpm_batch_last_error(const lbpm_batch* batch);
/* Add / remove a job (LBPM_E_STATE if the job has no fluids or is at an odd
 * step; LBPM_E_INVALID for another device, another precision or a repeat). */
lbpm_status lbpm_batch_add(lbpm_batch* batch, lbpm_ctx* job);
lbpm_status lbpm_batch_remove(lbpm_batch* batch, lbpm_ctx* job);
/* Re-read every job's parameters (e.g. after a body-force change). */
lbpm_status lbpm_batch_refresh(lbpm_batch* batch);
lbpm_status lbpm_batch_size(const lbpm_batch* batch, int* n_jobs, long long* n_sites);
/* Advance every job by nsteps (even, asynchronous). */
lbpm_status lbpm_batch_advance(lbpm_batch* batch, long long nsteps);
/* Measures of every job, out[j] for the j-th job in insertion order
 * (see lbpm_measures); LBPM_E_UNSTABLE if any job is flagged; LBPM_E_TIMEOUT
 * if a grid barrier of the fused kernel (below) gave up waiting since the last
 * measure (the jobs are then flagged unstable: their states are incomplete). */
lbpm_status lbpm_batch_measure(lbpm_batch* batch, lbpm_measures* out);
/* Launch shape: threads per block (128, 192, 256 or 512) and resident blocks per
 * SM of the persistent phase and collide grids (0 = occupancy limit, -1 = no
 * persistent grid: one block per tile, scheduled by the hardware; -2 for both
 * = one fused persistent kernel per bundle of steps: a cooperative grid of
 * every block that fits the GPU runs the phase pass, the collision and the
 * reservoir reset of all jobs, taking tiles from an atomic counter in each
 * pass, with a grid barrier between passes whose wait gives up after 2 s; 128,
 * 192 or 256 threads, batches of up to 112 jobs without pressure or flux faces,
 * other batches keep the separate launches). A new batch starts at 192 threads
 * and -1 for both kernels. */
lbpm_status lbpm_batch_set_launch(lbpm_batch* batch, int threads, int blocks_per_sm_phase,
                                  int blocks_per_sm_collide);
/* Autotuner: times each candidate launch shape over one advance call of
 * steps_per_candidate (even) real steps - all candidates compute identical
 * results - keeps the fastest, and caches it per GPU, precision and size
 * class (log2 of the batch's site count) for the process. Returns the chosen
 * shape. A call's first and last steps carry the populations and the others
 * the component sums (lbpm_set_step_form), so a count of 16 or more times
 * mostly the middle steps that dominate long runs. */
lbpm_status lbpm_batch_tune(lbpm_batch* batch, int steps_per_candidate, int* threads, int* blocks_per_sm_phase,
                            int* blocks_per_sm_collide);
/* Kernel launches the batch has issued so far (graph replays counted per
 * kernel node). Errors: LBPM_E_INVALID (NULL argument). */
lbpm_status lbpm_batch_launch_count(const lbpm_batch* batch, long long* launches);
/* Self-test of the fused kernel's bounded grid barrier (a library diagnostic;
 * the paper has no counterpart): one cooperative grid of one block per SM
 * meets at a barrier that expects `missing` more arrivals than there are
 * blocks, with a wait limit of limit_s seconds (0 < limit_s <= 10). With
 * missing = 0 the barrier completes (LBPM_OK); with missing > 0 nobody supplies
 * the arrivals, every block's wait runs out after the limit and the call
 * returns LBPM_E_TIMEOUT, with the GPU left usable. Errors: LBPM_E_INVALID,
 * LBPM_E_OOM, LBPM_E_CUDA. */
lbpm_status lbpm_batch_check_barrier(lbpm_batch* batch, int missing, double limit_s);

/*
 * Serving loop (continuous batching) for the protocols of Sec. 4: steady
 * state (Sec. 4.2: periodic flow driven by a body force), unsteady
 * displacement (Sec. 4.1: inlet/outlet reservoirs) and centrifuge-like runs
 * (Sec. 4.1: body force raised by force_factor each time the saturation
 * changes by less than sw_tol over an interval, up to force_cap). A job ends
 * when the Darcy flux along the drive changes by less than flux_tol (relative)
 * over one check interval - standing in for the capillary-number test of
 * Eq. convergence - or at max_steps.
 * The caller drives the server with lbpm_server_run: each call admits queued
 * jobs first come first served while a slot (max_jobs) and the device-memory
 * budget allow (admission by the job's estimated footprint), advances every
 * running job by one check interval in one batched launch sequence (jobs
 * admitted in this call join the running batch at once), measures them and
 * retires the finished ones. Finished jobs keep their device state, so their
 * fields stay readable (lbpm_server_job_ctx), until lbpm_server_release or
 * until that memory is needed to admit a queued job (oldest finished job
 * first; its status and last measures stay available).
 */
typedef struct lbpm_server lbpm_server;

enum { LBPM_JOB_STEADY = 0, LBPM_JOB_UNSTEADY = 1, LBPM_JOB_CENTRIFUGE = 2 };
enum { LBPM_JOB_QUEUED = 0, LBPM_JOB_RUNNING = 1, LBPM_JOB_DONE = 2, LBPM_JOB_FAILED = 3,
       LBPM_JOB_CANCELLED = 4 };

/* A job: image, wetting map (NULL = phi_s 0), initial phases and parameters,
 * as for lbpm_load_image / lbpm_set_affinity_map / lbpm_init_fluids /
 * lbpm_set_params. The arrays are copied by lbpm_server_submit. */
typedef struct {
    const uint16_t* labels;
    int nx, ny, nz;
    const float* affinity;
    const float* phi0;
    lbpm_params params;
    int kind;
    long long max_steps;
    double flux_tol;
    double sw_tol;
    double force_factor, force_cap;
    /* Steady-state jobs: body-force adaptation to a target capillary number
     * (Sec. 4.2, Eq. LB_body_force_adaptation). ca_target > 0 rescales the
     * force by lbpm_force_rescale every relax_steps steps (rounded up to the
     * check interval) while |Ca / ca_target - 1| >= ca_tol, and the job can
     * only converge once Ca is within ca_tol of the target. 0 = off. */
    double ca_target;
    long long relax_steps;
    double ca_tol;
} lbpm_job_spec;

/* Job status; times in seconds on the server's steady clock. */
typedef struct {
    int state;
    long long steps;
    long long n_sites;
    size_t footprint;
    double t_submit, t_admit, t_done;
    int force_raises;      /* centrifuge raises or capillary-number rescales so far */
    lbpm_measures last;
    double force[3];       /* body force in effect */
} lbpm_job_status;

/* hbm_budget_bytes = 0: 90 % of the free device memory. check_interval:
 * steps per round (even). */
lbpm_status lbpm_server_create(lbpm_server** out, int device, void* cuda_stream, size_t hbm_budget_bytes,
                               int max_jobs, int check_interval);
/* Free the server, its batch and every job's device state (finished or
 * not). NULL is a no-op. */
lbpm_status lbpm_server_destroy(lbpm_server* server);
/* Allocator hooks for every job and the batch (see lbpm_set_allocator);
 * LBPM_E_STATE once jobs were submitted. */
lbpm_status lbpm_server_set_allocator(lbpm_server* server, lbpm_alloc_fn alloc, lbpm_free_fn free_fn, void* user);
/* Message of the server's last failed call ("" if none; valid until the next call). */
const char* lbpm_server_last_error(const lbpm_server* server);
/* Queue a job (LBPM_E_OOM if its footprint exceeds the whole budget). */
lbpm_status lbpm_server_submit(lbpm_server* server, const lbpm_job_spec* spec, long long* ticket);
/* One round: admit, advance one interval, measure, retire. */
lbpm_status lbpm_server_run(lbpm_server* server, int* n_running, int* n_queued, int* n_finished);
lbpm_status lbpm_server_poll(lbpm_server* server, long long ticket, lbpm_job_status* out);
/* The job's context (NULL once released) for reading fields or distributions. */
lbpm_status lbpm_server_job_ctx(lbpm_server* server, long long ticket, lbpm_ctx** ctx);
lbpm_status lbpm_server_cancel(lbpm_server* server, long long ticket);
lbpm_status lbpm_server_release(lbpm_server* server, long long ticket);
lbpm_status lbpm_server_stats(const lbpm_server* server, long long* site_updates, size_t* used_bytes,
                              size_t* budget_bytes);

/* Body-force adaptation to a target capillary number (Sec. 4.2, Eq.
 * LB_body_force_adaptation): out = g * force with g = ca_target / ca clamped
 * to [1 / max_factor, max_factor] (the paper caps each change at a factor of
 * two: max_factor = 2). ca <= 0 (no flow yet) gives g = max_factor. Host
 * arithmetic only. *factor (may be NULL) receives g. Errors: LBPM_E_INVALID
 * for NULL force/out, ca_target <= 0, max_factor < 1 or a non-finite input. */
lbpm_status lbpm_force_rescale(const double force[3], double ca, double ca_target, double max_factor,
                               double out[3], double* factor);

/* Shell aggregation, one morphological step (Sec. 3.3): moves the interface
 * of fluid A (phi > 0) by the signed distance delta in voxels (dilation > 0,
 * erosion < 0) through its distance map Phi_A (< 0 inside A): Eq. lb-dist
 * solved for the distance where |phi| < tanh(3 beta), and beyond that the
 * nearest such band voxel within 4 voxels plus its own distance; sites with
 * no band voxel within 4 voxels keep their phase. The new phase is
 * phi' = -tanh(beta (Phi - delta)) (Eq. lb-dist-to-phase); with apply != 0
 * the component populations of the changed sites become w_q Na', w_q Nb' at
 * rest with Na' + Nb' equal to the site's current Na + Nb (the momentum
 * populations are left alone). *before / *after (may be NULL) receive the
 * number of sites with phi > 0 before and after. |delta| <= 3.
 * Errors: LBPM_E_INVALID, LBPM_E_STATE (no fluids), LBPM_E_OOM, LBPM_E_CUDA. */
lbpm_status lbpm_morph(lbpm_ctx* ctx, double delta, int apply, long long* before, long long* after);

/* Shell aggregation protocol (Sec. 3.3): change the volume of fluid A by the
 * factor target_ratio (> 1 grows it). Each round applies a dummy growth of
 * one voxel (not kept) to measure the volume response, rescales delta
 * linearly to the volume still missing, applies it, and relaxes the state by
 * relax_steps (even) LB steps; rounds stop once the measured volume ratio
 * reaches the target, or after max_rounds. *achieved (may be NULL) receives
 * the final ratio of A sites to those at the start, *rounds the rounds run. */
lbpm_status lbpm_shell_aggregation(lbpm_ctx* ctx, double target_ratio, long long relax_steps, int max_rounds,
                                   double* achieved, int* rounds);

/* ------------------------------------------------------------------------
 * Image preparation (Sec. 4.2 mixing region; Sec. 3.3 mixed-wet relabel).
 * Both run CUDA kernels on `device` on a copy of the caller's host image,
 * through cudaMalloc/cudaFree and the legacy default stream (they synchronise
 * before returning), and write the result back into the caller's buffer.
 * Voxel arrays are x-fastest, nx*ny*nz entries. Errors: LBPM_E_INVALID (NULL
 * buffer, bad sizes or arguments), LBPM_E_OOM, LBPM_E_CUDA; the host image is
 * unchanged on error.
 * ------------------------------------------------------------------------ */

/* Mixing region at the two faces of `axis` (0 = x, 1 = y, 2 = z), n_mix
 * voxel layers deep (Sec. 4.2): a solid voxel in the first n_mix layers
 * becomes pore (label 0) where the voxel on the same line in the last layer
 * (the outlet face) is pore, and a solid voxel in the last n_mix layers
 * becomes pore where the voxel on its line in the first layer (the inlet
 * face) is pore. Other voxels keep their labels. 1 <= n_mix <= extent / 2. */
lbpm_status lbpm_mixing_layer(int device, uint16_t* labels, int nx, int ny, int nz, int axis, int n_mix);

/* Mixed-wet relabel (Sec. 3.3): every solid voxel (label != 0) whose centre
 * lies within Euclidean distance `radius` of the centre of an oil voxel
 * (oil[v] != 0) gets label new_label; distances wrap on the periodic axes.
 * The paper computes a distance transform of the oil phase and relabels the
 * solid within 2 voxel units; only "distance <= radius" matters, so the kernel
 * tests the voxel offsets of that ball (33 offsets besides the centre at
 * radius 2). 0 < radius <= 8, new_label >= 1. */
lbpm_status lbpm_mixed_wet_relabel(int device, uint16_t* labels, const uint8_t* oil, int nx, int ny, int nz,
                                   const int periodic[3], double radius, int new_label);

/* Number of kernel launches issued by this ctx since creation. */
lbpm_status lbpm_launch_count(const lbpm_ctx* ctx, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* LBPM_H */
