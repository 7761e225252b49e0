// C ABI of the library (declared in include/lbpm.h): context, memory, image
// loading and indexing, parameters, time stepping, measures and exchange.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include <new>

#include "internal.h"

using namespace lbm;

namespace {

thread_local std::string g_create_error;

constexpr unsigned long long kSnapMagic = 0x4d50424c4c4f4332ull;  // snapshot header tag

struct SnapHeader {
    unsigned long long magic;
    long long n_sites;
    long long step;
    long long reserved;
};

lbpm_status fail(lbpm_ctx* c, lbpm_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

lbpm_status fail_cuda(lbpm_ctx* c, const char* what, cudaError_t e) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return fail(c, e == cudaErrorMemoryAllocation ? LBPM_E_OOM : LBPM_E_CUDA, buf);
}

#define LBPM_CK(c, call)                                    \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return fail_cuda(c, #call, e_); \
    } while (0)

#define LBPM_ALLOC(c, ptr, type, count)                                                     \
    do {                                                                                    \
        (ptr) = static_cast<type*>(dalloc((c), sizeof(type) * static_cast<size_t>(count))); \
        if (!(ptr) && (count) > 0)                                                          \
            return fail((c), LBPM_E_OOM, "device allocation of " #ptr " failed");           \
    } while (0)

lbpm_status enter(lbpm_ctx* c) {
    if (!c) return LBPM_E_INVALID;
    c->err.clear();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail_cuda(c, "cudaSetDevice", e);
    return LBPM_OK;
}

void drop_graphs(lbpm_ctx* c);

void free_state(lbpm_ctx* c) {
    drop_graphs(c);
    dfree(c, c->d_f);
    dfree(c, c->d_a);
    dfree(c, c->d_b);
    dfree(c, c->d_nsum);
    dfree(c, c->d_drho);
    dfree(c, c->d_phi_alt);
    dfree(c, c->d_rsum);
    dfree(c, c->d_acc);
    c->d_acc = nullptr;
    c->d_drho = nullptr;
    c->d_phi_alt = nullptr;
    c->d_rsum = nullptr;
    c->d_f = c->d_a = c->d_b = nullptr;
    c->d_nsum = nullptr;
    c->have_fluids = false;
}

void free_image(lbpm_ctx* c) {
    free_state(c);
    dfree(c, c->d_labels);
    dfree(c, c->d_site_vox);
    dfree(c, c->d_vsite);
    dfree(c, c->d_phi);
    dfree(c, c->d_halo_dst);
    dfree(c, c->d_halo_site);
    dfree(c, c->d_wall6);
    c->d_wall6 = nullptr;
    dfree(c, c->d_slab_site);
    dfree(c, c->d_slab_side);
    dfree(c, c->d_face_part);
    dfree(c, c->d_face_rho);
    c->d_face_part = nullptr;
    c->d_face_rho = nullptr;
    c->d_labels = nullptr;
    c->d_site_vox = c->d_vsite = c->d_halo_dst = c->d_halo_site = c->d_slab_site = nullptr;
    c->d_phi = nullptr;
    c->d_slab_side = nullptr;
    c->N = c->H = c->n_slab = 0;
    c->have_image = false;
}

size_t state_bytes(const lbpm_ctx* c, int q) {
    const size_t e = c->params.precision == LBPM_FP16 ? 2 : 4;
    return e * static_cast<size_t>(q) * static_cast<size_t>(c->N);
}

lbpm_status alloc_state(lbpm_ctx* c) {
    free_state(c);
    c->d_f = dalloc(c, state_bytes(c, 19));
    c->d_a = dalloc(c, state_bytes(c, 7));
    c->d_b = dalloc(c, state_bytes(c, 7));
    c->d_nsum = static_cast<float*>(dalloc(c, sizeof(float) * c->N));
    c->d_acc = static_cast<unsigned long long*>(dalloc(c, sizeof(unsigned long long) * 2 * c->N));
    bool ok = c->d_f && c->d_a && c->d_b && c->d_nsum && c->d_acc;
    if (c->params.precision == LBPM_FP16) {
        // the second phase grid starts as a copy of the first (solids, walls
        // and their periodic mirrors are static and the same in both)
        c->d_drho = static_cast<float*>(dalloc(c, sizeof(float) * c->N));
        c->d_rsum = static_cast<float*>(dalloc(c, sizeof(float) * c->N));
        c->d_phi_alt = static_cast<float*>(dalloc(c, sizeof(float) * c->Vp));
        ok = ok && c->d_drho && c->d_rsum && c->d_phi_alt;
        if (ok && cudaMemcpyAsync(c->d_phi_alt, c->d_phi, sizeof(float) * c->Vp, cudaMemcpyDeviceToDevice,
                                  c->stream) != cudaSuccess)
            ok = false;
    }
    if (!ok) {
        free_state(c);
        return fail(c, LBPM_E_OOM, "device allocation of the distributions failed");
    }
    return LBPM_OK;
}

// halo list (periodic mirrors of pore voxels) and reservoir site list
lbpm_status build_boundaries(lbpm_ctx* c) {
    drop_graphs(c);
    dfree(c, c->d_halo_dst);
    dfree(c, c->d_halo_site);
    c->d_halo_dst = c->d_halo_site = nullptr;
    c->H = 0;
    LBPM_CK(c, launch_fill_halo(c, c->stream));
    int* flags;
    int* scan;
    LBPM_ALLOC(c, flags, int, c->Vp);
    scan = static_cast<int*>(dalloc(c, sizeof(int) * c->Vp));
    if (!scan) {
        dfree(c, flags);
        return fail(c, LBPM_E_OOM, "device allocation of the halo scan failed");
    }
    cudaError_t e = launch_halo_flags(c, flags, c->stream);
    if (e == cudaSuccess) e = exclusive_scan(c, flags, scan, c->Vp);
    int tail[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[0], scan + c->Vp - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[1], flags + c->Vp - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
        c->H = static_cast<long long>(tail[0]) + tail[1];
        if (c->H > 0) {
            c->d_halo_dst = static_cast<int*>(dalloc(c, sizeof(int) * c->H));
            c->d_halo_site = static_cast<int*>(dalloc(c, sizeof(int) * c->H));
            if (!c->d_halo_dst || !c->d_halo_site) e = cudaErrorMemoryAllocation;
            else e = launch_halo_scatter(c, flags, scan, c->stream);
        }
    }
    if (e == cudaSuccess && !c->d_wall6) {
        c->d_wall6 = static_cast<unsigned char*>(dalloc(c, c->N));
        if (!c->d_wall6) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = launch_wall_mask(c, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, flags);
    dfree(c, scan);
    if (e != cudaSuccess) return fail_cuda(c, "halo construction", e);

    // reservoir slabs / boundary faces
    dfree(c, c->d_slab_site);
    dfree(c, c->d_slab_side);
    c->d_slab_site = nullptr;
    c->d_slab_side = nullptr;
    c->n_slab = 0;
    if (c->params.reservoir_z == 3 && !c->d_face_part) {
        c->d_face_part = static_cast<double*>(dalloc(c, sizeof(double) * 2 * kFaceBlocks));
        c->d_face_rho = static_cast<float*>(dalloc(c, sizeof(float) * 2));
        if (!c->d_face_part || !c->d_face_rho) return fail(c, LBPM_E_OOM, "device allocation of the flux inlet failed");
    }
    if (c->params.reservoir_z) {
        LBPM_ALLOC(c, flags, int, c->N);
        scan = static_cast<int*>(dalloc(c, sizeof(int) * c->N));
        if (!scan) {
            dfree(c, flags);
            return fail(c, LBPM_E_OOM, "device allocation of the slab scan failed");
        }
        e = launch_slab_flags(c, flags, c->stream);
        if (e == cudaSuccess) e = exclusive_scan(c, flags, scan, c->N);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[0], scan + c->N - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[1], flags + c->N - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            c->n_slab = static_cast<long long>(tail[0]) + tail[1];
            if (c->n_slab > 0) {
                c->d_slab_site = static_cast<int*>(dalloc(c, sizeof(int) * c->n_slab));
                c->d_slab_side = static_cast<signed char*>(dalloc(c, c->n_slab));
                if (!c->d_slab_site || !c->d_slab_side) e = cudaErrorMemoryAllocation;
                else e = launch_slab_scatter(c, flags, scan, c->stream);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dfree(c, flags);
        dfree(c, scan);
        if (e != cudaSuccess) return fail_cuda(c, "reservoir construction", e);
    }
    return LBPM_OK;
}

lbpm_status check_params(lbpm_ctx* c, const lbpm_params* p) {
    if (!p) return fail(c, LBPM_E_INVALID, "params is NULL");
    if (!(p->tau_a > 0.5) || !(p->tau_b > 0.5) || !std::isfinite(p->tau_a) || !std::isfinite(p->tau_b))
        return fail(c, LBPM_E_INVALID, "tau_a and tau_b must be finite and > 0.5");
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha)) return fail(c, LBPM_E_INVALID, "alpha must be >= 0");
    if (!(p->beta >= 0.0) || !std::isfinite(p->beta)) return fail(c, LBPM_E_INVALID, "beta must be >= 0");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(p->force[a])) return fail(c, LBPM_E_INVALID, "force must be finite");
        if (p->periodic[a] != 0 && p->periodic[a] != 1) return fail(c, LBPM_E_INVALID, "periodic flags must be 0 or 1");
    }
    if (p->precision != LBPM_FP32 && p->precision != LBPM_FP16)
        return fail(c, LBPM_E_INVALID, "precision must be LBPM_FP32 or LBPM_FP16");
    if (p->reservoir_z < 0 || p->reservoir_z > 3) return fail(c, LBPM_E_INVALID, "reservoir_z must be 0, 1, 2 or 3");
    if (p->reservoir_z >= 2 && !(p->rho_in > 0.0 && p->rho_out > 0.0 && std::isfinite(p->rho_in) &&
                                 std::isfinite(p->rho_out)))
        return fail(c, LBPM_E_INVALID, "the pressure boundary needs finite rho_in, rho_out > 0");
    if (p->reservoir_z == 3 && !(p->flux_in >= 0.0 && std::isfinite(p->flux_in)))
        return fail(c, LBPM_E_INVALID, "the flux inlet needs a finite flux_in >= 0");
    if (p->reservoir_z && p->periodic[2]) return fail(c, LBPM_E_INVALID, "reservoirs need a non-periodic z axis");
    if (!(p->rho_in > 0.0) || !(p->rho_out > 0.0)) return fail(c, LBPM_E_INVALID, "rho_in and rho_out must be > 0");
    return LBPM_OK;
}

void drop_graphs(lbpm_ctx* c) {
    for (auto& g : c->graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    for (auto& g : c->sum_graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Kinds of timestep: the population form, and the first, middle and last
// step of a run of the sum form (see lbpm_set_step_form).
enum StepKind { kStepPop = 0, kStepSumFirst = 1, kStepSumMid = 2, kStepSumLast = 3 };

// The two kernels of one timestep of the given kind.
cudaError_t launch_step_phase(lbpm_ctx* c, int kind, int par, cudaStream_t s) {
    if (kind == kStepPop || kind == kStepSumFirst) return launch_phase(c, par, s);
    return launch_phase_sum(c, par, kind == kStepSumLast, s);
}
cudaError_t launch_step_collide(lbpm_ctx* c, int kind, int par, cudaStream_t s) {
    if (kind == kStepPop || kind == kStepSumLast) return launch_collide(c, par, s);
    return launch_collide_sum(c, par, kind == kStepSumMid, s);
}
// The boundary kernel after the collision of a step of the given kind (reservoir
// slabs, pressure faces); it writes what the next step (parity par ^ 1) reads.
cudaError_t launch_step_boundary(lbpm_ctx* c, int kind, int par, cudaStream_t s) {
    if (!c->n_slab) return cudaSuccess;
    if (kind == kStepPop || kind == kStepSumLast) return launch_reservoir(c, par ^ 1, s);
    return launch_reservoir_sum(c, par ^ 1, s);
}

// One timestep: phase pass, fused collide-stream, reservoir reset.
cudaError_t enqueue_step(lbpm_ctx* c, int par, cudaStream_t s) {
    cudaError_t e = launch_phase(c, par, s);
    if (e == cudaSuccess) e = launch_collide(c, par, s);
    if (e == cudaSuccess && c->n_slab) e = launch_reservoir(c, par ^ 1, s);
    return e;
}

int kernels_per_step(const lbpm_ctx* c) { return c->n_slab ? 3 : 2; }

// Whether lbpm_advance(nsteps) runs in the sum form.
bool use_sum_form(const lbpm_ctx* c, long long nsteps) { return nsteps >= 2 && sum_form_capable(c); }

// Capture `steps` (even) middle timesteps of the sum form, starting at an even step.
cudaError_t capture_sum_bundle(lbpm_ctx* c, int steps, cudaGraphExec_t* out) {
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = cudaSuccess;
    for (int k = 0; k < steps && el == cudaSuccess; ++k) {
        el = launch_step_phase(c, kStepSumMid, k & 1, c->cap_stream);
        if (el == cudaSuccess) el = launch_step_collide(c, kStepSumMid, k & 1, c->cap_stream);
        if (el == cudaSuccess) el = launch_step_boundary(c, kStepSumMid, k & 1, c->cap_stream);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Capture `steps` (even) timesteps starting at an even step into a graph.
cudaError_t capture_bundle(lbpm_ctx* c, int steps, cudaGraphExec_t* out) {
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = cudaSuccess;
    for (int k = 0; k < steps && el == cudaSuccess; ++k) el = enqueue_step(c, k & 1, c->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

int next_event(lbpm_ctx* c) {
    if (c->ev_next >= c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->ev_pool.push_back(e);
    }
    return static_cast<int>(c->ev_next++);
}

}  // namespace

namespace lbm {

bool sum_form_capable(const lbpm_ctx* c) {
    return c->step_form == LBPM_STEP_AUTO && c->params.reservoir_z <= 1 && c->d_acc != nullptr;
}

cudaError_t clear_sums(const lbpm_ctx* c, int par, cudaStream_t s) {
    return cudaMemsetAsync(c->d_acc + static_cast<size_t>(par) * static_cast<size_t>(c->N), 0,
                           sizeof(unsigned long long) * static_cast<size_t>(c->N), s);
}

void* dalloc(lbpm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->stream, c->alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back(Allocation{p, bytes});
    return p;
}

void dfree(lbpm_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i) {
        if (c->allocs[i].ptr == p) {
            c->allocs[i] = c->allocs.back();
            c->allocs.pop_back();
            break;
        }
    }
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
}

}  // namespace lbm

namespace lbm {

// Measures of Sec. 4 / Sec. 3.4 from the NSUM device sums of one domain.
void fill_measures(const lbpm_ctx* c, const double* S, lbpm_measures* out) {
    std::memset(out, 0, sizeof *out);
    const double N = static_cast<double>(c->N), V = static_cast<double>(c->V);
    const double cnt_a = S[3], cnt_b = N - S[3];
    out->step = c->step;
    out->n_sites = c->N;
    out->sat_mass = (S[0] + S[1]) > 0 ? S[0] / (S[0] + S[1]) : 0.0;
    out->sat_count = N > 0 ? cnt_a / N : 0.0;
    out->mass_a = S[0];
    out->mass_b = S[1];
    out->mass_total = S[2];
    for (int a = 0; a < 3; ++a) {
        out->flux[a] = S[4 + a] / V;
        out->flux_a[a] = S[7 + a] / V;
        out->flux_b[a] = S[10 + a] / V;
        out->mom_a[a] = S[15 + a];
        out->mom_b[a] = S[18 + a];
    }
    out->ke_a = S[21];
    out->ke_b = S[22];
    out->p_a = cnt_a > 0 ? S[23] / cnt_a : 0.0;
    out->p_b = cnt_b > 0 ? S[24] / cnt_b : 0.0;
    out->vol_a = cnt_a;
    out->vol_b = cnt_b;
    if (c->params.alpha > 0.0) {
        const double mu_a = (c->params.tau_a - 0.5) / 3.0, mu_b = (c->params.tau_b - 0.5) / 3.0;
        const double ua = S[13] > 0 ? std::sqrt(S[15] * S[15] + S[16] * S[16] + S[17] * S[17]) / S[13] : 0.0;
        const double ub = S[14] > 0 ? std::sqrt(S[18] * S[18] + S[19] * S[19] + S[20] * S[20]) / S[14] : 0.0;
        out->ca = ((cnt_a / V) * mu_a * ua + (cnt_b / V) * mu_b * ub) / (6.0 * c->params.alpha);
    }
    out->status = (S[25] > 0 ? 1 : 0) | (S[26] > 0 ? 2 : 0);
}

}  // namespace lbm

extern "C" {

const char* lbpm_version(void) { return "lbpm-gb300 0.1 (sm_103a)"; }

lbpm_status lbpm_create(lbpm_ctx** out, int device, void* cuda_stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return LBPM_E_INVALID;
    }
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        g_create_error = std::string("no CUDA device ") + std::to_string(device) +
                         (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
        cudaGetLastError();
        return e != cudaSuccess ? LBPM_E_CUDA : LBPM_E_INVALID;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        return LBPM_E_CUDA;
    }
    // set-up of the allocation-free field read on this device (its static
    // staging array is placed now, not inside a later call)
    e = lbm::noalloc_setup(device);
    if (e != cudaSuccess) {
        g_create_error = std::string("allocation-free read set-up: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return LBPM_E_CUDA;
    }
    lbpm_ctx* c = new (std::nothrow) lbpm_ctx();
    if (!c) return LBPM_E_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    lbpm_params& p = c->params;
    p.tau_a = p.tau_b = 1.0;
    p.alpha = 0.0;
    p.beta = 0.0;
    p.force[0] = p.force[1] = p.force[2] = 0.0;
    p.precision = LBPM_FP32;
    p.periodic[0] = p.periodic[1] = p.periodic[2] = 1;
    p.reservoir_z = 0;
    p.rho_in = p.rho_out = 1.0;
    *out = c;
    return LBPM_OK;
}

lbpm_status lbpm_destroy(lbpm_ctx* c) {
    if (!c) return LBPM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    while (!c->allocs.empty()) dfree(c, c->allocs.back().ptr);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return LBPM_OK;
}

lbpm_status lbpm_set_allocator(lbpm_ctx* c, lbpm_alloc_fn alloc, lbpm_free_fn free_fn, void* user) {
    if (!c) return LBPM_E_INVALID;
    if (!c->allocs.empty()) return fail(c, LBPM_E_STATE, "set the allocator before loading an image");
    if (alloc && !free_fn) return fail(c, LBPM_E_INVALID, "an allocator needs a free function");
    c->alloc = alloc;
    c->free_fn = alloc ? free_fn : nullptr;
    c->alloc_user = user;
    return LBPM_OK;
}

const char* lbpm_last_error(const lbpm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

lbpm_status lbpm_set_params(lbpm_ctx* c, const lbpm_params* p) {
    lbpm_status s = enter(c);
    if (s) return s;
    if ((s = check_params(c, p))) return s;
    const lbpm_params old = c->params;
    c->params = *p;
    drop_graphs(c);
    if (!c->have_image) return LBPM_OK;
    const bool per_changed = std::memcmp(old.periodic, p->periodic, sizeof old.periodic) != 0;
    if (per_changed || old.reservoir_z != p->reservoir_z) {
        if ((s = build_boundaries(c))) return s;
        if (per_changed) c->have_fluids = false;
    }
    if (old.precision != p->precision) {
        if ((s = alloc_state(c))) return s;
    }
    return LBPM_OK;
}

lbpm_status lbpm_load_image(lbpm_ctx* c, const uint16_t* labels, int nx, int ny, int nz) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!labels) return fail(c, LBPM_E_INVALID, "labels is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(c, LBPM_E_INVALID, "dimensions must be >= 1");
    const long long px = nx + 2LL, py = ny + 2LL, pz = nz + 2LL;
    if (px * py * pz >= (1LL << 31)) return fail(c, LBPM_E_INVALID, "padded image must hold < 2^31 voxels");
    if (c->params.reservoir_z && c->params.periodic[2])
        return fail(c, LBPM_E_INVALID, "reservoirs need a non-periodic z axis");
    free_image(c);
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->px = static_cast<int>(px);
    c->py = static_cast<int>(py);
    c->pz = static_cast<int>(pz);
    c->V = static_cast<long long>(nx) * ny * nz;
    c->Vp = px * py * pz;
    LBPM_ALLOC(c, c->d_labels, uint16_t, c->V);
    LBPM_CK(c, cudaMemcpyAsync(c->d_labels, labels, sizeof(uint16_t) * c->V, cudaMemcpyHostToDevice, c->stream));
    int* flags;
    LBPM_ALLOC(c, flags, int, c->V);
    int* scan = static_cast<int*>(dalloc(c, sizeof(int) * c->V));
    if (!scan) {
        dfree(c, flags);
        return fail(c, LBPM_E_OOM, "device allocation of the pore scan failed");
    }
    int tail[2] = {0, 0};
    cudaError_t e = launch_flag_pore(c->d_labels, c->V, flags, c->stream);
    if (e == cudaSuccess) e = exclusive_scan(c, flags, scan, c->V);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[0], scan + c->V - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tail[1], flags + c->V - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dfree(c, flags);
        dfree(c, scan);
        return fail_cuda(c, "pore compaction", e);
    }
    c->N = static_cast<long long>(tail[0]) + tail[1];
    if (c->N == 0) {
        dfree(c, flags);
        dfree(c, scan);
        return fail(c, LBPM_E_INVALID, "the image has no pore voxel (label 0)");
    }
    c->d_site_vox = static_cast<int*>(dalloc(c, sizeof(int) * c->N));
    c->d_vsite = static_cast<int*>(dalloc(c, sizeof(int) * c->Vp));
    c->d_phi = static_cast<float*>(dalloc(c, sizeof(float) * c->Vp));
    if (!c->d_site_vox || !c->d_vsite || !c->d_phi) {
        dfree(c, flags);
        dfree(c, scan);
        return fail(c, LBPM_E_OOM, "device allocation of the index failed");
    }
    e = launch_scatter_sites(c, scan, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, flags);
    dfree(c, scan);
    if (e != cudaSuccess) return fail_cuda(c, "site scatter", e);
    c->have_image = true;
    if ((s = build_boundaries(c))) return s;
    if ((s = alloc_state(c))) return s;
    c->step = 0;
    c->launches += 6;
    return LBPM_OK;
}

lbpm_status lbpm_set_affinity_table(lbpm_ctx* c, const float* table, int n_labels) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!c->have_image) return fail(c, LBPM_E_STATE, "load an image first");
    if (!table || n_labels < 1 || n_labels > 65536) return fail(c, LBPM_E_INVALID, "bad affinity table");
    for (int k = 1; k < n_labels; ++k)
        if (!(std::fabs(table[k]) <= 1.0f)) return fail(c, LBPM_E_INVALID, "affinities must lie in [-1, 1]");
    float* d_t;
    LBPM_ALLOC(c, d_t, float, n_labels);
    cudaError_t e = cudaMemcpyAsync(d_t, table, sizeof(float) * n_labels, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_affinity_table(c, d_t, n_labels, c->stream);
    if (e == cudaSuccess) e = launch_fill_halo(c, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_t);
    if (e != cudaSuccess) return fail_cuda(c, "affinity table", e);
    c->launches += 2;
    return LBPM_OK;
}

lbpm_status lbpm_set_affinity_map(lbpm_ctx* c, const float* map) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!c->have_image) return fail(c, LBPM_E_STATE, "load an image first");
    if (!map) return fail(c, LBPM_E_INVALID, "affinity map is NULL");
    float* d_m;
    LBPM_ALLOC(c, d_m, float, c->V);
    cudaError_t e = cudaMemcpyAsync(d_m, map, sizeof(float) * c->V, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_affinity_map(c, d_m, c->stream);
    if (e == cudaSuccess) e = launch_fill_halo(c, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_m);
    if (e != cudaSuccess) return fail_cuda(c, "affinity map", e);
    c->launches += 2;
    return LBPM_OK;
}

lbpm_status lbpm_init_fluids(lbpm_ctx* c, const float* phi0) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!c->have_image) return fail(c, LBPM_E_STATE, "load an image first");
    if (!phi0) return fail(c, LBPM_E_INVALID, "phi0 is NULL");
    float* d_p;
    LBPM_ALLOC(c, d_p, float, c->V);
    cudaError_t e = cudaMemcpyAsync(d_p, phi0, sizeof(float) * c->V, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_init_fluids(c, d_p, c->stream);
    if (e == cudaSuccess) e = launch_reservoir(c, 0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_p);
    if (e != cudaSuccess) return fail_cuda(c, "fluid initialisation", e);
    c->step = 0;
    c->have_fluids = true;
    c->unstable = false;
    c->launches += c->params.precision == LBPM_FP16 ? 5 : 2;
    return LBPM_OK;
}

}  // extern "C"

namespace {

// One plain timestep of the given kind, with CUDA events around its two
// kernels when kernel timing is on.
lbpm_status plain_step(lbpm_ctx* c, int kind) {
    const int par = static_cast<int>(c->step & 1);
    int e0 = -1, e1 = -1, e2 = -1, e3 = -1;
    if (c->timing) {
        e0 = next_event(c);
        e1 = next_event(c);
        e2 = next_event(c);
        e3 = next_event(c);
    }
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], c->stream);
    LBPM_CK(c, launch_step_phase(c, kind, par, c->stream));
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], c->stream);
    if (e2 >= 0) cudaEventRecord(c->ev_pool[e2], c->stream);
    LBPM_CK(c, launch_step_collide(c, kind, par, c->stream));
    if (e3 >= 0) cudaEventRecord(c->ev_pool[e3], c->stream);
    if (e0 >= 0 && e1 >= 0) c->ev_phase.emplace_back(e0, e1);
    if (e2 >= 0 && e3 >= 0) c->ev_collide.emplace_back(e2, e3);
    c->launches += 2;
    if (c->n_slab) {
        LBPM_CK(c, launch_step_boundary(c, kind, par, c->stream));
        c->launches += 1;
    }
    c->step += 1;
    return LBPM_OK;
}

// lbpm_advance in the sum form (nsteps >= 2, no reservoirs): the first step
// reads the populations, the middle steps carry the components as per-site
// sums (replayed from CUDA graphs in bundles of 16 and 2), the last step
// writes the populations again.
lbpm_status advance_sum(lbpm_ctx* c, long long nsteps) {
    LBPM_CK(c, clear_sums(c, static_cast<int>((c->step + 1) & 1), c->stream));
    lbpm_status st = plain_step(c, kStepSumFirst);
    if (st) return st;
    long long mid = nsteps - 2;
    if (!c->timing && c->use_graphs) {
        if ((c->step & 1) && mid > 0) {
            if ((st = plain_step(c, kStepSumMid))) return st;
            --mid;
        }
        const int sizes[2] = {2, 16};
        for (int gi = 1; gi >= 0; --gi) {
            while (mid >= sizes[gi]) {
                if (!c->sum_graphs[gi]) LBPM_CK(c, capture_sum_bundle(c, sizes[gi], &c->sum_graphs[gi]));
                LBPM_CK(c, cudaGraphLaunch(c->sum_graphs[gi], c->stream));
                c->launches += static_cast<long long>(kernels_per_step(c)) * sizes[gi];
                c->step += sizes[gi];
                mid -= sizes[gi];
            }
        }
    }
    for (; mid > 0; --mid)
        if ((st = plain_step(c, kStepSumMid))) return st;
    return plain_step(c, kStepSumLast);
}

}  // namespace

extern "C" {

lbpm_status lbpm_set_step_form(lbpm_ctx* c, int form) {
    if (!c) return LBPM_E_INVALID;
    c->err.clear();
    if (form != LBPM_STEP_AUTO && form != LBPM_STEP_POPULATIONS) return fail(c, LBPM_E_INVALID, "unknown step form");
    c->step_form = form;
    return LBPM_OK;
}

lbpm_status lbpm_advance(lbpm_ctx* c, long long nsteps) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (nsteps < 0) return fail(c, LBPM_E_INVALID, "nsteps must be >= 0");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    if (c->unstable) return fail(c, LBPM_E_UNSTABLE, "the state was flagged unstable; re-initialise or restore");
    if (use_sum_form(c, nsteps)) return advance_sum(c, nsteps);
    long long k = 0;
    if (!c->timing && c->use_graphs) {
        // an odd start takes one plain step, then whole bundles run as graphs
        if ((c->step & 1) && nsteps > 0) {
            LBPM_CK(c, enqueue_step(c, 1, c->stream));
            c->launches += kernels_per_step(c);
            c->step += 1;
            k = 1;
        }
        const int sizes[2] = {2, 16};
        for (int gi = 1; gi >= 0; --gi) {
            while (nsteps - k >= sizes[gi]) {
                if (!c->graphs[gi]) LBPM_CK(c, capture_bundle(c, sizes[gi], &c->graphs[gi]));
                LBPM_CK(c, cudaGraphLaunch(c->graphs[gi], c->stream));
                c->launches += static_cast<long long>(sizes[gi]) * kernels_per_step(c);
                c->step += sizes[gi];
                k += sizes[gi];
            }
        }
    }
    for (; k < nsteps; ++k) {
        const int par = static_cast<int>(c->step & 1);
        int e0 = -1, e1 = -1, e2 = -1, e3 = -1;
        if (c->timing) {
            e0 = next_event(c);
            e1 = next_event(c);
            e2 = next_event(c);
            e3 = next_event(c);
        }
        if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], c->stream);
        LBPM_CK(c, launch_phase(c, par, c->stream));
        if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], c->stream);
        if (e2 >= 0) cudaEventRecord(c->ev_pool[e2], c->stream);
        LBPM_CK(c, launch_collide(c, par, c->stream));
        if (e3 >= 0) cudaEventRecord(c->ev_pool[e3], c->stream);
        if (e0 >= 0 && e1 >= 0) c->ev_phase.emplace_back(e0, e1);
        if (e2 >= 0 && e3 >= 0) c->ev_collide.emplace_back(e2, e3);
        c->launches += 2;
        if (c->n_slab) {
            LBPM_CK(c, launch_reservoir(c, par ^ 1, c->stream));
            c->launches += 1;
        }
        c->step += 1;
    }
    return LBPM_OK;
}

lbpm_status lbpm_sync(lbpm_ctx* c) {
    lbpm_status s = enter(c);
    if (s) return s;
    LBPM_CK(c, cudaStreamSynchronize(c->stream));
    LBPM_CK(c, cudaGetLastError());
    return LBPM_OK;
}

lbpm_status lbpm_measure(lbpm_ctx* c, lbpm_measures* out) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!out) return fail(c, LBPM_E_INVALID, "out is NULL");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    double* d_out;
    LBPM_ALLOC(c, d_out, double, NSUM);
    double S[NSUM];
    cudaError_t e = launch_measure(c, static_cast<int>(c->step & 1), d_out, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S, d_out, sizeof S, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_out);
    if (e != cudaSuccess) return fail_cuda(c, "measure", e);
    c->launches += 2;
    fill_measures(c, S, out);
    if (out->status) {
        c->unstable = true;
        return fail(c, LBPM_E_UNSTABLE, "non-finite or negative densities in the state");
    }
    return LBPM_OK;
}

lbpm_status lbpm_read_field(lbpm_ctx* c, int which, float* out) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!out) return fail(c, LBPM_E_INVALID, "out is NULL");
    if (which < LBPM_FIELD_PHI || which > LBPM_FIELD_RHO) return fail(c, LBPM_E_INVALID, "unknown field");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    float* d;
    LBPM_ALLOC(c, d, float, c->V);
    cudaError_t e = launch_field(c, static_cast<int>(c->step & 1), which, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(float) * c->V, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d);
    if (e != cudaSuccess) return fail_cuda(c, "read_field", e);
    c->launches += 2;
    return LBPM_OK;
}

lbpm_status lbpm_read_distributions(lbpm_ctx* c, int which, float* out) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!out) return fail(c, LBPM_E_INVALID, "out is NULL");
    if (which < LBPM_DIST_F || which > LBPM_DIST_B) return fail(c, LBPM_E_INVALID, "unknown distribution");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    const long long count = (which == LBPM_DIST_F ? 19 : 7) * c->N;
    float* d;
    LBPM_ALLOC(c, d, float, count);
    cudaError_t e = launch_export_dist(c, static_cast<int>(c->step & 1), which, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(float) * count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d);
    if (e != cudaSuccess) return fail_cuda(c, "read_distributions", e);
    c->launches += 1;
    return LBPM_OK;
}

lbpm_status lbpm_read_box(lbpm_ctx* c, int which, const int* lo, const int* hi, float* out) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!lo || !hi || !out) return fail(c, LBPM_E_INVALID, "lo, hi and out must not be NULL");
    if (which < LBPM_DIST_F || which > LBPM_DIST_B) return fail(c, LBPM_E_INVALID, "unknown distribution");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    const int dims[3] = {c->nx, c->ny, c->nz};
    long long nbox = 1;
    for (int a = 0; a < 3; ++a) {
        if (lo[a] < 0 || hi[a] > dims[a] || lo[a] >= hi[a]) return fail(c, LBPM_E_INVALID, "box outside the image or empty");
        nbox *= hi[a] - lo[a];
    }
    const long long count = (which == LBPM_DIST_F ? 19 : 7) * nbox;
    float* d;
    LBPM_ALLOC(c, d, float, count);
    cudaError_t e = launch_read_box(c, static_cast<int>(c->step & 1), which, lo, hi, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(float) * count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d);
    if (e != cudaSuccess) return fail_cuda(c, "read_box", e);
    c->launches += 1;
    return LBPM_OK;
}

lbpm_status lbpm_write_distributions(lbpm_ctx* c, int which, const float* in) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!in) return fail(c, LBPM_E_INVALID, "input is NULL");
    if (which < LBPM_DIST_F || which > LBPM_DIST_B) return fail(c, LBPM_E_INVALID, "unknown distribution");
    if (!c->have_image || !c->d_f) return fail(c, LBPM_E_STATE, "load an image first");
    const long long count = (which == LBPM_DIST_F ? 19 : 7) * c->N;
    float* d;
    LBPM_ALLOC(c, d, float, count);
    cudaError_t e = cudaMemcpyAsync(d, in, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_import_dist(c, static_cast<int>(c->step & 1), which, d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d);
    if (e != cudaSuccess) return fail_cuda(c, "write_distributions", e);
    c->have_fluids = true;
    c->launches += 1;
    return LBPM_OK;
}

lbpm_status lbpm_num_sites(const lbpm_ctx* c, long long* n) {
    if (!c || !n) return LBPM_E_INVALID;
    *n = c->N;
    return LBPM_OK;
}

lbpm_status lbpm_step_count(const lbpm_ctx* c, long long* step) {
    if (!c || !step) return LBPM_E_INVALID;
    *step = c->step;
    return LBPM_OK;
}

lbpm_status lbpm_get_index(lbpm_ctx* c, int64_t* site2vox, int32_t* nbr) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!c->have_image) return fail(c, LBPM_E_STATE, "load an image first");
    long long* d_s = nullptr;
    int* d_n = nullptr;
    if (site2vox) LBPM_ALLOC(c, d_s, long long, c->N);
    if (nbr) {
        d_n = static_cast<int*>(dalloc(c, sizeof(int) * 18 * c->N));
        if (!d_n) {
            dfree(c, d_s);
            return fail(c, LBPM_E_OOM, "device allocation of the neighbour table failed");
        }
    }
    cudaError_t e = launch_export_index(c, d_s, d_n, c->stream);
    if (e == cudaSuccess && site2vox)
        e = cudaMemcpyAsync(site2vox, d_s, sizeof(long long) * c->N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && nbr)
        e = cudaMemcpyAsync(nbr, d_n, sizeof(int) * 18 * c->N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_s);
    dfree(c, d_n);
    if (e != cudaSuccess) return fail_cuda(c, "get_index", e);
    c->launches += 1;
    return LBPM_OK;
}

lbpm_status lbpm_snapshot(lbpm_ctx* c, void* host_buf, size_t* bytes) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!bytes) return fail(c, LBPM_E_INVALID, "bytes is NULL");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    const size_t need = sizeof(SnapHeader) + sizeof(float) * 33 * static_cast<size_t>(c->N);
    if (!host_buf) {
        *bytes = need;
        return LBPM_OK;
    }
    if (*bytes < need) return fail(c, LBPM_E_INVALID, "snapshot buffer too small");
    SnapHeader h{kSnapMagic, c->N, c->step, 0};
    std::memcpy(host_buf, &h, sizeof h);
    float* p = reinterpret_cast<float*>(static_cast<char*>(host_buf) + sizeof h);
    if ((s = lbpm_read_distributions(c, LBPM_DIST_F, p))) return s;
    if ((s = lbpm_read_distributions(c, LBPM_DIST_A, p + 19 * c->N))) return s;
    if ((s = lbpm_read_distributions(c, LBPM_DIST_B, p + 26 * c->N))) return s;
    *bytes = need;
    return LBPM_OK;
}

lbpm_status lbpm_restore(lbpm_ctx* c, const void* host_buf, size_t bytes) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!host_buf) return fail(c, LBPM_E_INVALID, "snapshot is NULL");
    if (!c->have_image) return fail(c, LBPM_E_STATE, "load the image of the snapshot first");
    SnapHeader h;
    if (bytes < sizeof h) return fail(c, LBPM_E_INVALID, "snapshot too short");
    std::memcpy(&h, host_buf, sizeof h);
    if (h.magic != kSnapMagic) return fail(c, LBPM_E_INVALID, "not a snapshot of this library");
    if (h.n_sites != c->N) return fail(c, LBPM_E_INVALID, "snapshot was taken on another image");
    if (h.step < 0) return fail(c, LBPM_E_INVALID, "corrupt snapshot step");
    if (bytes != sizeof h + sizeof(float) * 33 * static_cast<size_t>(c->N))
        return fail(c, LBPM_E_INVALID, "snapshot size does not match the image");
    const float* p = reinterpret_cast<const float*>(static_cast<const char*>(host_buf) + sizeof h);
    c->step = h.step;
    if ((s = lbpm_write_distributions(c, LBPM_DIST_F, p))) return s;
    if ((s = lbpm_write_distributions(c, LBPM_DIST_A, p + 19 * c->N))) return s;
    if ((s = lbpm_write_distributions(c, LBPM_DIST_B, p + 26 * c->N))) return s;
    c->have_fluids = true;
    c->unstable = false;
    return LBPM_OK;
}

namespace {
constexpr int kMorphRadius = 4;   // far-field search radius of the distance map (voxels)
}

lbpm_status lbpm_morph(lbpm_ctx* c, double delta, int apply, long long* before, long long* after) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!(std::fabs(delta) <= 3.0)) return fail(c, LBPM_E_INVALID, "|delta| must be <= 3 voxels");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    if (!(c->params.beta > 0.0)) return fail(c, LBPM_E_INVALID, "the distance map needs beta > 0");
    // ball offsets of the far-field search and their lengths
    std::vector<int3> off;
    std::vector<float> len;
    std::vector<long long> lin;
    for (int z = -kMorphRadius; z <= kMorphRadius; ++z)
        for (int y = -kMorphRadius; y <= kMorphRadius; ++y)
            for (int x = -kMorphRadius; x <= kMorphRadius; ++x) {
                const int r2 = x * x + y * y + z * z;
                if (r2 == 0 || r2 > kMorphRadius * kMorphRadius) continue;
                off.push_back(make_int3(x, y, z));
                len.push_back(static_cast<float>(std::sqrt(static_cast<double>(r2))));
                lin.push_back(x + static_cast<long long>(c->nx) * (y + static_cast<long long>(c->ny) * z));
            }
    float *d_phi, *d_dist, *d_ntot, *d_len;
    int3* d_off;
    long long* d_lin;
    unsigned long long* d_cnt;
    LBPM_ALLOC(c, d_phi, float, c->V);
    d_dist = static_cast<float*>(dalloc(c, sizeof(float) * c->V));
    d_ntot = static_cast<float*>(dalloc(c, sizeof(float) * std::max<long long>(c->N, 1)));
    d_len = static_cast<float*>(dalloc(c, sizeof(float) * len.size()));
    d_off = static_cast<int3*>(dalloc(c, sizeof(int3) * off.size()));
    d_lin = static_cast<long long*>(dalloc(c, sizeof(long long) * lin.size()));
    d_cnt = static_cast<unsigned long long*>(dalloc(c, 2 * sizeof(unsigned long long)));
    unsigned long long cnt[2] = {0, 0};
    cudaError_t e = (d_dist && d_ntot && d_len && d_off && d_lin && d_cnt) ? cudaSuccess : cudaErrorMemoryAllocation;
    // voxels without a site: NaN distance (fminf ignores it)
    if (e == cudaSuccess) e = cudaMemsetAsync(d_dist, 0xff, sizeof(float) * c->V, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, off.data(), sizeof(int3) * off.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_len, len.data(), sizeof(float) * len.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lin, lin.data(), sizeof(long long) * lin.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_morph(c, static_cast<int>(c->step & 1), static_cast<float>(delta), kMorphRadius, apply != 0,
                         d_phi, d_dist, d_ntot, d_off, d_lin, d_len, static_cast<int>(off.size()), d_cnt, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    for (void* p : {static_cast<void*>(d_phi), static_cast<void*>(d_dist), static_cast<void*>(d_ntot),
                    static_cast<void*>(d_len), static_cast<void*>(d_off), static_cast<void*>(d_lin),
                    static_cast<void*>(d_cnt)})
        dfree(c, p);
    if (e != cudaSuccess) return fail_cuda(c, "morph", e);
    c->launches += 2;
    if (before) *before = static_cast<long long>(cnt[0]);
    if (after) *after = static_cast<long long>(cnt[1]);
    return LBPM_OK;
}

lbpm_status lbpm_shell_aggregation(lbpm_ctx* c, double target_ratio, long long relax_steps, int max_rounds,
                                   double* achieved, int* rounds) {
    lbpm_status s = enter(c);
    if (s) return s;
    if (!(target_ratio > 0.0) || !std::isfinite(target_ratio) || relax_steps < 0 || max_rounds < 1)
        return fail(c, LBPM_E_INVALID, "bad shell aggregation settings");
    long long v0 = 0, cur = 0, v1 = 0;
    if ((s = lbpm_morph(c, 0.0, 0, &v0, nullptr))) return s;
    if (v0 == 0) return fail(c, LBPM_E_STATE, "fluid A occupies no site");
    const double goal = target_ratio * static_cast<double>(v0);
    const double sgn = target_ratio >= 1.0 ? 1.0 : -1.0;
    cur = v0;
    int r = 0;
    while (r < max_rounds && (sgn > 0 ? cur < goal : cur > goal)) {
        ++r;
        // dummy growth of one voxel, not kept: the volume response
        if ((s = lbpm_morph(c, sgn, 0, &cur, &v1))) return s;
        if (v1 == cur) break;   // no interface left to move
        double delta = sgn * std::fabs(goal - static_cast<double>(cur)) / std::fabs(static_cast<double>(v1 - cur));
        delta = std::max(-3.0, std::min(3.0, delta));
        if ((s = lbpm_morph(c, delta, 1, nullptr, nullptr))) return s;
        if (relax_steps > 0 && (s = lbpm_advance(c, relax_steps))) return s;
        if ((s = lbpm_morph(c, 0.0, 0, &cur, nullptr))) return s;
    }
    if (achieved) *achieved = static_cast<double>(cur) / static_cast<double>(v0);
    if (rounds) *rounds = r;
    return LBPM_OK;
}

lbpm_status lbpm_enable_kernel_timing(lbpm_ctx* c, int enable) {
    if (!c) return LBPM_E_INVALID;
    c->timing = enable != 0;
    return LBPM_OK;
}

lbpm_status lbpm_kernel_timing(lbpm_ctx* c, double* ms_collide, long long* n_collide, double* ms_phase,
                               long long* n_phase) {
    lbpm_status s = enter(c);
    if (s) return s;
    LBPM_CK(c, cudaStreamSynchronize(c->stream));
    double tc = 0.0, tp = 0.0;
    for (auto& pr : c->ev_collide) {
        float ms = 0.0f;
        LBPM_CK(c, cudaEventElapsedTime(&ms, c->ev_pool[pr.first], c->ev_pool[pr.second]));
        tc += ms;
    }
    for (auto& pr : c->ev_phase) {
        float ms = 0.0f;
        LBPM_CK(c, cudaEventElapsedTime(&ms, c->ev_pool[pr.first], c->ev_pool[pr.second]));
        tp += ms;
    }
    if (ms_collide) *ms_collide = tc;
    if (n_collide) *n_collide = static_cast<long long>(c->ev_collide.size());
    if (ms_phase) *ms_phase = tp;
    if (n_phase) *n_phase = static_cast<long long>(c->ev_phase.size());
    c->ev_collide.clear();
    c->ev_phase.clear();
    c->ev_next = 0;
    return LBPM_OK;
}

lbpm_status lbpm_launch_count(const lbpm_ctx* c, long long* launches) {
    if (!c || !launches) return LBPM_E_INVALID;
    *launches = c->launches;
    return LBPM_OK;
}

}  // extern "C"
