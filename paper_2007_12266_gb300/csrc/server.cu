// Serving loop: continuous batching of simulation jobs on one GPU.
//
// The protocols of Sec. 4 run as job kinds:
//   steady state  (Sec. 4.2): periodic flow driven by a body force at fixed
//                 saturation, until the Darcy flux settles;
//   unsteady      (Sec. 4.1): inlet / outlet reservoirs displace one fluid by
//                 the other, until the flux settles;
//   centrifuge    (Sec. 4.1, centrifuge paragraph): the body force is raised
//                 by a factor each time the saturation reaches a plateau, up to
//                 a cap, until the flux settles at the cap.
// Convergence: |q(t) - q(t - interval)| / |q(t)| < tol on the Darcy flux along
// the force (standing in for the capillary-number change of Eq. convergence),
// checked every `interval` steps, or a step ceiling.
//
// The caller drives the server: lbpm_server_run performs one round - admit
// queued jobs while a slot and the device-memory budget allow (first come,
// first served), advance every running job by one interval in ONE batched
// launch sequence, measure them all, apply the protocol rules, retire the
// finished ones. Jobs admitted in a round join the running batch at once
// (continuous batching); finished jobs keep their device state until
// released, so results can be read back later, or until their memory is
// needed to admit a queued job (the oldest finished job is evicted first; its
// status and last measures stay available).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// The paper caps each body-force rescale at a factor of two (Sec. 4.2).
constexpr double kMaxForceRescale = 2.0;

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Job {
    long long ticket = 0;
    lbpm_job_spec spec{};
    std::vector<uint16_t> labels;
    std::vector<float> affinity, phi0;
    long long n_pore = 0;
    size_t footprint = 0;
    int state = LBPM_JOB_QUEUED;
    lbpm_ctx* ctx = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
    long long steps = 0;
    double q_prev = 0, sw_prev = 0;
    bool have_prev = false;
    int force_raises = 0;
    long long since_rescale = 0;
    lbpm_measures last{};
    std::string note;
};

}  // namespace

struct lbpm_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    int max_jobs = 0;
    int interval = 500;
    std::string err;
    lbpm_alloc_fn alloc = nullptr;
    lbpm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    lbpm_batch* batch = nullptr;
    long long next_ticket = 1;
    std::deque<Job*> queue;
    std::vector<Job*> running;
    std::map<long long, std::unique_ptr<Job>> jobs;
    long long site_updates = 0;
    std::deque<Job*> finished;   // retired jobs still holding device state, oldest first
};

namespace {

lbpm_status sfail(lbpm_server* s, lbpm_status st, const std::string& m) {
    if (s) s->err = m;
    return st;
}

// Device bytes of a job: state, index grids and the transient scans of the
// indexer (the peak while the image is loaded).
size_t estimate_footprint(const lbpm_job_spec& sp, long long n_pore) {
    const double V = static_cast<double>(sp.nx) * sp.ny * sp.nz;
    const double Vp = (sp.nx + 2.0) * (sp.ny + 2.0) * (sp.nz + 2.0);
    const double N = static_cast<double>(n_pore);
    const double es = sp.params.precision == LBPM_FP16 ? 2.0 : 4.0;
    const bool h = sp.params.precision == LBPM_FP16;
    // populations, nsum (+ drho, rsum and the second phase grid with fp16 storage)
    const double state = 33.0 * es * N + (h ? 12.0 : 4.0) * N + (h ? 4.0 * Vp : 0.0);
    // labels, vsite, phi, site_vox, wall mask
    const double grids = 2.0 * V + 8.0 * Vp + 5.0 * N;
    const double transient = 8.0 * Vp;
    return static_cast<size_t>(state + grids + transient + (1 << 20));
}

lbpm_status build_job(lbpm_server* s, Job* j) {
    lbpm_ctx* c = nullptr;
    lbpm_status st = lbpm_create(&c, s->device, s->stream);
    if (st) return sfail(s, st, std::string("job create: ") + lbpm_last_error(nullptr));
    j->ctx = c;
    if (s->alloc && (st = lbpm_set_allocator(c, s->alloc, s->free_fn, s->alloc_user))) return st;
    if ((st = lbpm_set_params(c, &j->spec.params))) return sfail(s, st, lbpm_last_error(c));
    if ((st = lbpm_load_image(c, j->labels.data(), j->spec.nx, j->spec.ny, j->spec.nz)))
        return sfail(s, st, lbpm_last_error(c));
    if (!j->affinity.empty() && (st = lbpm_set_affinity_map(c, j->affinity.data())))
        return sfail(s, st, lbpm_last_error(c));
    if ((st = lbpm_init_fluids(c, j->phi0.data()))) return sfail(s, st, lbpm_last_error(c));
    return LBPM_OK;
}

void release_job_device(lbpm_server* s, Job* j) {
    if (j->ctx) {
        lbpm_destroy(j->ctx);
        j->ctx = nullptr;
        s->used -= std::min(s->used, j->footprint);
    }
}

// Darcy flux along the driving force (z if there is none: reservoirs).
double driving_flux(const Job* j, const lbpm_measures& m) {
    const double* F = j->spec.params.force;
    const double fn = std::sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    if (fn > 0.0) return (m.flux[0] * F[0] + m.flux[1] * F[1] + m.flux[2] * F[2]) / fn;
    return m.flux[2];
}

}  // namespace

extern "C" {

lbpm_status lbpm_force_rescale(const double force[3], double ca, double ca_target, double max_factor,
                               double out[3], double* factor) {
    if (!force || !out || !(ca_target > 0.0) || !(max_factor >= 1.0) || !std::isfinite(ca) ||
        !std::isfinite(ca_target) || !std::isfinite(max_factor))
        return LBPM_E_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(force[a])) return LBPM_E_INVALID;
    // F <- (Ca* / Ca) F, never changed by more than max_factor either way
    const double g = ca > 0.0 ? std::min(max_factor, std::max(1.0 / max_factor, ca_target / ca)) : max_factor;
    for (int a = 0; a < 3; ++a) out[a] = g * force[a];
    if (factor) *factor = g;
    return LBPM_OK;
}

lbpm_status lbpm_server_create(lbpm_server** out, int device, void* cuda_stream, size_t hbm_budget_bytes,
                               int max_jobs, int check_interval) {
    if (!out) return LBPM_E_INVALID;
    *out = nullptr;
    if (max_jobs < 1 || check_interval < 2 || (check_interval & 1)) return LBPM_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return LBPM_E_INVALID;
    }
    lbpm_server* s = new (std::nothrow) lbpm_server();
    if (!s) return LBPM_E_OOM;
    s->device = device;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->max_jobs = max_jobs;
    s->interval = check_interval;
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = fr / 10 * 9;
    }
    s->budget = hbm_budget_bytes;
    lbpm_status st = lbpm_batch_create(&s->batch, device, cuda_stream);
    if (st) {
        delete s;
        return st;
    }
    now_s();
    *out = s;
    return LBPM_OK;
}

lbpm_status lbpm_server_set_allocator(lbpm_server* s, lbpm_alloc_fn alloc, lbpm_free_fn free_fn, void* user) {
    if (!s) return LBPM_E_INVALID;
    if (!s->jobs.empty()) return sfail(s, LBPM_E_STATE, "set the allocator before submitting jobs");
    s->alloc = alloc;
    s->free_fn = free_fn;
    s->alloc_user = user;
    return lbpm_batch_set_allocator(s->batch, alloc, free_fn, user);
}

const char* lbpm_server_last_error(const lbpm_server* s) { return s ? s->err.c_str() : ""; }

lbpm_status lbpm_server_destroy(lbpm_server* s) {
    if (!s) return LBPM_OK;
    cudaSetDevice(s->device);
    lbpm_batch_destroy(s->batch);
    for (auto& kv : s->jobs) release_job_device(s, kv.second.get());
    delete s;
    return LBPM_OK;
}

lbpm_status lbpm_server_submit(lbpm_server* s, const lbpm_job_spec* spec, long long* ticket) {
    if (!s) return LBPM_E_INVALID;
    s->err.clear();
    if (!spec || !spec->labels || !spec->phi0) return sfail(s, LBPM_E_INVALID, "spec, labels and phi0 are required");
    if (spec->nx < 1 || spec->ny < 1 || spec->nz < 1) return sfail(s, LBPM_E_INVALID, "bad dimensions");
    if (spec->kind < LBPM_JOB_STEADY || spec->kind > LBPM_JOB_CENTRIFUGE) return sfail(s, LBPM_E_INVALID, "bad kind");
    if (spec->max_steps < 0 || !(spec->flux_tol > 0.0)) return sfail(s, LBPM_E_INVALID, "bad convergence settings");
    if (spec->kind == LBPM_JOB_CENTRIFUGE && !(spec->force_factor > 1.0))
        return sfail(s, LBPM_E_INVALID, "centrifuge jobs need force_factor > 1");
    if (spec->ca_target < 0.0 || !std::isfinite(spec->ca_target) || spec->relax_steps < 0 ||
        (spec->ca_target > 0.0 && !(spec->ca_tol > 0.0)))
        return sfail(s, LBPM_E_INVALID, "bad capillary-number target settings");
    if (spec->ca_target > 0.0 && spec->kind != LBPM_JOB_STEADY)
        return sfail(s, LBPM_E_INVALID, "a capillary-number target applies to steady-state jobs");
    auto j = std::make_unique<Job>();
    j->ticket = s->next_ticket++;
    j->spec = *spec;
    const size_t V = static_cast<size_t>(spec->nx) * spec->ny * spec->nz;
    j->labels.assign(spec->labels, spec->labels + V);
    if (spec->affinity) j->affinity.assign(spec->affinity, spec->affinity + V);
    j->phi0.assign(spec->phi0, spec->phi0 + V);
    j->spec.labels = nullptr;
    j->spec.affinity = nullptr;
    j->spec.phi0 = nullptr;
    j->n_pore = std::count(j->labels.begin(), j->labels.end(), static_cast<uint16_t>(0));
    if (j->n_pore == 0) return sfail(s, LBPM_E_INVALID, "the image has no pore voxel");
    j->footprint = estimate_footprint(j->spec, j->n_pore);
    if (j->footprint > s->budget) return sfail(s, LBPM_E_OOM, "job larger than the server's memory budget");
    j->t_submit = now_s();
    if (ticket) *ticket = j->ticket;
    s->queue.push_back(j.get());
    s->jobs.emplace(j->ticket, std::move(j));
    return LBPM_OK;
}

lbpm_status lbpm_server_run(lbpm_server* s, int* n_running, int* n_queued, int* n_finished) {
    if (!s) return LBPM_E_INVALID;
    s->err.clear();
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, LBPM_E_CUDA, "cudaSetDevice");
    lbpm_status st;
    // 1. admission, first come first served, by slots and device-memory budget;
    //    finished jobs give their device state back (oldest first) when a
    //    queued job needs the memory
    while (!s->queue.empty() && static_cast<int>(s->running.size()) < s->max_jobs) {
        while (s->used + s->queue.front()->footprint > s->budget && !s->finished.empty()) {
            release_job_device(s, s->finished.front());
            s->finished.pop_front();
        }
        if (s->used + s->queue.front()->footprint > s->budget) break;
        Job* j = s->queue.front();
        s->queue.pop_front();
        s->used += j->footprint;
        if ((st = build_job(s, j)) || (st = lbpm_batch_add(s->batch, j->ctx))) {
            j->state = LBPM_JOB_FAILED;
            j->note = s->err.empty() ? lbpm_batch_last_error(s->batch) : s->err;
            j->t_done = now_s();
            release_job_device(s, j);
            continue;
        }
        j->state = LBPM_JOB_RUNNING;
        j->t_admit = now_s();
        s->running.push_back(j);
    }
    int finished = 0;
    if (!s->running.empty()) {
        // 2. one interval for every running job, in one batched launch sequence
        if ((st = lbpm_batch_advance(s->batch, s->interval))) return sfail(s, st, lbpm_batch_last_error(s->batch));
        std::vector<lbpm_measures> m(s->running.size());
        st = lbpm_batch_measure(s->batch, m.data());
        if (st && st != LBPM_E_UNSTABLE) return sfail(s, st, lbpm_batch_last_error(s->batch));
        // 3. protocol rules and convergence
        bool params_changed = false;
        std::vector<Job*> keep;
        for (size_t k = 0; k < s->running.size(); ++k) {
            Job* j = s->running[k];
            j->steps += s->interval;
            s->site_updates += j->ctx->N * s->interval;
            j->last = m[k];
            bool done = false;
            if (m[k].status) {
                j->state = LBPM_JOB_FAILED;
                j->note = "unstable";
                done = true;
            } else {
                const double q = driving_flux(j, m[k]);
                const double sw = m[k].sat_mass;
                bool ramped = false;
                if (j->spec.kind == LBPM_JOB_CENTRIFUGE && j->have_prev &&
                    std::fabs(sw - j->sw_prev) < j->spec.sw_tol) {
                    double* F = j->spec.params.force;
                    const double fn = std::sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
                    if (fn > 0.0 && fn < j->spec.force_cap) {
                        const double g = std::min(j->spec.force_factor, j->spec.force_cap / fn);
                        for (int a = 0; a < 3; ++a) F[a] *= g;
                        lbpm_set_params(j->ctx, &j->spec.params);
                        j->force_raises += 1;
                        params_changed = true;
                        ramped = true;
                    }
                }
                // body-force adaptation to the target capillary number
                bool on_target = true;
                j->since_rescale += s->interval;
                if (j->spec.ca_target > 0.0) {
                    on_target = std::fabs(m[k].ca / j->spec.ca_target - 1.0) < j->spec.ca_tol;
                    if (!on_target && j->since_rescale >= j->spec.relax_steps) {
                        double* F = j->spec.params.force;
                        double Fn[3];
                        if (lbpm_force_rescale(F, m[k].ca, j->spec.ca_target, kMaxForceRescale, Fn, nullptr) ==
                            LBPM_OK) {
                            for (int a = 0; a < 3; ++a) F[a] = Fn[a];
                            lbpm_set_params(j->ctx, &j->spec.params);
                            j->force_raises += 1;
                            j->since_rescale = 0;
                            params_changed = true;
                            ramped = true;
                        }
                    }
                }
                if (!ramped && on_target && j->have_prev && std::fabs(q) > 0.0 &&
                    std::fabs(q - j->q_prev) / std::fabs(q) < j->spec.flux_tol) {
                    j->state = LBPM_JOB_DONE;
                    j->note = "converged";
                    done = true;
                } else if (j->steps >= j->spec.max_steps) {
                    j->state = LBPM_JOB_DONE;
                    j->note = "step ceiling";
                    done = true;
                }
                j->q_prev = q;
                j->sw_prev = sw;
                j->have_prev = !ramped;
            }
            if (done) {
                j->t_done = now_s();
                lbpm_batch_remove(s->batch, j->ctx);
                s->finished.push_back(j);
                ++finished;
            } else {
                keep.push_back(j);
            }
        }
        s->running.swap(keep);
        if (params_changed) lbpm_batch_refresh(s->batch);
    }
    if (n_running) *n_running = static_cast<int>(s->running.size());
    if (n_queued) *n_queued = static_cast<int>(s->queue.size());
    if (n_finished) *n_finished = finished;
    return LBPM_OK;
}

lbpm_status lbpm_server_poll(lbpm_server* s, long long ticket, lbpm_job_status* out) {
    if (!s || !out) return LBPM_E_INVALID;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, LBPM_E_INVALID, "unknown ticket");
    const Job* j = it->second.get();
    std::memset(out, 0, sizeof *out);
    out->state = j->state;
    out->steps = j->steps;
    out->n_sites = j->n_pore;
    out->footprint = j->footprint;
    out->t_submit = j->t_submit;
    out->t_admit = j->t_admit;
    out->t_done = j->t_done;
    out->force_raises = j->force_raises;
    for (int a = 0; a < 3; ++a) out->force[a] = j->spec.params.force[a];
    out->last = j->last;
    return LBPM_OK;
}

lbpm_status lbpm_server_job_ctx(lbpm_server* s, long long ticket, lbpm_ctx** ctx) {
    if (!s || !ctx) return LBPM_E_INVALID;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, LBPM_E_INVALID, "unknown ticket");
    *ctx = it->second->ctx;
    return LBPM_OK;
}

lbpm_status lbpm_server_release(lbpm_server* s, long long ticket) {
    if (!s) return LBPM_E_INVALID;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, LBPM_E_INVALID, "unknown ticket");
    Job* j = it->second.get();
    if (j->state == LBPM_JOB_RUNNING) return sfail(s, LBPM_E_STATE, "job is running; cancel it first");
    if (j->state == LBPM_JOB_QUEUED) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), j));
    auto f = std::find(s->finished.begin(), s->finished.end(), j);
    if (f != s->finished.end()) s->finished.erase(f);
    release_job_device(s, j);
    s->jobs.erase(it);
    return LBPM_OK;
}

lbpm_status lbpm_server_cancel(lbpm_server* s, long long ticket) {
    if (!s) return LBPM_E_INVALID;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(s, LBPM_E_INVALID, "unknown ticket");
    Job* j = it->second.get();
    if (j->state == LBPM_JOB_QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), j));
    } else if (j->state == LBPM_JOB_RUNNING) {
        lbpm_batch_remove(s->batch, j->ctx);
        s->running.erase(std::find(s->running.begin(), s->running.end(), j));
        s->finished.push_back(j);
    } else {
        return LBPM_OK;
    }
    j->state = LBPM_JOB_CANCELLED;
    j->t_done = now_s();
    return LBPM_OK;
}

lbpm_status lbpm_server_stats(const lbpm_server* s, long long* site_updates, size_t* used_bytes, size_t* budget_bytes) {
    if (!s) return LBPM_E_INVALID;
    if (site_updates) *site_updates = s->site_updates;
    if (used_bytes) *used_bytes = s->used;
    if (budget_bytes) *budget_bytes = s->budget;
    return LBPM_OK;
}

}  // extern "C"
