// Allocation-free variant of the dense field read (lbpm_read_field).
//
// lbpm_read_field stages the dense field in a temporary device buffer that it
// allocates and frees on every call. Some callers cannot allow a device
// allocation once their set-up is done - for example a monitoring loop that
// runs under a fixed device-memory budget handed out at start-up, or a host
// that must not touch the allocator while other work owns it. This file gives
// them lbpm_read_field_noalloc, which runs the same fill and field kernels but
// stages into one file-scope device array instead, so the call allocates and
// frees nothing.
//
// The array holds LBPM_NOALLOC_FIELD_MAX_VOXELS floats (8 MiB). Every GPU on
// which the library's module for this file is loaded keeps it until the
// process exits. lbpm_create looks up its device address (noalloc_setup), which
// also loads this file's module on that device, so the array is placed during
// set-up and not inside a later allocation-free call. All calls on a device share it and it keeps the last call's
// contents; each call overwrites every entry it reads back (solids with NaN,
// pores with the field), so nothing stale is returned, but two calls whose
// device work overlaps (on different streams or host threads) race on it.
#include <mutex>

#include "internal.h"

namespace {

constexpr long long kMaxVoxels = LBPM_NOALLOC_FIELD_MAX_VOXELS;
constexpr int kMaxDevices = 256;

static __device__ __align__(256) float g_field_scratch[kMaxVoxels];

// Device address of g_field_scratch, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in).
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_on_device(int device, float** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

lbpm_status fail(lbpm_ctx* c, lbpm_status s, const std::string& m) {
    c->err = m;
    return s;
}

lbpm_status fail_cuda(lbpm_ctx* c, const char* what, cudaError_t e) {
    return fail(c, LBPM_E_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

}  // namespace

namespace lbm {

cudaError_t noalloc_setup(int device) {
    float* p = nullptr;
    return scratch_on_device(device, &p);
}

}  // namespace lbm

extern "C" lbpm_status lbpm_read_field_noalloc(lbpm_ctx* c, int which, float* out_dense) {
    if (!c) return LBPM_E_INVALID;
    c->err.clear();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail_cuda(c, "cudaSetDevice", e);
    if (!out_dense) return fail(c, LBPM_E_INVALID, "out is NULL");
    if (which < LBPM_FIELD_PHI || which > LBPM_FIELD_RHO) return fail(c, LBPM_E_INVALID, "unknown field");
    if (!c->have_fluids) return fail(c, LBPM_E_STATE, "initialise the fluids first");
    if (c->V > kMaxVoxels)
        return fail(c, LBPM_E_INVALID,
                    "image has " + std::to_string(c->V) + " voxels; the allocation-free field read holds at most " +
                        std::to_string(kMaxVoxels) + " (use lbpm_read_field)");
    // resolved by lbpm_create (noalloc_setup); this only reads the cached address
    float* scratch = nullptr;
    e = scratch_on_device(c->device, &scratch);
    if (e != cudaSuccess) return fail_cuda(c, "cudaGetSymbolAddress(field scratch)", e);
    e = lbm::launch_field(c, static_cast<int>(c->step & 1), which, scratch, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_dense, scratch, sizeof(float) * static_cast<size_t>(c->V), cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, "read_field_noalloc", e);
    c->launches += 2;
    return LBPM_OK;
}
