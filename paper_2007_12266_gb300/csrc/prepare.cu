// Image preparation kernels (declared in include/lbpm.h):
//   mixing region at the inlet/outlet faces of the flow axis (Sec. 4.2), and
//   mixed-wet relabel of the solid near the oil phase (Sec. 3.3).
// Both are one pass over the voxels, one thread per voxel, integer results.
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace {

constexpr int kThreads = 256;

struct Dims {
    int n[3];          // nx, ny, nz
    long long stride[3];
};

// Grid: x in blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y, z = blockIdx.z
// (no index division); the extents are below 65,536 in y and z.
__device__ __forceinline__ bool voxel_of(const Dims& d, int c[3], long long& v) {
    c[0] = blockIdx.x * kThreads + threadIdx.x;
    c[1] = blockIdx.y;
    c[2] = blockIdx.z;
    v = c[0] + c[1] * d.stride[1] + c[2] * d.stride[2];
    return c[0] < d.n[0];
}

// Sec. 4.2: solids in the inlet layers are removed where the outlet face is
// pore, and solids in the outlet layers where the inlet face is pore. The
// faces are read from the input copy, so the two rules see the original image.
__global__ void __launch_bounds__(kThreads) k_mixing_layer(const uint16_t* __restrict__ in, uint16_t* __restrict__ out,
                                                          Dims d, int axis, int n_mix) {
    int c[3];
    long long v;
    if (!voxel_of(d, c, v)) return;
    const int a = axis == 0 ? c[0] : (axis == 1 ? c[1] : c[2]);
    const int L = axis == 0 ? d.n[0] : (axis == 1 ? d.n[1] : d.n[2]);
    const long long st = axis == 0 ? d.stride[0] : (axis == 1 ? d.stride[1] : d.stride[2]);
    uint16_t lab = in[v];
    if (lab != 0 && (a < n_mix || a >= L - n_mix)) {
        const long long base = v - static_cast<long long>(a) * st;
        if (a < n_mix && in[base + static_cast<long long>(L - 1) * st] == 0) lab = 0;
        if (a >= L - n_mix && in[base] == 0) lab = 0;
    }
    out[v] = lab;
}

// Sec. 3.3: relabel the solid within `radius` of the oil phase. Voxels at
// least R from every face test the ball through precomputed linear offsets;
// the others wrap (periodic axes) or skip (non-periodic) per component.
__global__ void __launch_bounds__(kThreads) k_mixed_wet(const uint16_t* __restrict__ in,
                                                       const uint8_t* __restrict__ oil, uint16_t* __restrict__ out,
                                                       Dims d, int px, int py, int pz, const int3* __restrict__ off,
                                                       const long long* __restrict__ lin, int n_off, int R,
                                                       uint16_t new_label) {
    int c[3];
    long long v;
    if (!voxel_of(d, c, v)) return;
    uint16_t lab = in[v];
    if (lab != 0) {
        bool near = false;
        const bool interior = c[0] >= R && c[0] < d.n[0] - R && c[1] >= R && c[1] < d.n[1] - R && c[2] >= R &&
                              c[2] < d.n[2] - R;
        if (interior) {
            for (int i = 0; i < n_off && !near; ++i) near = oil[v + lin[i]] != 0;
        } else {
            const int per[3] = {px, py, pz};
            for (int i = 0; i < n_off && !near; ++i) {
                const int o[3] = {off[i].x, off[i].y, off[i].z};
                long long u = 0;
                bool inside = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int x = c[a] + o[a];
                    if (x < 0 || x >= d.n[a]) {
                        if (!per[a]) {
                            inside = false;
                            break;
                        }
                        x = ((x % d.n[a]) + d.n[a]) % d.n[a];
                    }
                    u += static_cast<long long>(x) * d.stride[a];
                }
                near = inside && oil[u] != 0;
            }
        }
        if (near) lab = new_label;
    }
    out[v] = lab;
}

dim3 grid_of(int nx, int ny, int nz) {
    return dim3(static_cast<unsigned>((nx + kThreads - 1) / kThreads), static_cast<unsigned>(ny),
                static_cast<unsigned>(nz));
}

Dims dims_of(int nx, int ny, int nz) {
    Dims d;
    d.n[0] = nx;
    d.n[1] = ny;
    d.n[2] = nz;
    d.stride[0] = 1;
    d.stride[1] = nx;
    d.stride[2] = static_cast<long long>(nx) * ny;
    return d;
}

// device buffers of one call, freed on every path
struct Scratch {
    std::vector<void*> p;
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    T* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, n * sizeof(T) + 16) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return static_cast<T*>(q);
    }
};

lbpm_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? LBPM_OK : (e == cudaErrorMemoryAllocation ? LBPM_E_OOM : LBPM_E_CUDA);
}

}  // namespace

extern "C" {

lbpm_status lbpm_mixing_layer(int device, uint16_t* labels, int nx, int ny, int nz, int axis, int n_mix) {
    if (!labels || nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535 || axis < 0 || axis > 2)
        return LBPM_E_INVALID;
    const int ext[3] = {nx, ny, nz};
    if (n_mix < 1 || 2 * n_mix > ext[axis]) return LBPM_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return LBPM_E_INVALID;
    }
    const long long V = static_cast<long long>(nx) * ny * nz;
    Scratch s;
    uint16_t* din = s.get<uint16_t>(V);
    uint16_t* dout = s.get<uint16_t>(V);
    if (!din || !dout) return LBPM_E_OOM;
    cudaError_t e = cudaMemcpy(din, labels, V * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_mixing_layer<<<grid_of(nx, ny, nz), kThreads>>>(din, dout, dims_of(nx, ny, nz), axis, n_mix);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(labels, dout, V * sizeof(uint16_t), cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

lbpm_status lbpm_mixed_wet_relabel(int device, uint16_t* labels, const uint8_t* oil, int nx, int ny, int nz,
                                   const int periodic[3], double radius, int new_label) {
    if (!labels || !oil || !periodic || nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535 ||
        !(radius > 0.0) || !(radius <= 8.0) || new_label < 1 || new_label > 65535)
        return LBPM_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return LBPM_E_INVALID;
    }
    // voxel offsets of the ball |o| <= radius, centre excluded (the centre is solid)
    std::vector<int3> off;
    const int R = static_cast<int>(std::floor(radius));
    const double r2 = radius * radius;
    for (int z = -R; z <= R; ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x)
                if ((x || y || z) && static_cast<double>(x * x + y * y + z * z) <= r2) off.push_back(make_int3(x, y, z));
    const long long V = static_cast<long long>(nx) * ny * nz;
    std::vector<long long> lin(off.size());
    for (size_t i = 0; i < off.size(); ++i)
        lin[i] = off[i].x + static_cast<long long>(off[i].y) * nx + static_cast<long long>(off[i].z) * nx * ny;
    Scratch s;
    uint16_t* din = s.get<uint16_t>(V);
    uint16_t* dout = s.get<uint16_t>(V);
    uint8_t* doil = s.get<uint8_t>(V);
    int3* doff = s.get<int3>(off.size());
    long long* dlin = s.get<long long>(lin.size());
    if (!din || !dout || !doil || !doff || !dlin) return LBPM_E_OOM;
    cudaError_t e = cudaMemcpy(din, labels, V * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(doil, oil, V, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(doff, off.data(), off.size() * sizeof(int3), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dlin, lin.data(), lin.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_mixed_wet<<<grid_of(nx, ny, nz), kThreads>>>(din, doil, dout, dims_of(nx, ny, nz), periodic[0] != 0,
                                                      periodic[1] != 0, periodic[2] != 0, doff, dlin,
                                                      static_cast<int>(off.size()), R, static_cast<uint16_t>(new_label));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(labels, dout, V * sizeof(uint16_t), cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

}  // extern "C"
