// Allocation-free message passing over a caller-supplied graph.
//
// fdtd_step_edgelist keeps the hidden state between the two layers in device
// memory the context allocated.  Some callers cannot allocate at all: a host
// application whose allocator owns every byte of device memory and forbids
// outside allocations, or a real-time loop that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree imply.
// fdtd_mp_steps_noalloc serves them: the caller passes the two layers (CSR by
// destination, as fdtd_export_graph produces them) and the node state, and the
// intermediate state after layer 1 lives in the fixed array below instead of in
// memory obtained from an allocator.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gem_fdtd.h"

namespace {

// Scratch for the node state between layer 1 and layer 2.  Every GPU that loads
// this library holds it (16 MiB) until the process exits.
__device__ __align__(256) float g_mp_scratch[FDTD_MP_NOALLOC_MAX_NODES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// The array's name is a host-side stand-in in host code, not a device address:
// ask the runtime for the address once per device, with that device current.
// The cached address belongs to the device's primary context; a context that
// cudaDeviceReset destroyed and a new one recreated may hold the array elsewhere.
int scratch_for_current_device(float** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FDTD_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mp_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return FDTD_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FDTD_OK;
}

// y[r] = sum over the row's edges of w * x[col]
__global__ void k_mp_layer_noalloc(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const float* __restrict__ w, const float* __restrict__ x, float* __restrict__ y,
                                   int64_t n) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float acc = 0.f;
    const int32_t e1 = rowptr[r + 1];
    for (int32_t e = rowptr[r]; e < e1; e++) acc += w[e] * x[col[e]];
    y[r] = acc;
}

}  // namespace

extern "C" int fdtd_mp_steps_noalloc(const int32_t* rowptr1, const int32_t* col1, const float* w1,
                                     const int32_t* rowptr2, const int32_t* col2, const float* w2, float* h,
                                     int64_t n_nodes, int64_t n_steps, void* cuda_stream) {
    if (!rowptr1 || !col1 || !w1 || !rowptr2 || !col2 || !w2 || !h) return FDTD_EINVAL;
    if (n_nodes < 1 || n_nodes > FDTD_MP_NOALLOC_MAX_NODES || n_steps < 0) return FDTD_EINVAL;
    if (n_steps == 0) return FDTD_OK;
    float* mid = nullptr;
    int rc = scratch_for_current_device(&mid);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int tb = 256;
    const unsigned blocks = (unsigned)((n_nodes + tb - 1) / tb);
    for (int64_t s = 0; s < n_steps; s++) {
        // layer 1 writes every one of the n_nodes scratch entries before layer 2 reads them
        k_mp_layer_noalloc<<<blocks, tb, 0, st>>>(rowptr1, col1, w1, h, mid, n_nodes);
        k_mp_layer_noalloc<<<blocks, tb, 0, st>>>(rowptr2, col2, w2, mid, h, n_nodes);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA;
}
