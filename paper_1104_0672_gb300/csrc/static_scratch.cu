// Allocation-free forward convolution: arkcos_convolve with its workspace taken from a fixed
// device array that is part of the library image instead of from the caller.
//
// Some callers cannot hand the library a device workspace: a host program whose device memory
// is owned by another framework's pool and must not be allocated behind its back, or a loop
// that may not call cudaMalloc (which can synchronise the device) once it is running.  For
// them, arkcos_convolve_static uses the array below as its scratch.  Its size is fixed when the
// library is built, every GPU that loads the library reserves it until the process exits, and
// all calls share it.
#include <stdio.h>

#include <mutex>

#include "arkcos_impl.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a stand-in for the symbol; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" arkcos_status arkcos_convolve_static(arkcos_grid grid, const arkcos_kernel *kernels,
                                                int64_t nkernels, const float *map_in,
                                                float *map_out, int64_t nmaps, void *stream,
                                                uint32_t flags)
{
    size_t need = 0;
    arkcos_status st = arkcos_workspace_size(grid, kernels, nkernels, nmaps, flags, 0, &need);
    if (st != ARKCOS_OK) return st;
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "arkcos_convolve_static: this call needs %zu bytes of scratch, the built-in "
                 "scratch holds %zu; use arkcos_convolve with a caller workspace",
                 need, kStaticScratchBytes);
        arkcos::set_last_error(msg);
        return ARKCOS_EWORKSPACE;
    }
    void *ws = nullptr;
    cudaError_t e = scratch_address(&ws);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "arkcos_convolve_static: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        arkcos::set_last_error(msg);
        return ARKCOS_ECUDA;
    }
    // every stage of the forward pass overwrites the scratch it later reads, so nothing in it
    // has to start at zero and the previous call's contents are harmless
    return arkcos_convolve(grid, kernels, nkernels, map_in, map_out, nmaps, ws,
                           kStaticScratchBytes, stream, flags);
}
