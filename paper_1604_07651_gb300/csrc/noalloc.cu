// radon_fwd_noalloc: the forward transform with its work memory in a fixed
// static device array, for callers that cannot call cudaMalloc.
//
// Some callers may not allocate device memory when they call us: code whose
// host framework has already reserved the whole device for its own memory
// pool, deployments that must keep a fixed, known device footprint, and
// latency-critical loops that cannot afford the device-wide synchronisation
// cudaMalloc/cudaFree can cause. For them this entry point takes its work
// buffers (spectra, lattices, the device copy of the piece descriptors) from
// g_noalloc_work below instead of the plan's own buffers, and calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// g_noalloc_work exists on every GPU that loads this library, from load until
// exit. In host code its name is only a host-side stand-in, not a device
// address: the device address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, with that device
// current) and cached.
#include <cuda_runtime.h>

#include <mutex>

#include "hradon.h"
#include "internal.h"

static __device__ __align__(256) unsigned char g_noalloc_work[RADON_NOALLOC_MAX_BYTES];

namespace {

const int kMaxDevices = 256;
void* g_work_addr[kMaxDevices];  // device address of g_noalloc_work, per device
std::mutex g_work_mutex;

struct CurrentDevice {
    int prev = -1;
    bool changed = false;
    explicit CurrentDevice(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~CurrentDevice() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" radon_status radon_fwd_noalloc(radon_plan p, const float* f, float* g, void* stream) {
    if (!p) return (radon_status)hr::set_error(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g) return (radon_status)hr::set_error(RADON_ERR_INVALID_ARG, "NULL data pointer");
    const int dev = hr::plan_device(p);
    if (dev < 0 || dev >= kMaxDevices)
        return (radon_status)hr::set_error(RADON_ERR_UNSUPPORTED, "device ordinal above 255");
    CurrentDevice cur(dev);
    void* work = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_work_mutex);
        if (!g_work_addr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_work);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return (radon_status)hr::set_error(RADON_ERR_CUDA,
                                                   "cudaGetSymbolAddress of the static work area failed");
            }
            g_work_addr[dev] = ptr;
        }
        work = g_work_addr[dev];
    }
    return (radon_status)hr::plan_forward_in_work(p, f, g, work, RADON_NOALLOC_MAX_BYTES, stream);
}
