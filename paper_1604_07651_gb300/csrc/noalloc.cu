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

namespace hr {

// The piece descriptors of one call travel as a kernel parameter (about 13 KB
// for 32 pieces, under the 32 KB parameter limit) and one small kernel writes
// them into the work area: no host-to-device copy from pageable memory, which
// would make the host wait for the stream.
struct PieceTable {
    int n;
    PieceDev p[kWorkMaxPieces];
};
static_assert(sizeof(PieceTable) <= 32000, "kernel parameters are limited to 32764 bytes");
static_assert(sizeof(PieceDev) % sizeof(int) == 0, "descriptors are copied as ints");

__global__ void k_write_pieces(const __grid_constant__ PieceTable T, PieceDev* dst) {
    const int words = (int)(sizeof(PieceDev) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(T.p);
    int* out = reinterpret_cast<int*>(dst);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.n * words; i += gridDim.x * blockDim.x)
        out[i] = src[i];
}

int launch_write_pieces(const PieceDev* pieces, int n, PieceDev* dst, void* stream) {
    if (n < 0 || n > kWorkMaxPieces) return (int)cudaErrorInvalidValue;
    PieceTable T;
    T.n = n;
    for (int i = 0; i < n; ++i) T.p[i] = pieces[i];
    k_write_pieces<<<1, 256, 0, (cudaStream_t)stream>>>(T, dst);
    return (int)cudaGetLastError();
}

}  // namespace hr

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
