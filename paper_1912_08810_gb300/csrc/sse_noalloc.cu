// sse_execute_noalloc: the mixed-precision evaluation of Sigma without a plan and without
// any memory allocation by this library.
//
// Who needs this: callers that must not (or cannot) have a library call cudaMalloc on their
// behalf -- a framework whose caching allocator owns the device memory and accounts for
// every byte, a service running under a fixed device-memory budget, or a latency-critical
// loop where cudaMalloc/cudaFree could synchronise the device and stall for milliseconds.
// The regular path (sse_plan) allocates a small device status word per plan and copies the
// neighbour list to the host to validate it; this entry point does neither.
//
// Instead, the scratch the kernels need lives in one file-scope device array,
// `sse_noalloc_scratch`, of a fixed size (kScratchWords 32-bit words) that every GPU which
// loads this library holds until the process exits.  Host code cannot use the array's name
// as a device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; make that first call
// before any stream capture.  All calls on a device share the array: the words a call
// relies on starting at zero are cleared at the start of every call, and two calls whose
// work overlaps on the GPU (other streams, other threads) race on it.  Every call reads
// the neighbour check's result and the kernel's wait status back to the host, so it
// synchronises its stream twice and blocks the calling thread until Sigma is written.
#include <cuda_runtime.h>

#include <mutex>

#include "sse_internal.h"

namespace sse {
namespace {

constexpr int kScratchWords = 64;  // 256 bytes; the call below uses kUsedWords of them
constexpr int kUsedWords = 4;
// word 0: number of out-of-range neighbour entries; word 1: smallest bad entry index
// (low 32 bits); word 2: device-wait status of the mixed kernel; word 3: unused padding
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t sse_noalloc_scratch[kScratchWords];

std::mutex g_mu;
int32_t *g_scratch_addr[kMaxDevices] = {};

// Range-check the neighbour list on the device: every entry must be in [-1, na).
__global__ void check_neighbours(const int32_t *__restrict__ neigh, long long n, int32_t na) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int32_t f = neigh[i];
        if (f < -1 || f >= na) {
            atomicAdd(&sse_noalloc_scratch[0], 1);
            atomicMin(&sse_noalloc_scratch[1], (int32_t)(i > 0x7fffffffLL ? 0x7fffffff : i));
        }
    }
}

__global__ void init_scratch() {
    if (threadIdx.x < kUsedWords) sse_noalloc_scratch[threadIdx.x] = threadIdx.x == 1 ? 0x7fffffff : 0;
}

bool on_device(const void *ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sse_status scratch_address(int32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error("device index %d out of range", dev), SSE_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, sse_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(sse_noalloc_scratch)");
        g_scratch_addr[dev] = (int32_t *)p;
    }
    *out = g_scratch_addr[dev];
    return SSE_OK;
}

}  // namespace
}  // namespace sse

using namespace sse;

extern "C" SSE_API sse_status sse_execute_noalloc(const sse_geometry *geo, const sse_io *io, void *stream) {
    if (!geo || !io) return set_error("geometry or io is NULL"), SSE_E_INVALID_ARG;
    if (geo->mode != SSE_MODE_MIXED) return set_error("sse_execute_noalloc runs the mixed mode only"), SSE_E_INVALID_ARG;
    if (geo->nkz <= 0 || geo->nqz <= 0 || geo->ne <= 0 || geo->nw <= 0 || geo->na <= 0 || geo->nb_max <= 0 ||
        geo->norb != kNorb || geo->omega_first <= -(1 << 20) || geo->omega_first >= (1 << 20) || (geo->dtype != SSE_C128 && geo->dtype != SSE_C64) ||
        !geo->neigh || !geo->dH)
        return set_error("invalid geometry for sse_execute_noalloc"), SSE_E_INVALID_ARG;
    if (geo->nkz > 5 || geo->nb_max > 32)
        return set_error("sse_execute_noalloc supports Nkz <= 5 and nb_max <= 32 (got %d, %d)", geo->nkz,
                         geo->nb_max),
               SSE_E_INVALID_ARG;
    if (!on_device(geo->neigh) || !on_device(geo->dH))
        return set_error("neigh and dH must be device pointers"), SSE_E_INVALID_ARG;
    if (io->S_gt && (!on_device(io->G_gt) || !on_device(io->D_gt) || !on_device(io->S_gt)))
        return set_error("G_gt, D_gt and S_gt must be device pointers"), SSE_E_INVALID_ARG;
    if (io->S_lt && (!on_device(io->G_lt) || !on_device(io->D_lt) || !on_device(io->S_lt)))
        return set_error("G_lt, D_lt and S_lt must be device pointers"), SSE_E_INVALID_ARG;
    if (!io->S_gt && !io->S_lt) return SSE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *scratch = nullptr;
    sse_status rs = scratch_address(&scratch);
    if (rs != SSE_OK) return rs;

    // clear the words this call relies on, then validate the neighbour list on the device
    init_scratch<<<1, 32, 0, st>>>();
    const long long n = (long long)geo->na * geo->nb_max;
    const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    check_neighbours<<<blocks, 256, 0, st>>>(geo->neigh, n, geo->na);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch neighbour check");
    int32_t words[kUsedWords];
    e = cudaMemcpyAsync(words, scratch, sizeof words, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "read neighbour check");
    if (words[0] != 0)
        return set_error("neigh has %d entries outside [-1, %d); first at flat index %d", words[0], geo->na, words[1]),
               SSE_E_INVALID_ARG;

    Plan p{};
    p.geo = *geo;
    p.d = Dims{geo->nkz, geo->nqz, geo->ne, geo->nw, geo->na, geo->nb_max, geo->omega_first};
    cudaGetDevice(&p.device);
    p.kernel_id = 1;
    p.d_status = scratch + 2;
    rs = launch_mixed(p, *io, st);
    if (rs != SSE_OK) return rs;
    e = cudaMemcpyAsync(words, scratch, sizeof words, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise sse_execute_noalloc");
    if (words[2] & kStatusBounds) return set_error("a kernel computed an index outside one of its buffers"), SSE_E_BOUNDS;
    if (words[2] != 0) return set_error("a device-side wait of the mixed kernel expired"), SSE_E_TIMEOUT;
    return SSE_OK;
}
