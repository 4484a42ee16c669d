// gee_noalloc.cu -- gee_embed_noalloc: the edge-list embedding without any
// device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// service whose device memory was divided up at start-up by another
// allocator (a framework's caching pool may own everything that is left), or
// latency-critical code that must not risk a call into the driver's
// allocator in the middle of its work.  For them this entry point keeps its
// scratch -- the status word, the class sizes n_k and the compact labels --
// in one fixed array in device global memory that is part of the library
// image, so every GPU that loads the library holds it until the process
// exits.  The caller still owns edges, weights, Y and Z.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call re-initialises what must start at zero.  Calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <mutex>

#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr size_t kHeaderBytes = 2048;  // status word + n_k, 256-aligned
constexpr size_t kScratchBytes = (size_t)GEE_NOALLOC_SCRATCH_BYTES;
static_assert(kScratchBytes > kHeaderBytes, "scratch too small");

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices];

// Device address of g_scratch on the current device, looked up once per
// device (the first call on a device does this set-up) and kept for the
// life of the process: after a cudaDeviceReset it would name memory of the
// destroyed context, so the header asks callers not to reset a device they
// use this entry point on.
cudaError_t scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

gee_status noalloc_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return GEE_OK;
    return e == cudaErrorMemoryAllocation ? GEE_ERR_OOM : GEE_ERR_CUDA;
}

}  // namespace

}  // namespace gee

using namespace gee;

extern "C" GEE_API gee_status gee_embed_noalloc(const int32_t *edges,
                                                const float *weights,
                                                int64_t s, const int32_t *Y,
                                                int64_t n, int32_t K, float *Z,
                                                gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (s < 0 || n < 0 || K < 1)
        return GEE_ERR_INVALID_ARG;
    if (K > kMaxClasses || n > (int64_t)GEE_NOALLOC_MAX_NODES)
        return GEE_ERR_UNSUPPORTED;
    if ((s > 0 && edges == nullptr) || (n > 0 && (Y == nullptr || Z == nullptr)) ||
        (reinterpret_cast<uintptr_t>(edges) & 7) != 0 ||
        ((reinterpret_cast<uintptr_t>(weights) | reinterpret_cast<uintptr_t>(Y) |
          reinterpret_cast<uintptr_t>(Z)) & 3) != 0)
        return GEE_ERR_INVALID_ARG;
    if (s > 0 && n == 0)
        return GEE_ERR_NODE_RANGE;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return noalloc_status(e);
    DevStatus *st = reinterpret_cast<DevStatus *>(base);
    uint32_t *counts = reinterpret_cast<uint32_t *>(base + 256);
    uint8_t *Yc = base + kHeaderBytes;
    // what must start at zero is cleared on every call
    if ((e = launch_status_init(st, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * K, stream)) !=
            cudaSuccess ||
        (e = launch_labels(Y, n, K, nullptr, Yc, counts, st, stream)) !=
            cudaSuccess ||
        (e = launch_validate_edges(edges, s, n, st, stream)) != cudaSuccess ||
        (e = launch_zero(Z, n * K, st, stream)) != cudaSuccess ||
        (e = launch_scatter_atomic(edges, weights, nullptr, s, n, K, Yc, Z,
                                   false, 256, st, stream)) != cudaSuccess)
        return noalloc_status(e);
    e = (weights != nullptr)
            ? launch_finalize_weighted(Z, nullptr, n, K, counts, st, stream)
            : launch_finalize_count(Z, n, K, counts, st, stream);
    if (e != cudaSuccess)
        return noalloc_status(e);
    DevStatus h;
    e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return noalloc_status(e);
    return static_cast<gee_status>(h.code);
}
