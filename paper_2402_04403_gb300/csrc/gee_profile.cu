// gee_profile.cu -- launch tracing: per-kernel CUDA-event timings.
//
// When enabled, each kernel launch of the library is bracketed by two CUDA
// events recorded on the stream the kernel is launched on; gee_profile_read
// waits for them and reports launches, total and largest duration per kernel
// name.  Used by the benchmark to time the edge-pass kernel inside a running
// step, and to count the library's launches.  Every launch is also an NVTX
// range named for its kernel, whether or not timing is enabled.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gee_internal.cuh"

namespace gee {

namespace {

struct Record {
    const char *name;
    cudaEvent_t begin, end;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_free;

cudaEvent_t take_event()
{
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_free.empty()) {
            cudaEvent_t e = g_free.back();
            g_free.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess)
        return nullptr;
    return e;
}

}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t stream)
    : name_(name), stream_(stream)
{
    // a named host range around the launch for NVTX tools (a no-op without
    // one attached)
    nvtxRangePushA(name_);
    if (!g_on.load(std::memory_order_relaxed))
        return;
    // launches captured into a CUDA graph are not traced
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream_, &cap) != cudaSuccess ||
        cap != cudaStreamCaptureStatusNone)
        return;
    begin_ = take_event();
    if (begin_ != nullptr && cudaEventRecord(begin_, stream_) != cudaSuccess)
        begin_ = nullptr;
}

ProfScope::~ProfScope()
{
    nvtxRangePop();
    if (begin_ == nullptr)
        return;
    cudaEvent_t end = take_event();
    if (end == nullptr || cudaEventRecord(end, stream_) != cudaSuccess)
        return;
    std::lock_guard<std::mutex> lock(g_mu);
    g_records.push_back(Record{name_, begin_, end});
}

}  // namespace gee

extern "C" {

GEE_API void gee_profile_enable(int32_t on)
{
    gee::g_on.store(on != 0);
}

GEE_API int32_t gee_profile_read(gee_kernel_time *out, int32_t max_entries)
{
    using namespace gee;
    std::vector<Record> recs;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        recs.swap(g_records);
    }
    std::map<std::string, gee_kernel_time> agg;
    for (const Record &r : recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.end) == cudaSuccess &&
            cudaEventElapsedTime(&ms, r.begin, r.end) == cudaSuccess) {
            gee_kernel_time &t = agg[r.name];
            std::strncpy(t.name, r.name, sizeof(t.name) - 1);
            t.launches += 1;
            t.total_ms += ms;
            if (ms > t.max_ms)
                t.max_ms = ms;
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_mu);
        for (const Record &r : recs) {
            g_free.push_back(r.begin);
            g_free.push_back(r.end);
        }
    }
    int32_t i = 0;
    for (auto &kv : agg) {
        if (out != nullptr && i < max_entries)
            out[i] = kv.second;
        ++i;
    }
    return i;
}

}  // extern "C"
