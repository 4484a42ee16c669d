// gee_tune.cu -- the autotuner behind GEE_AUTO for edge-list calls.
//
// gee_autotune times every edge-list strategy (ATOMIC at three block
// sizes, PRIVATE where the copy of Z fits in shared memory, SEGMENTED) on
// seeded synthetic problems over a grid of Z sizes (cells = n*K) and edge
// densities (2s / cells), and installs, for the current device, the fastest
// choice per grid point.  gee_pick_strategy (and so gee_embed with
// GEE_AUTO) then takes the nearest grid point's choice; without a table it
// falls back to its built-in rule.  Tables can be read and installed again
// (gee_tune_get / gee_tune_set) so a service tunes once per machine.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>

#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kMaxDevices = 64;
constexpr int kTuneK = 16;
constexpr int kBlocks[3] = {128, 256, 512};

std::mutex g_tmu;
std::vector<gee_tune_cell> g_tables[kMaxDevices];

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        dev = 0;  // no device (host-side use): table 0
    }
    return dev;
}

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014): one 64-bit mix per draw
__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// uniform random multigraph and labels of a tuning problem
__global__ void k_tune_problem(int2 *E, int64_t s, int32_t *Y, int64_t n,
                               int32_t K, uint64_t seed)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < s; i += nth) {
        const uint64_t r = mix64(seed ^ (uint64_t)i);
        E[i] = make_int2((int)(((r & 0xFFFFFFFFull) * (uint64_t)n) >> 32),
                         (int)(((r >> 32) * (uint64_t)n) >> 32));
    }
    for (int64_t i = tid; i < n; i += nth) {
        const uint64_t r = mix64(~seed ^ (uint64_t)i);
        Y[i] = (int32_t)(((r & 0xFFFFFFFFull) * (uint64_t)K) >> 32);
    }
}

}  // namespace

bool tuned_choice(int64_t s, int64_t n, int32_t K, gee_strategy *strategy,
                  int32_t *block)
{
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_tmu);
    const std::vector<gee_tune_cell> &t = g_tables[dev];
    if (t.empty())
        return false;
    const double cells = std::max<double>(1.0, (double)n * (double)K);
    const double lc = std::log2(cells);
    const double ld = std::log2(std::max(2.0 * (double)s / cells, 1.0 / 1024));
    const gee_tune_cell *best = nullptr;
    double bd = 0.0;
    for (const gee_tune_cell &c : t) {
        const double d = std::fabs(c.log2_cells - lc) + std::fabs(c.log2_density - ld);
        if (best == nullptr || d < bd) {
            best = &c;
            bd = d;
        }
    }
    *strategy = static_cast<gee_strategy>(best->strategy);
    *block = best->block;
    return true;
}

}  // namespace gee

using namespace gee;

extern "C" {

gee_status gee_tune_set(const gee_tune_cell *cells, int32_t count)
{
    if (count < 0 || (count > 0 && cells == nullptr))
        return GEE_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i) {
        const gee_tune_cell &c = cells[i];
        if (c.strategy < GEE_ATOMIC || c.strategy > GEE_BINNED ||
            (c.block != 0 && (c.block % 32 != 0 || c.block < 32 || c.block > 1024)))
            return GEE_ERR_INVALID_ARG;
    }
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tables[dev].assign(cells, cells + count);
    return GEE_OK;
}

int32_t gee_tune_get(gee_tune_cell *out, int32_t max_cells)
{
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_tmu);
    const std::vector<gee_tune_cell> &t = g_tables[dev];
    if (out != nullptr)
        for (int32_t i = 0; i < max_cells && i < (int32_t)t.size(); ++i)
            out[i] = t[(size_t)i];
    return (int32_t)t.size();
}

gee_status gee_autotune(int32_t effort, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (effort < 0 || effort > 2)
        return GEE_ERR_INVALID_ARG;
    const int step = effort >= 1 ? 1 : 2;                 // log2 grid steps
    const int reps = effort >= 2 ? 5 : 3;
    const int64_t max_edges = int64_t(1) << (effort >= 1 ? 26 : 24);
    std::vector<int> lcs, lds;
    for (int lc = 10; lc <= 24; lc += step)
        lcs.push_back(lc);
    for (int ld = -2; ld <= 4; ld += step)
        lds.push_back(ld);
    const int64_t max_cells = int64_t(1) << lcs.back();
    // one scratch problem large enough for every grid point
    Workspace ws(stream);
    int2 *E = nullptr;
    int32_t *Y = nullptr;
    float *Z = nullptr;
    cudaError_t e = ws.alloc((void **)&E, sizeof(int2) * max_edges);
    if (e == cudaSuccess)
        e = ws.alloc((void **)&Y, sizeof(int32_t) * (max_cells / kTuneK + 1));
    if (e == cudaSuccess)
        e = ws.alloc((void **)&Z, sizeof(float) * max_cells);
    if (e != cudaSuccess)
        return from_cuda(e);
    std::vector<gee_tune_cell> table;
    const int64_t plimit = private_cells_limit();
    for (int lc : lcs) {
        for (int ld : lds) {
            const int64_t cells = int64_t(1) << lc;
            const int64_t n = cells / kTuneK;
            const double dens = std::ldexp(1.0, ld);
            int64_t s = (int64_t)(dens * (double)cells / 2.0);
            s = std::min(std::max<int64_t>(s, 1), max_edges);
            k_tune_problem<<<grid_for(std::max(s, n), 256, sm_count() * 8), 256, 0,
                             stream>>>(E, s, Y, n, kTuneK,
                                       0x5EEDull * (uint64_t)(lc * 64 + ld + 8));
            if ((e = cudaGetLastError()) != cudaSuccess)
                return from_cuda(e);
            gee_tune_cell c{};
            c.log2_cells = lc;
            c.log2_density = ld;
            float best = 0.0f;
            auto time_it = [&](gee_strategy st, int32_t block) -> float {
                gee_options o;
                gee_options_default(&o);
                o.strategy = st;
                o.block = block;
                o.validate_edges = 1;
                std::vector<double> ms;
                for (int r = 0; r <= reps; ++r) {
                    const auto t0 = std::chrono::steady_clock::now();
                    const gee_status rc = gee_embed(reinterpret_cast<const int32_t *>(E),
                                                    nullptr, s, Y, n, kTuneK, 0, Z,
                                                    &o, stream_);
                    const auto t1 = std::chrono::steady_clock::now();
                    if (rc != GEE_OK)
                        return -1.0f;
                    if (r > 0)  // the first run warms up
                        ms.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
                }
                std::sort(ms.begin(), ms.end());
                return (float)ms[ms.size() / 2];
            };
            auto consider = [&](gee_strategy st, int32_t block, float t) {
                if (t >= 0.0f && (best == 0.0f || t < best)) {
                    best = t;
                    c.strategy = st;
                    c.block = block;
                }
            };
            float atomic_best = -1.0f;
            for (int b : kBlocks) {
                const float t = time_it(GEE_ATOMIC, b);
                consider(GEE_ATOMIC, b, t);
                if (t >= 0.0f && (atomic_best < 0.0f || t < atomic_best))
                    atomic_best = t;
            }
            c.ms_atomic = atomic_best;
            c.ms_private = cells <= plimit ? time_it(GEE_PRIVATE, 0) : -1.0f;
            consider(GEE_PRIVATE, 0, c.ms_private);
            c.ms_segmented = time_it(GEE_SEGMENTED, 0);
            consider(GEE_SEGMENTED, 0, c.ms_segmented);
            if (best == 0.0f)
                return GEE_ERR_CUDA;
            table.push_back(c);
        }
    }
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tables[dev] = table;
    return GEE_OK;
}

}  // extern "C"
