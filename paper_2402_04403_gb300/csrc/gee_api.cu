// gee_api.cu -- the C ABI of libgee (declared in include/gee.h): argument
// checks, scratch memory, strategy choice, launch sequence and status
// read-back.  Every kernel lives in gee_coo.cu or gee_csr.cu.
#include <atomic>
#include <mutex>
#include <vector>

#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices];
int g_smem[kMaxDevices];
std::atomic<int32_t> g_fail_allocs{0};
cudaMemPool_t g_pool[kMaxDevices];
bool g_pool_ready[kMaxDevices];

}  // namespace

gee_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess)
        return GEE_OK;
    if (e == cudaErrorMemoryAllocation)
        return GEE_ERR_OOM;
    return GEE_ERR_CUDA;
}

// The library's stream-ordered pool on the current device.  Freed blocks stay
// cached in the pool (release threshold = max) so repeated calls do not go
// back to the driver.
cudaError_t device_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess)
            return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold,
                                    &keep);
        if (e != cudaSuccess)
            return e;
        g_pool[dev] = pool;
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// Device address of page-locked (registered or cudaMallocHost) host memory,
// or null for pageable or unaligned memory.
float *mapped_host(float *p)
{
    if (p == nullptr || (reinterpret_cast<uintptr_t>(p) & 3) != 0)
        return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // pageable memory may report an error: clear it
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr)
        return nullptr;
    return static_cast<float *>(at.devicePointer);
}

namespace {

// Long-lived arrays of a resident graph.
class GraphAllocator : public Allocator {
  public:
    explicit GraphAllocator(std::vector<void *> *owned) : owned_(owned) {}
    cudaError_t alloc(void **p, size_t bytes) override
    {
        if (injected_alloc_failure())
            return cudaErrorMemoryAllocation;
        if (bytes == 0)
            bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess)
            owned_->push_back(*p);
        return e;
    }

  private:
    std::vector<void *> *owned_;
};

// Waits for the stream and returns the first status a kernel reported.
gee_status read_status(const DevStatus *st, cudaStream_t stream)
{
    DevStatus h;
    cudaError_t e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost,
                                    stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return from_cuda(e);
    return static_cast<gee_status>(h.code);
}

// Deterministic float sums need the pull form (fixed-point cells owned by
// one row tile or hub chunk): AUTO becomes SEGMENTED; the scatter forms
// (global float atomics) cannot give them.
gee_status deterministic_strategy(gee_options &o, bool weighted,
                                  int32_t laplacian)
{
    if (!o.deterministic || !(weighted || laplacian))
        return GEE_OK;
    if (o.strategy == GEE_AUTO)
        o.strategy = GEE_SEGMENTED;
    return o.strategy == GEE_SEGMENTED ? GEE_OK : GEE_ERR_UNSUPPORTED;
}

bool binned_fits(int64_t n, int32_t K)
{
    int32_t coarse = 0, group = 0;
    const int32_t rows = bin_rows(K, true);
    return bin_layout((n + rows - 1) / rows, &coarse, &group);
}

gee_options resolve_options(const gee_options *opts)
{
    gee_options o;
    gee_options_default(&o);
    if (opts != nullptr)
        o = *opts;
    return o;
}

gee_status check_common(int64_t s, int64_t n, int32_t K, int32_t threads)
{
    if (s < 0 || n < 0 || K < 1)
        return GEE_ERR_INVALID_ARG;
    if (K > kMaxClasses)
        return GEE_ERR_UNSUPPORTED;
    if (n > INT32_MAX || s > (INT64_MAX / 4))
        return GEE_ERR_OVERFLOW;
    if (threads != 0 && (threads % 32 != 0 || threads < 32 || threads > 1024))
        return GEE_ERR_INVALID_ARG;
    return GEE_OK;
}

// Edge lists are read one int2 per edge.
inline bool edges_misaligned(const int32_t *E)
{
    return (reinterpret_cast<uintptr_t>(E) & 7) != 0;
}

// Y, weights, counts and Z are read and written as 4-byte words (or wider,
// where the address allows).
inline bool words_misaligned(const void *a, const void *b = nullptr,
                             const void *c = nullptr)
{
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
             reinterpret_cast<uintptr_t>(c)) & 3) != 0;
}

#define GEE_CHECK_CUDA(x)                                                      \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess)                                                 \
            return from_cuda(e_);                                              \
    } while (0)

// Scratch of one call: status word, n_k, compact labels (n + 16 bytes).
gee_status step_begin(Workspace &ws, int64_t n, int32_t K, DevStatus **st,
                      uint32_t **counts, uint8_t **Yc, cudaStream_t stream,
                      int32_t L = 1)
{
    GEE_CHECK_CUDA(ws.alloc((void **)st, sizeof(DevStatus)));
    GEE_CHECK_CUDA(ws.alloc((void **)counts,
                            sizeof(uint32_t) * (L * K > kMaxClasses
                                                    ? L * K
                                                    : kMaxClasses)));
    GEE_CHECK_CUDA(ws.alloc((void **)Yc,
                            (size_t)n * (L > 1 ? label_stride(L) : 1) + 16));
    {
        ProfScope p("k_status_init", stream);
        GEE_CHECK_CUDA(launch_status_init(*st, stream));
    }
    GEE_CHECK_CUDA(
        cudaMemsetAsync(*counts, 0, sizeof(uint32_t) * K * L, stream));
    return GEE_OK;
}

// S1 + S2: label check, class sizes, compact labels (in rank order when the
// graph has degree ranks).
gee_status labels_launch(const int32_t *Y, int64_t n, int32_t K,
                         const int32_t *rank, uint8_t *Yc, uint32_t *counts,
                         DevStatus *st, cudaStream_t stream)
{
    if (n > 0) {
        ProfScope p("k_labels", stream);
        GEE_CHECK_CUDA(launch_labels(Y, n, K, rank, Yc, counts, st, stream));
    }
    return GEE_OK;
}

gee_status labels_step(Workspace &ws, const int32_t *Y, int64_t n, int32_t K,
                       const int32_t *rank, DevStatus **st, uint32_t **counts,
                       uint8_t **Yc, cudaStream_t stream)
{
    gee_status rc = step_begin(ws, n, K, st, counts, Yc, stream);
    if (rc != GEE_OK)
        return rc;
    return labels_launch(Y, n, K, rank, *Yc, *counts, *st, stream);
}

// Fork/join of a side stream for work that overlaps the call's stream.
class SideStream {
  public:
    explicit SideStream(cudaStream_t main) : main_(main) {}
    ~SideStream()
    {
        if (fork_)
            cudaEventDestroy(fork_);
        if (join_)
            cudaEventDestroy(join_);
        if (side_)
            cudaStreamDestroy(side_);  // released once its work is done
    }
    SideStream(const SideStream &) = delete;
    SideStream &operator=(const SideStream &) = delete;
    cudaError_t fork()
    {
        cudaError_t e = cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&join_, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventRecord(fork_, main_);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(side_, fork_, 0);
        return e;
    }
    cudaError_t join()
    {
        cudaError_t e = cudaEventRecord(join_, side_);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(main_, join_, 0);
        return e;
    }
    cudaStream_t stream() const { return side_; }

  private:
    cudaStream_t main_;
    cudaStream_t side_ = nullptr;
    cudaEvent_t fork_ = nullptr, join_ = nullptr;
};

// S4 + S5 over a CSR (resident or built for this call), for L label
// vectors of K classes (Z rows of L*K columns).  host_z: Z is page-locked
// host memory, so the row tiles are bound by the host link; they then run
// on a quarter of the SMs while the hub chunks run on the rest at the same
// time (partial sums only), and the fixup writes every hub row after both.
gee_status pull_step(Workspace &ws, const Csr &g, int32_t K, bool laplacian,
                     const uint8_t *Yc, const uint32_t *counts, float *Z,
                     const DevStatus *st, cudaStream_t stream, int32_t L = 1,
                     bool host_z = false, const int32_t *split = nullptr,
                     int64_t split_tiles = 0, bool fixed = false)
{
    // fixed: weighted arc values are added as 64-bit fixed-point integers
    const int shift = fixed ? fixed_shift(g, laplacian) : 0;
    const size_t part_cell = fixed ? 8 : 4;
    const int32_t cols = L * K;
    if (L >= kWideMinLabels) {
        if (fixed)
            return GEE_ERR_UNSUPPORTED;
        unsigned long long *work = nullptr;
        void *hub_part = nullptr;
        GEE_CHECK_CUDA(ws.alloc((void **)&work, sizeof(unsigned long long)));
        GEE_CHECK_CUDA(
            ws.alloc(&hub_part, part_cell * (g.chunks * cols + 1)));
        {
            ProfScope p("k_wide_rows", stream);
            GEE_CHECK_CUDA(launch_wide_rows(g, L, K, g.weighted, laplacian, Yc,
                                            counts, Z, work, st, stream));
        }
        if (g.chunks > 0) {
            ProfScope p("k_wide_chunks", stream);
            GEE_CHECK_CUDA(launch_wide_chunks(g, L, K, g.weighted, laplacian,
                                              Yc, counts, Z, hub_part, st,
                                              stream));
        }
        if (g.hubs > 0) {
            ProfScope p("k_hub_fixup", stream);
            GEE_CHECK_CUDA(launch_hub_fixup(g, cols, g.weighted, laplacian,
                                            counts, Z, hub_part, false, st,
                                            stream));
        }
        return GEE_OK;
    }
    // the row-tile partition: the graph's kept one, else split here
    int64_t ntiles = split_tiles;
    const int32_t *tile_row = split;
    void *hub_part = nullptr;
    unsigned long long *work = nullptr;
    GEE_CHECK_CUDA(ws.alloc((void **)&work, 2 * sizeof(unsigned long long)));
    GEE_CHECK_CUDA(
        ws.alloc(&hub_part, part_cell * (g.chunks * cols + 1)));
    if (tile_row == nullptr) {
        ntiles = pull_tiles(g, cols, host_z);
        int32_t *own = nullptr;
        GEE_CHECK_CUDA(ws.alloc((void **)&own, sizeof(int32_t) * (ntiles + 1)));
        ProfScope p("k_partition", stream);
        GEE_CHECK_CUDA(launch_partition(g, cols, own, ntiles, host_z, stream));
        tile_row = own;
    }
    if (host_z && g.chunks > 0) {
        const int sms = sm_count();
        const int light_ctas = sms / 4 > 0 ? sms / 4 : 1;
        // light rows on a quarter of the SMs; hub chunks, then every hub
        // row, on the rest -- the two sides write disjoint cells of Z, so
        // the hub rows cross the host link while the light rows do
        SideStream side(stream);
        GEE_CHECK_CUDA(side.fork());
        {
            ProfScope p("k_pull_heavy", side.stream());
            GEE_CHECK_CUDA(launch_pull_heavy(g, L, K, g.weighted, laplacian, Yc,
                                             counts, Z, hub_part, true, work + 1,
                                             st, side.stream(),
                                             sms - light_ctas, fixed, shift));
        }
        {
            ProfScope p("k_hub_fixup", side.stream());
            GEE_CHECK_CUDA(launch_hub_fixup(g, cols, g.weighted, laplacian,
                                            counts, Z, hub_part, true, st,
                                            side.stream(), fixed, shift));
        }
        {
            ProfScope p("k_pull_light", stream);
            GEE_CHECK_CUDA(launch_pull_light(g, L, K, g.weighted, laplacian,
                                             tile_row, ntiles, Yc, counts, Z,
                                             work, st, stream, light_ctas,
                                             true, fixed, shift));
        }
        GEE_CHECK_CUDA(side.join());
        return GEE_OK;
    }
    {
        ProfScope p("k_pull_light", stream);
        GEE_CHECK_CUDA(launch_pull_light(g, L, K, g.weighted, laplacian,
                                         tile_row, ntiles, Yc, counts, Z,
                                         work, st, stream, 0, host_z, fixed,
                                         shift));
    }
    if (g.chunks > 0) {
        ProfScope p("k_pull_heavy", stream);
        GEE_CHECK_CUDA(launch_pull_heavy(g, L, K, g.weighted, laplacian, Yc,
                                         counts, Z, hub_part, false, work + 1,
                                         st, stream, 0, fixed, shift));
    }
    if (g.hubs > 0) {
        ProfScope p("k_hub_fixup", stream);
        GEE_CHECK_CUDA(launch_hub_fixup(g, cols, g.weighted, laplacian, counts,
                                        Z, hub_part, false, st, stream, fixed,
                                        shift));
    }
    return GEE_OK;
}

// Edge-list embedding on device buffers; the caller reads the status.
gee_status embed_coo(Workspace &ws, const int32_t *E, const float *w,
                     int64_t s, const int32_t *Y, int64_t n, int32_t K,
                     int32_t laplacian, float *Z, const gee_options &o,
                     cudaStream_t stream, DevStatus **st_out)
{
    DevStatus *st;
    uint32_t *counts;
    uint8_t *Yc;
    gee_status rc = step_begin(ws, n, K, &st, &counts, &Yc, stream);
    *st_out = st;
    if (rc != GEE_OK)
        return rc;
    const gee_strategy strat = gee_pick_strategy(s, n, K, &o);
    int threads = o.block != 0 ? o.block : 256;
    if (o.strategy == GEE_AUTO && o.block == 0) {
        gee_strategy tuned;
        int32_t block = 0;
        if (tuned_choice(s, n, K, &tuned, &block) && tuned == strat && block != 0)
            threads = block;
    }
    if (strat == GEE_BINNED) {
        rc = labels_launch(Y, n, K, nullptr, Yc, counts, st, stream);
        if (rc != GEE_OK)
            return rc;
        float *r = nullptr;
        if (laplacian) {
            double *d;
            GEE_CHECK_CUDA(ws.alloc((void **)&d, sizeof(double) * (n + 1)));
            GEE_CHECK_CUDA(ws.alloc((void **)&r, sizeof(float) * (n + 1)));
            GEE_CHECK_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (n + 1), stream));
            if (s > 0) {
                ProfScope p("k_degree", stream);
                GEE_CHECK_CUDA(launch_degree(E, w, s, n, d, st, stream));
            }
            if (n > 0) {
                ProfScope p("k_rsqrt", stream);
                GEE_CHECK_CUDA(launch_rsqrt(d, n, r, st, stream));
            }
        }
        GEE_CHECK_CUDA(launch_binned(ws, E, w, s, n, K, Yc, r, counts, Z, st,
                                     stream));
        return GEE_OK;
    }
    if (strat == GEE_SEGMENTED) {
        Csr g;
        GEE_CHECK_CUDA(build_csr(E, w, s, n, ws, ws, g, st, stream));
        rc = labels_launch(Y, n, K, g.rank, Yc, counts, st, stream);
        if (rc != GEE_OK)
            return rc;
        rc = read_status(st, stream);
        if (rc != GEE_OK)
            return rc;
        if (laplacian) {
            if (g.negative_weight)
                return GEE_ERR_INVALID_ARG;
            GEE_CHECK_CUDA(build_laplacian_values(g, ws, ws, stream));
        }
        return pull_step(ws, g, K, laplacian != 0, Yc, counts, Z, st, stream,
                         1, false, nullptr, 0,
                         o.deterministic != 0 && (w != nullptr || laplacian));
    }
    rc = labels_launch(Y, n, K, nullptr, Yc, counts, st, stream);
    if (rc != GEE_OK)
        return rc;
    float *r = nullptr;
    bool check = false;
    if (laplacian) {
        double *d;
        GEE_CHECK_CUDA(ws.alloc((void **)&d, sizeof(double) * (n + 1)));
        GEE_CHECK_CUDA(ws.alloc((void **)&r, sizeof(float) * (n + 1)));
        GEE_CHECK_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (n + 1), stream));
        if (s > 0) {
            ProfScope p("k_degree", stream);
            GEE_CHECK_CUDA(launch_degree(E, w, s, n, d, st, stream));
        }
        if (n > 0) {
            ProfScope p("k_rsqrt", stream);
            GEE_CHECK_CUDA(launch_rsqrt(d, n, r, st, stream));
        }
    } else if (o.validate_edges) {
        if (s > 0) {
            ProfScope p("k_validate_edges", stream);
            GEE_CHECK_CUDA(launch_validate_edges(E, s, n, st, stream));
        }
    } else {
        check = true;
    }
    if (n > 0) {
        ProfScope p("k_zero", stream);
        GEE_CHECK_CUDA(launch_zero(Z, n * K, st, stream));
    }
    if (s > 0) {
        ProfScope p(strat == GEE_PRIVATE ? "k_scatter_private"
                                         : "k_scatter_atomic",
                    stream);
        if (strat == GEE_PRIVATE)
            GEE_CHECK_CUDA(launch_scatter_private(E, w, r, s, n, K, Yc, Z,
                                                  check, threads, st, stream));
        else
            GEE_CHECK_CUDA(launch_scatter_atomic(E, w, r, s, n, K, Yc, Z,
                                                 check, threads, st, stream));
    }
    if (n > 0) {
        ProfScope p("k_finalize", stream);
        if (w != nullptr || laplacian)
            GEE_CHECK_CUDA(
                launch_finalize_weighted(Z, r, n, K, counts, st, stream));
        else
            GEE_CHECK_CUDA(launch_finalize_count(Z, n, K, counts, st, stream));
    }
    return GEE_OK;
}

}  // namespace

int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return 148;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_sms[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount,
                                   dev) != cudaSuccess ||
            sms <= 0)
            sms = 148;
        g_sms[dev] = sms;
    }
    return g_sms[dev];
}

bool injected_alloc_failure()
{
    int32_t left = g_fail_allocs.load(std::memory_order_relaxed);
    while (left > 0)
        if (g_fail_allocs.compare_exchange_weak(left, left - 1))
            return true;
    return false;
}

int max_block_smem()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return 48 << 10;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_smem[dev] == 0) {
        int b = 0;
        if (cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                   dev) != cudaSuccess ||
            b <= 0)
            b = 48 << 10;
        g_smem[dev] = b;
    }
    return g_smem[dev];
}

}  // namespace gee

using namespace gee;

struct gee_graph {
    int device = 0;
    Csr csr;
    std::vector<void *> owned;
    std::mutex mu;
    bool lap_ready = false;
    cudaEvent_t lap_done = nullptr;
    // row-tile partitions already computed, by Z columns and tile shape:
    // they depend on the graph alone, so passes with the same K reuse them
    struct TileSplit {
        int32_t cols = 0;
        bool host_z = false;
        int64_t ntiles = 0;
        int32_t *tile_row = nullptr;
        cudaEvent_t ready = nullptr;
    };
    std::vector<TileSplit> splits;
};

namespace {

gee_status ensure_laplacian(gee_graph *g, cudaStream_t stream)
{
    std::lock_guard<std::mutex> lock(g->mu);
    if (g->csr.negative_weight)
        return GEE_ERR_INVALID_ARG;
    if (!g->lap_ready) {
        Workspace ws(stream);
        GraphAllocator keep(&g->owned);
        GEE_CHECK_CUDA(build_laplacian_values(g->csr, keep, ws, stream));
        GEE_CHECK_CUDA(cudaEventRecord(g->lap_done, stream));
        g->lap_ready = true;
    }
    GEE_CHECK_CUDA(cudaStreamWaitEvent(stream, g->lap_done, 0));
    return GEE_OK;
}

constexpr size_t kMaxSplits = 8;

// The graph's row-tile partition for `cols` Z columns, computed on first
// use (on `stream`, which later users wait for); null (the pass splits
// its own) once kMaxSplits partitions are kept.
gee_status tile_split(gee_graph *g, int32_t cols, bool host_z,
                      cudaStream_t stream, const int32_t **tile_row,
                      int64_t *ntiles)
{
    *tile_row = nullptr;
    *ntiles = 0;
    std::lock_guard<std::mutex> lock(g->mu);
    for (const gee_graph::TileSplit &t : g->splits)
        if (t.cols == cols && t.host_z == host_z) {
            GEE_CHECK_CUDA(cudaStreamWaitEvent(stream, t.ready, 0));
            *tile_row = t.tile_row;
            *ntiles = t.ntiles;
            return GEE_OK;
        }
    if (g->splits.size() >= kMaxSplits)
        return GEE_OK;
    gee_graph::TileSplit t;
    t.cols = cols;
    t.host_z = host_z;
    t.ntiles = pull_tiles(g->csr, cols, host_z);
    GraphAllocator keep(&g->owned);
    GEE_CHECK_CUDA(keep.alloc((void **)&t.tile_row,
                              sizeof(int32_t) * (t.ntiles + 1)));
    GEE_CHECK_CUDA(cudaEventCreateWithFlags(&t.ready, cudaEventDisableTiming));
    g->splits.push_back(t);  // the event is destroyed with the graph
    {
        ProfScope p("k_partition", stream);
        GEE_CHECK_CUDA(launch_partition(g->csr, cols, t.tile_row, t.ntiles,
                                        host_z, stream));
    }
    GEE_CHECK_CUDA(cudaEventRecord(t.ready, stream));
    *tile_row = t.tile_row;
    *ntiles = t.ntiles;
    return GEE_OK;
}

}  // namespace

bool gee::graph_weighted(const gee_graph *graph) { return graph->csr.weighted; }

uint32_t gee::graph_max_degree(const gee_graph *graph) { return graph->csr.max_deg; }

gee_status gee::graph_pass_enqueue(Workspace &ws, gee_graph *graph,
                                   const int32_t *Y, int32_t L, int32_t K,
                                   int32_t laplacian, float *Z,
                                   DevStatus **st_out, cudaStream_t stream,
                                   bool host_z, bool deterministic)
{
    // bit-reproducible float sums: fixed-point accumulation (single pass
    // forms); counts are exact already
    const bool fixed = deterministic && (graph->csr.weighted || laplacian);
    if (fixed && L >= kWideMinLabels)
        return GEE_ERR_UNSUPPORTED;
    if (laplacian) {
        gee_status rc = ensure_laplacian(graph, stream);
        if (rc != GEE_OK)
            return rc;
    }
    DevStatus *st;
    uint32_t *counts;
    uint8_t *Yc;
    gee_status rc;
    if (L == 1) {
        rc = labels_step(ws, Y, graph->csr.n, K, graph->csr.rank, &st, &counts,
                         &Yc, stream);
    } else {
        rc = step_begin(ws, graph->csr.n, K, &st, &counts, &Yc, stream, L);
        if (rc == GEE_OK && graph->csr.n > 0) {
            ProfScope p("k_labels_multi", stream);
            GEE_CHECK_CUDA(launch_labels_multi(Y, graph->csr.n, L, K,
                                               graph->csr.rank, Yc, counts, st,
                                               stream));
        }
    }
    if (rc != GEE_OK)
        return rc;
    *st_out = st;
    const int32_t *tile_row = nullptr;
    int64_t ntiles = 0;
    if (L < kWideMinLabels) {
        rc = tile_split(graph, L * K, host_z, stream, &tile_row, &ntiles);
        if (rc != GEE_OK)
            return rc;
    }
    return pull_step(ws, graph->csr, K, laplacian != 0, Yc, counts, Z, st,
                     stream, L, host_z, tile_row, ntiles, fixed);
}

namespace {

gee_status embed_graph_dev(Workspace &ws, gee_graph *graph, const int32_t *Y,
                           int32_t K, int32_t laplacian, float *Z,
                           cudaStream_t stream, int32_t L = 1,
                           bool host_z = false, bool deterministic = false)
{
    DevStatus *st = nullptr;
    gee_status rc = graph_pass_enqueue(ws, graph, Y, L, K, laplacian, Z, &st,
                                       stream, host_z, deterministic);
    if (rc != GEE_OK)
        return rc;
    return read_status(st, stream);
}

}  // namespace

extern "C" {

void gee_debug_fail_allocs(int32_t count)
{
    gee::g_fail_allocs.store(count > 0 ? count : 0);
}

void gee_options_default(gee_options *opts)
{
    if (opts == nullptr)
        return;
    opts->strategy = GEE_AUTO;
    opts->validate_edges = 1;
    opts->private_max_cells = 0;
    opts->block = 0;
    opts->deterministic = 0;
}

const char *gee_status_string(gee_status status)
{
    switch (status) {
    case GEE_OK: return "ok";
    case GEE_ERR_INVALID_ARG: return "invalid argument";
    case GEE_ERR_LABEL_RANGE: return "label outside [-1, K)";
    case GEE_ERR_NODE_RANGE: return "edge endpoint outside [0, n)";
    case GEE_ERR_OVERFLOW: return "size overflows the index types";
    case GEE_ERR_OOM: return "out of device memory";
    case GEE_ERR_CUDA: return "CUDA runtime error";
    case GEE_ERR_TIMEOUT: return "device wait timed out";
    case GEE_ERR_UNSUPPORTED: return "unsupported argument";
    case GEE_ERR_CANCELLED: return "request cancelled";
    }
    return "unknown status";
}

gee_strategy gee_pick_strategy(int64_t s, int64_t n, int32_t K,
                               const gee_options *opts)
{
    const gee_options o = resolve_options(opts);
    const int64_t limit = private_cells_limit();
    const int64_t cells = n * (int64_t)K;
    if (o.strategy == GEE_PRIVATE && cells > limit)
        return GEE_ATOMIC;  // the copy would not fit in shared memory
    if (o.strategy == GEE_BINNED && !binned_fits(n, K))
        return GEE_ATOMIC;  // beyond the two-level layout of row tiles
    if (o.strategy != GEE_AUTO)
        return static_cast<gee_strategy>(o.strategy);
    // past the tuning grid: a Z this large misses L2, so pushing updates
    // into it costs a DRAM read-modify-write each
    if (cells > kBinnedMinCells && binned_fits(n, K))
        return GEE_BINNED;
    gee_strategy tuned;
    int32_t tuned_block = 0;
    if (tuned_choice(s, n, K, &tuned, &tuned_block))
        return tuned == GEE_PRIVATE && cells > limit ? GEE_ATOMIC : tuned;
    const int64_t cap =
        o.private_max_cells > 0 && o.private_max_cells < limit
            ? o.private_max_cells
            : limit;
    // PRIVATE pays once every SM's CTA has several edges per cell to merge.
    if (cells <= cap && 2 * s >= 4 * cells * (int64_t)sm_count())
        return GEE_PRIVATE;
    return GEE_ATOMIC;
}

size_t gee_workspace_bytes(int64_t s, int64_t n, int32_t K, int32_t weighted,
                           int32_t laplacian, const gee_options *opts)
{
    size_t b = 4096 + (size_t)n + 16 + 256 * 4;
    const gee_strategy st = gee_pick_strategy(s, n, K, opts);
    if (laplacian)
        b += (size_t)(n + 1) * 12;
    if (st == GEE_BINNED) {
        const bool wt = weighted || laplacian;
        const int32_t rows = bin_rows(K, wt);
        b += bin_scratch_bytes(2 * s, (n + rows - 1) / rows, wt) + 512;
    }
    if (st == GEE_SEGMENTED) {
        b += (size_t)(n + 1) * (8 * 4 + 4 * 4);  // rowptr, scan and fill temps
        b += (size_t)(2 * s + 8) * 4 * (weighted || laplacian ? 3 : 1);
        b += (size_t)((2 * s + n * K) / kTileUnits + 2) * 4;
        b += (size_t)((2 * s) / kHubDegree + 2) * ((size_t)K * 4 + 12);
    }
    return b;
}

gee_status gee_histogram(const int32_t *Y, int64_t n, int32_t K,
                         uint32_t *counts, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    gee_status rc = check_common(0, n, K, 0);
    if (rc != GEE_OK)
        return rc;
    if (counts == nullptr || (n > 0 && Y == nullptr) ||
        words_misaligned(counts, Y))
        return GEE_ERR_INVALID_ARG;
    gee_status out;
    {
        Workspace ws(stream);
        DevStatus *st;
        uint32_t *c;
        uint8_t *Yc;
        rc = labels_step(ws, Y, n, K, nullptr, &st, &c, &Yc, stream);
        if (rc != GEE_OK)
            return rc;
        cudaError_t e = cudaMemcpyAsync(counts, c, sizeof(uint32_t) * K,
                                        cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess)
            return from_cuda(e);
        out = read_status(st, stream);
    }
    return out;
}

gee_status gee_embed(const int32_t *edges, const float *weights, int64_t s,
                     const int32_t *Y, int64_t n, int32_t K, int32_t laplacian,
                     float *Z, const gee_options *opts, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const gee_options o = resolve_options(opts);
    gee_status rc = check_common(s, n, K, o.block);
    if (rc != GEE_OK)
        return rc;
    if ((s > 0 && edges == nullptr) || (n > 0 && (Y == nullptr || Z == nullptr)))
        return GEE_ERR_INVALID_ARG;
    if (edges_misaligned(edges) || words_misaligned(weights, Y, Z))
        return GEE_ERR_INVALID_ARG;
    if (s > 0 && n == 0)
        return GEE_ERR_NODE_RANGE;
    if (o.strategy < GEE_AUTO || o.strategy > GEE_BINNED)
        return GEE_ERR_INVALID_ARG;
    gee_options oo = o;
    rc = deterministic_strategy(oo, weights != nullptr, laplacian);
    if (rc != GEE_OK)
        return rc;
    Workspace ws(stream);
    DevStatus *st = nullptr;
    rc = embed_coo(ws, edges, weights, s, Y, n, K, laplacian, Z, oo, stream,
                   &st);
    if (rc != GEE_OK)
        return rc;
    return read_status(st, stream);
}

gee_status gee_embed_host(const int32_t *edges_h, const float *weights_h,
                          int64_t s, const int32_t *Y_h, int64_t n, int32_t K,
                          int32_t laplacian, float *Z_h,
                          const gee_options *opts, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    gee_options o = resolve_options(opts);
    gee_status rc = check_common(s, n, K, o.block);
    if (rc != GEE_OK)
        return rc;
    if ((s > 0 && edges_h == nullptr) ||
        (n > 0 && (Y_h == nullptr || Z_h == nullptr)))
        return GEE_ERR_INVALID_ARG;
    if (s > 0 && n == 0)
        return GEE_ERR_NODE_RANGE;
    if (o.strategy < GEE_AUTO || o.strategy > GEE_BINNED)
        return GEE_ERR_INVALID_ARG;
    rc = deterministic_strategy(o, weights_h != nullptr, laplacian);
    if (rc != GEE_OK)
        return rc;
    Workspace ws(stream);
    int32_t *E = nullptr, *Y = nullptr;
    float *w = nullptr, *Z = nullptr;
    GEE_CHECK_CUDA(ws.alloc((void **)&E, sizeof(int32_t) * 2 * (s + 1)));
    GEE_CHECK_CUDA(ws.alloc((void **)&Y, sizeof(int32_t) * (n + 1)));
    GEE_CHECK_CUDA(ws.alloc((void **)&Z, sizeof(float) * (n * K + 1)));
    GEE_CHECK_CUDA(cudaMemcpyAsync(E, edges_h, sizeof(int32_t) * 2 * s,
                                   cudaMemcpyHostToDevice, stream));
    GEE_CHECK_CUDA(cudaMemcpyAsync(Y, Y_h, sizeof(int32_t) * n,
                                   cudaMemcpyHostToDevice, stream));
    if (weights_h != nullptr) {
        GEE_CHECK_CUDA(ws.alloc((void **)&w, sizeof(float) * (s + 1)));
        GEE_CHECK_CUDA(cudaMemcpyAsync(w, weights_h, sizeof(float) * s,
                                       cudaMemcpyHostToDevice, stream));
    }
    DevStatus *st = nullptr;
    rc = embed_coo(ws, E, w, s, Y, n, K, laplacian, Z, o, stream, &st);
    if (rc != GEE_OK)
        return rc;
    rc = read_status(st, stream);
    if (rc != GEE_OK)
        return rc;
    GEE_CHECK_CUDA(cudaMemcpyAsync(Z_h, Z, sizeof(float) * n * K,
                                   cudaMemcpyDeviceToHost, stream));
    GEE_CHECK_CUDA(cudaStreamSynchronize(stream));
    return GEE_OK;
}

void gee_graph_destroy(gee_graph *graph)
{
    if (graph == nullptr)
        return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(graph->device);
    cudaDeviceSynchronize();
    for (void *p : graph->owned)
        cudaFree(p);
    if (graph->lap_done)
        cudaEventDestroy(graph->lap_done);
    for (const gee_graph::TileSplit &t : graph->splits)
        if (t.ready)
            cudaEventDestroy(t.ready);
    cudaSetDevice(prev);
    delete graph;
}

gee_status gee_embed_batch(const gee_problem *problems, int32_t count,
                           gee_status *statuses, const gee_options *opts,
                           gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (count < 0 || (count > 0 && problems == nullptr))
        return GEE_ERR_INVALID_ARG;
    const gee_options o = resolve_options(opts);
    std::vector<BatchProblem> P((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        const gee_problem &q = problems[i];
        gee_status rc = check_common(q.s, q.n, q.K, 0);
        if (rc == GEE_OK &&
            ((q.s > 0 && q.edges == nullptr) ||
             (q.n > 0 && (q.Y == nullptr || q.Z == nullptr)) ||
             edges_misaligned(q.edges) ||
             words_misaligned(q.weights, q.Y, q.Z) || q.reserved != 0))
            rc = GEE_ERR_INVALID_ARG;
        if (rc == GEE_OK && q.s > 0 && q.n == 0)
            rc = GEE_ERR_NODE_RANGE;
        if (rc == GEE_OK && o.deterministic && q.weights != nullptr)
            rc = GEE_ERR_UNSUPPORTED;  // float sums in scheduling order
        if (rc != GEE_OK) {
            if (statuses != nullptr)
                statuses[i] = rc;
            return rc;
        }
        BatchProblem &p = P[(size_t)i];
        p = BatchProblem{};
        p.E = q.edges;
        p.w = q.weights;
        p.Y = q.Y;
        p.Z = q.Z;
        p.s = q.s;
        p.n = q.n;
        p.K = q.K;
    }
    if (count == 0)
        return GEE_OK;
    BatchHeader hh{};
    batch_layout(P.data(), count, hh);
    Workspace ws(stream);
    BatchHeader *dh = nullptr;
    BatchProblem *dP = nullptr;
    DevStatus *st = nullptr;
    uint32_t *counts = nullptr;
    uint8_t *Yc = nullptr;
    GEE_CHECK_CUDA(ws.alloc((void **)&dh, sizeof(BatchHeader)));
    GEE_CHECK_CUDA(ws.alloc((void **)&dP, sizeof(BatchProblem) * count));
    GEE_CHECK_CUDA(ws.alloc((void **)&st, sizeof(DevStatus) * count));
    GEE_CHECK_CUDA(ws.alloc((void **)&counts, sizeof(uint32_t) * hh.count_cells));
    GEE_CHECK_CUDA(ws.alloc((void **)&Yc, (size_t)hh.yc_bytes + 16));
    for (int32_t i = 0; i < count; ++i) {
        BatchProblem &p = P[(size_t)i];
        p.st = st + i;
        p.counts = counts + p.counts_off;
        p.Yc = Yc + p.yc_off;
    }
    hh.counts = counts;
    GEE_CHECK_CUDA(cudaMemcpyAsync(dh, &hh, sizeof(hh), cudaMemcpyHostToDevice,
                                   stream));
    GEE_CHECK_CUDA(cudaMemcpyAsync(dP, P.data(), sizeof(BatchProblem) * count,
                                   cudaMemcpyHostToDevice, stream));
    // the edge pass: binned (records grouped by row tile, no atomics on Z)
    // when most of the batch's cells belong to problems whose Z is beyond
    // 2^24 cells, else pushed into Z with atomics -- problems taken in
    // order keep a small Z in L2 while its atomics land (4,096 graphs of
    // 1e3-1e5 nodes: 39.6 ms pushed, 60.0 ms binned)
    const bool binned =
        (o.strategy == GEE_BINNED ||
         (o.strategy == GEE_AUTO && batch_prefers_binned(P.data(), count))) &&
        binned_batch_tiles(P.data(), count) > 0;
    if (binned) {
        GEE_CHECK_CUDA(batch_labels_enqueue(dh, dP, stream));
        GEE_CHECK_CUDA(launch_binned_batch(ws, P.data(), count, stream));
    } else {
        GEE_CHECK_CUDA(batch_enqueue(dh, dP, hh, o.validate_edges != 0, stream));
    }
    std::vector<DevStatus> hs((size_t)count);
    GEE_CHECK_CUDA(cudaMemcpyAsync(hs.data(), st, sizeof(DevStatus) * count,
                                   cudaMemcpyDeviceToHost, stream));
    GEE_CHECK_CUDA(cudaStreamSynchronize(stream));
    gee_status first = GEE_OK;
    for (int32_t i = 0; i < count; ++i) {
        const gee_status r = static_cast<gee_status>(hs[(size_t)i].code);
        if (statuses != nullptr)
            statuses[i] = r;
        if (first == GEE_OK)
            first = r;
    }
    return first;
}

gee_status gee_graph_create(const int32_t *edges, const float *weights,
                            int64_t s, int64_t n, gee_stream_t stream_,
                            gee_graph **out)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (out == nullptr)
        return GEE_ERR_INVALID_ARG;
    *out = nullptr;
    gee_status rc = check_common(s, n, 1, 0);
    if (rc != GEE_OK)
        return rc;
    if ((s > 0 && edges == nullptr) || edges_misaligned(edges) ||
        words_misaligned(weights))
        return GEE_ERR_INVALID_ARG;
    if (s > 0 && n == 0)
        return GEE_ERR_NODE_RANGE;
    gee_graph *g = new gee_graph();
    cudaGetDevice(&g->device);
    gee_status result;
    {
        Workspace ws(stream);
        GraphAllocator keep(&g->owned);
        DevStatus *st = nullptr;
        cudaError_t e = ws.alloc((void **)&st, sizeof(DevStatus));
        if (e == cudaSuccess)
            e = launch_status_init(st, stream);
        if (e == cudaSuccess)
            e = build_csr(edges, weights, s, n, keep, ws, g->csr, st, stream);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&g->lap_done,
                                         cudaEventDisableTiming);
        result = (e == cudaSuccess) ? read_status(st, stream) : from_cuda(e);
    }
    if (result != GEE_OK) {
        gee_graph_destroy(g);
        return result;
    }
    *out = g;
    return GEE_OK;
}

gee_status gee_graph_info(const gee_graph *graph, int64_t *n, int64_t *s,
                          int64_t *hub_rows, int64_t *hub_arcs,
                          int64_t *device_bytes)
{
    if (graph == nullptr)
        return GEE_ERR_INVALID_ARG;
    const Csr &c = graph->csr;
    if (n)
        *n = c.n;
    if (s)
        *s = c.s;
    if (hub_rows)
        *hub_rows = c.hubs;
    if (hub_arcs)
        *hub_arcs = c.hub_arcs;
    if (device_bytes) {
        int64_t b = (c.n + 1) * 8 + (c.nnz_main + 4) * 4 + (c.hub_arcs + 4) * 4;
        if (c.weighted)
            b += (c.nnz_main + c.hub_arcs + 8) * 4;
        if (c.lap_val)
            b += (c.nnz_main + c.hub_arcs + 8) * 4;
        b += c.hubs * 16 + c.chunks * 12 + (c.n + 1) * 4 +
             ((c.n + 31) / 32 + 1) * 4;
        *device_bytes = b;
    }
    return GEE_OK;
}

gee_status gee_graph_gathers(const gee_graph *graph, int32_t K,
                             int64_t *hub_shared, int64_t *hub_other,
                             int64_t *light, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (graph == nullptr || K < 1 || K > kMaxClasses)
        return GEE_ERR_INVALID_ARG;
    const Csr &c = graph->csr;
    unsigned long long hs = 0ull;
    {
        Workspace ws(stream);
        unsigned long long *d = nullptr;
        GEE_CHECK_CUDA(ws.alloc((void **)&d, sizeof(unsigned long long)));
        GEE_CHECK_CUDA(count_hub_shared_arcs(c, K, d, stream));
        GEE_CHECK_CUDA(cudaMemcpyAsync(&hs, d, sizeof(hs),
                                       cudaMemcpyDeviceToHost, stream));
        GEE_CHECK_CUDA(cudaStreamSynchronize(stream));
    }
    if (hub_shared)
        *hub_shared = (int64_t)hs;
    if (hub_other)
        *hub_other = c.hub_arcs - (int64_t)hs;
    if (light)
        *light = c.nnz_main;
    return GEE_OK;
}

gee_status gee_embed_graph(gee_graph *graph, const int32_t *Y, int32_t K,
                           int32_t laplacian, float *Z,
                           const gee_options *opts, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (graph == nullptr)
        return GEE_ERR_INVALID_ARG;
    const gee_options o = resolve_options(opts);
    gee_status rc = check_common(0, graph->csr.n, K, o.block);
    if (rc != GEE_OK)
        return rc;
    if ((graph->csr.n > 0 && (Y == nullptr || Z == nullptr)) ||
        words_misaligned(Y, Z))
        return GEE_ERR_INVALID_ARG;
    Workspace ws(stream);
    return embed_graph_dev(ws, graph, Y, K, laplacian, Z, stream, 1, false,
                           o.deterministic != 0);
}

gee_status gee_embed_graph_multi(gee_graph *graph, const int32_t *Y,
                                 int32_t L, int32_t K, int32_t laplacian,
                                 float *Z, const gee_options *opts,
                                 gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (graph == nullptr || L < 1)
        return GEE_ERR_INVALID_ARG;
    const gee_options o = resolve_options(opts);
    gee_status rc = check_common(0, graph->csr.n, K, o.block);
    if (rc != GEE_OK)
        return rc;
    if ((int64_t)L * K > GEE_MAX_COLUMNS)
        return GEE_ERR_UNSUPPORTED;
    if ((graph->csr.n > 0 && (Y == nullptr || Z == nullptr)) ||
        words_misaligned(Y, Z))
        return GEE_ERR_INVALID_ARG;
    Workspace ws(stream);
    return embed_graph_dev(ws, graph, Y, K, laplacian, Z, stream, L, false,
                           o.deterministic != 0);
}

gee_status gee_embed_graph_host(gee_graph *graph, const int32_t *Y_h,
                                int32_t K, int32_t laplacian, float *Z_h,
                                const gee_options *opts, gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (graph == nullptr)
        return GEE_ERR_INVALID_ARG;
    const gee_options o = resolve_options(opts);
    const int64_t n = graph->csr.n;
    gee_status rc = check_common(0, n, K, o.block);
    if (rc != GEE_OK)
        return rc;
    if (n > 0 && (Y_h == nullptr || Z_h == nullptr))
        return GEE_ERR_INVALID_ARG;
    Workspace ws(stream);
    int32_t *Y = nullptr;
    GEE_CHECK_CUDA(ws.alloc((void **)&Y, sizeof(int32_t) * (n + 1)));
    GEE_CHECK_CUDA(cudaMemcpyAsync(Y, Y_h, sizeof(int32_t) * n,
                                   cudaMemcpyHostToDevice, stream));
    // A page-locked Z_h is written by the pass itself over the host link, so
    // the transfer overlaps the pass instead of following it; labels are
    // checked before any Z row is written, so Z_h stays untouched on error.
    float *Zdirect = mapped_host(Z_h);
    if (Zdirect != nullptr)
        return embed_graph_dev(ws, graph, Y, K, laplacian, Zdirect, stream, 1,
                               true, o.deterministic != 0);
    float *Z = nullptr;
    GEE_CHECK_CUDA(ws.alloc((void **)&Z, sizeof(float) * (n * K + 1)));
    rc = embed_graph_dev(ws, graph, Y, K, laplacian, Z, stream, 1, false,
                         o.deterministic != 0);
    if (rc != GEE_OK)
        return rc;
    GEE_CHECK_CUDA(cudaMemcpyAsync(Z_h, Z, sizeof(float) * n * K,
                                   cudaMemcpyDeviceToHost, stream));
    GEE_CHECK_CUDA(cudaStreamSynchronize(stream));
    return GEE_OK;
}

}  // extern "C"
