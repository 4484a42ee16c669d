// gee_internal.cuh -- shared device helpers and kernel launchers of libgee.
//
// Layout in device memory (see gee.h for the public contract):
//   Yc      uint8 [n]       compact labels, 255 = class unknown
//   counts  uint32 [K]      class sizes n_k
//   Z       float  [n][K]   row-major; the ATOMIC/PRIVATE count path uses the
//                           same bytes as uint32 counts before finalising
//   CSR     int64 rowptr[n+1], int32 col[], float val[] (resident graphs)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gee.h"

namespace gee {

constexpr uint32_t kNoLabel = 255;
constexpr int kMaxClasses = GEE_MAX_CLASSES;
// Row tiles of the pull pass cover kTileUnits "merged units": one unit per
// arc plus max(K, 16) units per row (the row's Z write), so that every tile
// moves about the same number of bytes.  Rows with more than kHubDegree arcs
// are processed apart, in chunks of kHubChunk arcs.
constexpr int kTileUnits = 1024;
constexpr int kHubDegree = GEE_HUB_DEGREE;
constexpr int kHubChunk = 2048;

// First error a kernel saw.  `index` is the smallest offending element.
struct DevStatus {
    int32_t code;
    int32_t aux;
    unsigned long long index;
};

__device__ __forceinline__ void report(DevStatus *st, int code,
                                       unsigned long long index)
{
    atomicCAS(&st->code, 0, code);
    atomicMin(&st->index, index);
}

__device__ __forceinline__ bool failed(const DevStatus *st)
{
    return *reinterpret_cast<const volatile int32_t *>(&st->code) != 0;
}

// L2 eviction policies (PTX createpolicy): labels are gathered at random and
// should stay in L2; edges, arcs and Z rows stream through once.
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint32_t load_label(const uint8_t *p, uint64_t pol)
{
    uint32_t r;
    asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;"
        : "=r"(r)
        : "l"(p), "l"(pol));
    return r;
}

// Z value of a class count: RN32(c / n_k).  Exact float division when both
// operands are below 2^24 (exactly representable); otherwise the quotient is
// formed in double and rounded once more to float.
__device__ __forceinline__ float count_to_z(uint32_t c, uint32_t nk)
{
    if (c == 0u)
        return 0.0f;
    if ((c | nk) < (1u << 24))
        return __fdiv_rn(static_cast<float>(c), static_cast<float>(nk));
    return __double2float_rn(
        __ddiv_rn(static_cast<double>(c), static_cast<double>(nk)));
}

// Weighted/Laplacian cell: accumulated weight sum divided by n_k.
__device__ __forceinline__ float sum_to_z(float acc, uint32_t nk)
{
    if (nk == 0u)
        return 0.0f;
    return __fdiv_rn(acc, static_cast<float>(nk));
}

// Deterministic weighted cell: an exact sum of fixed-point arc values
// (multiples of inv = 2^-shift) divided by n_k in FP64, rounded once to
// float.  Integer sums do not depend on the order of the additions.
__device__ __forceinline__ float fixed_to_z(unsigned long long q, double inv,
                                            uint32_t nk)
{
    if (nk == 0u || q == 0ull)
        return 0.0f;
    return __double2float_rn(__ddiv_rn(
        static_cast<double>(static_cast<long long>(q)) * inv,
        static_cast<double>(nk)));
}

// Laplacian degree factor r = RN32(1/sqrt(d)) of an FP64 degree d: the
// square root and the reciprocal in FP64 (each correctly rounded), then
// one rounding to float; 0 for d <= 0 (a node without edges).
__device__ __forceinline__ float rsqrt_rn32(double d)
{
    if (!(d > 0.0))
        return 0.0f;
    return __double2float_rn(__ddiv_rn(1.0, __dsqrt_rn(d)));
}

inline int grid_for(int64_t work, int threads, int max_blocks)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1)
        b = 1;
    if (b > max_blocks)
        b = max_blocks;
    return static_cast<int>(b);
}

// Number of SMs of the current device (cached per device).
int sm_count();
// Dynamic shared memory one CTA may opt into on the current device.
int max_block_smem();

// True when gee_debug_fail_allocs asks the next allocation to fail (the
// request is consumed).
bool injected_alloc_failure();

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `stream` and return cudaGetLastError().

cudaError_t launch_status_init(DevStatus *st, cudaStream_t stream);

// S1 + S2: validate labels, write compact labels, class histogram.
// counts must be zeroed by the caller.  With rank != null the compact label
// of node i goes to Yc[rank[i]] (rank order), else to Yc[i].
cudaError_t launch_labels(const int32_t *Y, int64_t n, int32_t K,
                          const int32_t *rank, uint8_t *Yc, uint32_t *counts,
                          DevStatus *st, cudaStream_t stream);
// Bytes per node of the multi-label compact array: L padded to 4 or 8 for
// fewer than kWideMinLabels vectors, else to a multiple of 32 (one L2 sector
// per block of 32 labels), so a node's labels load as whole words.
constexpr int kWideMinLabels = 8;
inline int label_stride(int L)
{
    return L <= 4 ? 4 : (L < kWideMinLabels ? 8 : (L + 31) & ~31);
}
// The same for L label vectors Y[l*n + i]: Yc[rank[i]*Ls + l] (padding
// bytes hold 255, "unknown") and counts[l*K + k]; L*K <= GEE_MAX_COLUMNS.
cudaError_t launch_labels_multi(const int32_t *Y, int64_t n, int32_t L,
                                int32_t K, const int32_t *rank, uint8_t *Yc,
                                uint32_t *counts, DevStatus *st,
                                cudaStream_t stream);

cudaError_t launch_validate_edges(const int32_t *E, int64_t s, int64_t n,
                                  DevStatus *st, cudaStream_t stream);

// S3 (edge-list form): d[u] += w for both endpoints, checks endpoints and the
// sign of weights; then r[u] = 1/sqrt(d[u]) (0 for d = 0).
cudaError_t launch_degree(const int32_t *E, const float *w, int64_t s,
                          int64_t n, double *d, DevStatus *st,
                          cudaStream_t stream);
cudaError_t launch_rsqrt(const double *d, int64_t n, float *r,
                         const DevStatus *st, cudaStream_t stream);

cudaError_t launch_zero(void *p, int64_t words, const DevStatus *st,
                        cudaStream_t stream);

// S4 (edge-list form).  Count path: C (uint32, same bytes as Z) += 1.
// Weighted path: Z += w (times r of the sending node for the Laplacian).
cudaError_t launch_scatter_atomic(const int32_t *E, const float *w,
                                  const float *r, int64_t s, int64_t n,
                                  int32_t K, const uint8_t *Yc, void *Z,
                                  bool check_nodes, int threads, DevStatus *st,
                                  cudaStream_t stream);
cudaError_t launch_scatter_private(const int32_t *E, const float *w,
                                   const float *r, int64_t s, int64_t n,
                                   int32_t K, const uint8_t *Yc, void *Z,
                                   bool check_nodes, int threads,
                                   DevStatus *st, cudaStream_t stream);
int64_t private_cells_limit();

// S5 (edge-list form), in place over Z.
cudaError_t launch_finalize_count(void *Z, int64_t n, int32_t K,
                                  const uint32_t *counts, const DevStatus *st,
                                  cudaStream_t stream);
cudaError_t launch_finalize_weighted(float *Z, const float *r, int64_t n,
                                     int32_t K, const uint32_t *counts,
                                     const DevStatus *st, cudaStream_t stream);

// ------------------------------------------------------------ CSR (gee_csr)
struct Csr {
    int64_t n = 0, s = 0;
    int64_t nnz_main = 0;       // arcs of non-hub rows
    int64_t hubs = 0;           // rows with more than kHubDegree arcs
    int64_t chunks = 0;         // hub chunks of <= kHubChunk arcs
    int64_t hub_arcs = 0;
    bool weighted = false;
    int32_t negative_weight = 0;
    uint32_t max_deg = 0;       // arcs of the longest row
    float max_abs_w = 0.0f;     // largest |weight| (weighted graphs)
    int64_t *rowptr = nullptr;      // [n+1], hub rows empty
    int32_t *rank = nullptr;        // [n] degree rank of each node
    int32_t *col = nullptr;         // [nnz_main + pad] target ranks
    float *val = nullptr;           // [nnz_main + pad] or null
    int32_t *hub_row = nullptr;     // [hubs]
    uint32_t *hub_bits = nullptr;   // [n/32 + 1] bit i of word i/32: row i is a hub row
    int64_t *hub_ptr = nullptr;     // [hubs+1] into col_h
    int32_t *col_h = nullptr;       // [hub_arcs + pad]
    float *val_h = nullptr;
    int32_t *chunk_hub = nullptr;   // [chunks]
    int64_t *chunk_begin = nullptr; // [chunks]
    int32_t *hub_chunk0 = nullptr;  // [hubs+1] first chunk of each hub
    float *lap_val = nullptr;       // Laplacian arc values (lazy)
    float *lap_val_h = nullptr;
};

// Shift of the fixed-point form of a graph's arc values: every cell sums at
// most max_deg values of magnitude <= bound (|w|, or 1 for Laplacian values
// of non-negative weights), so cell sums stay below 2^62.
int fixed_shift(const Csr &g, bool laplacian);

// Allocation callback used by the CSR builder (pool or cudaMalloc).
struct Allocator {
    virtual cudaError_t alloc(void **p, size_t bytes) = 0;
    virtual ~Allocator() {}
};

gee_status from_cuda(cudaError_t e);

// The library's stream-ordered pool on the current device.  Freed blocks stay
// cached in the pool (release threshold = max) so repeated calls do not go
// back to the driver.
cudaError_t device_pool(cudaMemPool_t *out);

// Device address of page-locked (registered or cudaMallocHost) host memory,
// or null for pageable or unaligned memory.
float *mapped_host(float *p);

// Scratch of one call: stream-ordered allocations, released (to the pool) on
// the same stream when the Workspace is destroyed -- after the work enqueued
// before, so a Workspace may go out of scope as soon as its work is queued.
class Workspace : public Allocator {
  public:
    explicit Workspace(cudaStream_t s) : stream_(s) {}
    ~Workspace() override
    {
        for (void *p : ptrs_)
            cudaFreeAsync(p, stream_);
    }
    Workspace(const Workspace &) = delete;
    Workspace &operator=(const Workspace &) = delete;
    cudaError_t alloc(void **p, size_t bytes) override
    {
        if (injected_alloc_failure())
            return cudaErrorMemoryAllocation;
        if (!pool_) {
            cudaError_t e = device_pool(&pool_);
            if (e != cudaSuccess)
                return e;
        }
        if (bytes == 0)
            bytes = 16;
        // round up so vector accesses past the logical end stay inside
        bytes = (bytes + 255) & ~size_t(255);
        cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool_, stream_);
        if (e == cudaSuccess)
            ptrs_.push_back(*p);
        return e;
    }

  private:
    cudaStream_t stream_;
    cudaMemPool_t pool_ = nullptr;
    std::vector<void *> ptrs_;
};

// Builds the symmetric CSR of an edge list (validating endpoints into st).
// `persist` provides the arrays kept in g, `tmp` the scratch.  Synchronises
// the stream (twice) to size the arrays.
cudaError_t build_csr(const int32_t *E, const float *w, int64_t s, int64_t n,
                      Allocator &persist, Allocator &tmp, Csr &g,
                      DevStatus *st, cudaStream_t stream);

// Labels of ranks [0, hot_labels) are read from the hub kernel's shared
// copy for a pass of L label vectors of `classes` classes (*packed: as 6-bit
// codes, five per word).
int32_t hot_labels(int64_t n, int32_t L, int32_t classes, int32_t *packed);
// Hub-row arcs whose target's label the hub kernel takes from its
// shared-memory copy in a single-vector pass with K classes (*d_out,
// device, one counter).
cudaError_t count_hub_shared_arcs(const Csr &g, int32_t K,
                                  unsigned long long *d_out,
                                  cudaStream_t stream);

// Laplacian arc values w / sqrt(d_u d_v) from the CSR's row sums.
cudaError_t build_laplacian_values(Csr &g, Allocator &persist, Allocator &tmp,
                                   cudaStream_t stream);

// Row-tile partition for K: tile_row[ntiles+1].
int64_t pull_tiles(const Csr &g, int32_t K, bool host_z = false);
cudaError_t launch_partition(const Csr &g, int32_t K, int32_t *tile_row,
                             int64_t ntiles, bool host_z, cudaStream_t stream);

// S4 + S5 (CSR form), three launches in this order on one stream:
// light rows (every Z row of the tile range; hub rows get zeros), hub-row
// chunks (single-chunk hub rows written directly) and the fixup of hub rows
// with several chunks.  Yc is in rank order.  hub_part: scratch
// [chunks * K] of 4-byte per-chunk partial sums; work: an 8-byte scratch
// counter per launch (the light and the heavy launch each need their own).
// K arguments of the CSR launches count Z columns (L vectors x classes).
// ctas: persistent CTAs (0 = one per SM).  partials_only: k_pull_heavy
// leaves every chunk's sums in hub_part (never writing Z) and
// launch_hub_fixup(all_rows = true) writes every hub row -- so the two
// pull kernels may run at the same time on disjoint SMs.  host_z: Z is
// page-locked host memory written over the host link -- k_pull_light takes
// the larger tiles (fewer partial lines at tile ends; pull_tiles and
// launch_partition must be given the same flag) and leaves the cells of hub
// rows untouched instead of zeroing them, so launch_hub_fixup(all_rows =
// true) may run at the same time too.
cudaError_t launch_pull_light(const Csr &g, int32_t L, int32_t classes,
                              bool weighted, bool laplacian,
                              const int32_t *tile_row,
                              int64_t ntiles, const uint8_t *Yc,
                              const uint32_t *counts, float *Z,
                              unsigned long long *work, const DevStatus *st,
                              cudaStream_t stream, int ctas = 0,
                              bool host_z = false, bool fixed = false,
                              int shift = 0);
cudaError_t launch_pull_heavy(const Csr &g, int32_t L, int32_t classes,
                              bool weighted, bool laplacian, const uint8_t *Yc,
                              const uint32_t *counts, float *Z,
                              void *hub_part, bool partials_only,
                              unsigned long long *work, const DevStatus *st,
                              cudaStream_t stream, int ctas = 0,
                              bool fixed = false, int shift = 0);
// fixed (weighted passes): arc values are added as 64-bit fixed-point
// integers with `shift` fractional bits (fixed_shift), so every cell's sum
// is exact and independent of the order of the additions; hub_part then
// holds 8-byte partials.
cudaError_t launch_hub_fixup(const Csr &g, int32_t K, bool weighted,
                             bool laplacian, const uint32_t *counts, float *Z,
                             const void *hub_part, bool all_rows,
                             const DevStatus *st, cudaStream_t stream,
                             bool fixed = false, int shift = 0);

// S4 + S5 (CSR form) for many label vectors (gee_wide.cu): the lanes of a
// warp take the labels of one arc.  Same order and contract as the three
// launches above, with launch_hub_fixup(g, L*K, ...) last; no row tiles.
// For L >= kWideMinLabels.
cudaError_t launch_wide_rows(const Csr &g, int32_t L, int32_t K,
                             bool weighted, bool laplacian, const uint8_t *Yc,
                             const uint32_t *counts, float *Z,
                             unsigned long long *work, const DevStatus *st,
                             cudaStream_t stream);
cudaError_t launch_wide_chunks(const Csr &g, int32_t L, int32_t K,
                               bool weighted, bool laplacian,
                               const uint8_t *Yc, const uint32_t *counts,
                               float *Z, void *hub_part, const DevStatus *st,
                               cudaStream_t stream);

// ------------------------------------------------------------ batches
// Many independent edge-list problems in one launch sequence (gee_batch.cu).
// Work is cut into per-warp chunks of each kind; every problem's chunks are
// numbered consecutively in problem order.
constexpr int64_t kBatchNodeChunk = 4096;
constexpr int64_t kBatchEdgeChunk = 1024;
constexpr int64_t kBatchCellChunk = 16384;
enum { kChunkNodes = 0, kChunkEdges = 1, kChunkCells = 2 };
enum { kWorkLabels = 0, kWorkValidate, kWorkZero, kWorkScatter, kWorkFinalize,
       kWorkCounters };

// One problem as the kernels see it (device copy of the table).
struct BatchProblem {
    const int32_t *E;       // int32 [s][2]
    const float *w;         // [s] or null (unit weights)
    const int32_t *Y;       // [n]
    float *Z;               // [n][K]
    int64_t s, n;
    int32_t K, pad;
    uint32_t *counts;       // [K] class sizes (scratch)
    uint8_t *Yc;            // [n] compact labels (scratch)
    DevStatus *st;          // this problem's status (scratch)
    int64_t node_chunk0, edge_chunk0, cell_chunk0;  // first chunk of each kind
    int64_t counts_off, yc_off;  // scratch layout (host side)
};

struct BatchHeader {
    int64_t count;          // problems
    int64_t count_cells;    // total K over problems (the counts array)
    int64_t node_chunks, edge_chunks, cell_chunks;
    int64_t yc_bytes;
    uint32_t *counts;
    unsigned long long work[kWorkCounters];  // chunk counters, reset by init
};

// Host: numbers the chunks of every problem and lays out the scratch
// (counts_off, yc_off); fills the header's sizes.  Returns yc_bytes.
int64_t batch_layout(BatchProblem *P, int count, BatchHeader &h);
// Enqueues the phases (init, labels, [validate,] zero, scatter, finalize)
// for a header and problem table already in device memory (hh, the host
// copy of the header, is not needed by the launches).  The launch
// parameters are only dh and dP, so the sequence can be captured once ...
cudaError_t batch_enqueue(BatchHeader *dh, const BatchProblem *dP,
                          const BatchHeader &hh, bool validate,
                          cudaStream_t stream);
// Only the first two phases (status words and class counts zeroed, labels
// checked, compacted and counted), for a batch whose edge pass runs binned.
cudaError_t batch_labels_enqueue(BatchHeader *dh, const BatchProblem *dP,
                                 cudaStream_t stream);
// ... into an executable CUDA graph and replayed for every batch whose
// header and table are written to the same dh and dP.
cudaError_t batch_graph_create(BatchHeader *dh, const BatchProblem *dP,
                               bool validate, cudaStream_t stream,
                               cudaGraphExec_t *exec);

// ------------------------------------------------------------ binned pass
// GEE_BINNED (gee_bin.cu): updates written out as records grouped by the
// row tile of Z they land in, each tile summed in shared memory and
// written once.

// One edge-list problem of a binned launch (device copy).
struct BinProblem {
    const int32_t *E;           // int32 [s][2]
    const float *w;             // [s] or null
    int64_t s, n;
    const uint8_t *Yc;          // [n] compact labels
    const float *r;             // [n] Laplacian factors, or null
    float *Z;                   // [n][K]
    const uint32_t *counts;     // [K] n_k
    DevStatus *st;
    int64_t tile0, tiles;       // its row tiles: global [tile0, tile0 + tiles)
    int64_t chunk0;             // its first global edge chunk
    int32_t K, rows;            // classes; rows per tile (a power of two)
    uint32_t kmagic;            // floor((2^32 - 1) / K) + 1 (K > 1)
    uint32_t row_shift;         // log2(rows)
};

// The launch's sizes and scratch (kernel parameter, by value).
struct BinPlan {
    int32_t problems, coarse, group;
    int32_t paired;  // tile records laid out by tile pair (see gee_bin.cu)
    int64_t tiles, edge_chunks, records;   // records: capacity (2 s)
    uint32_t group_shift, pad2;             // log2(group): tile -> coarse bin
    unsigned long long *cnt1, *fill1, *off1, *chunk1;  // [coarse + 1]
    unsigned long long *cnt2, *fill2, *off2;           // [coarse * group + 1]
    unsigned long long *work;                          // tile counter
    uint32_t *key1;             // coarse records: tile << 16 | cell
    float *val1;                // their values (weighted)
    uint16_t *key2;             // tile records: the cell within the tile
    float *val2;
};

// Z cells beyond which pushed updates miss L2: GEE_AUTO takes BINNED for
// larger edge-list problems (the autotuner's grid ends here).
constexpr int64_t kBinnedMinCells = int64_t(1) << 24;
// A batch (or server group) of problems runs binned when most of its cells
// belong to problems beyond kBinnedMinCells; small problems keep their Z
// in L2 while pushed atomics land.
inline bool batch_prefers_binned(const BatchProblem *P, int count)
{
    int64_t cells = 0, big = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t c = P[i].n * (int64_t)P[i].K;
        cells += c;
        if (c > kBinnedMinCells)
            big += c;
    }
    return 2 * big > cells;
}

// Rows per tile for K classes: the largest power of two whose cells fit
// a tile's accumulators (so rows and bins split by shifts); bin_layout is
// false when `tiles` row tiles exceed the two-level layout (about 10^6
// tiles).  group is a power of two.
int32_t bin_rows(int32_t K, bool weighted);
bool bin_layout(int64_t tiles, int32_t *coarse, int32_t *group);
// Scratch of a binned launch over `records` record slots and `tiles` tiles.
size_t bin_scratch_bytes(int64_t records, int64_t tiles, bool weighted);
// Enqueues the binned sequence for a problem table already in device
// memory; pl's sizes set by the caller, its arrays allocated here.
cudaError_t bin_enqueue(Allocator &al, BinPlan &pl, const BinProblem *dP,
                        bool weighted, bool laplacian, cudaStream_t stream);
// S4 + S5 of a batch's problems in one binned sequence (problems in the
// host table P with their device Yc, counts and status set; labels done).
// Float sums for all problems if any has weights (unit weights then sum
// exactly).  cudaErrorInvalidValue if the tiles exceed the layout.
cudaError_t launch_binned_batch(Allocator &al, const BatchProblem *P,
                                int count, cudaStream_t stream);
// Row tiles of a batch's binned sequence (0 beyond the layout's limit).
int64_t binned_batch_tiles(const BatchProblem *P, int count);
// S4 + S5 of one edge list: endpoints checked (GEE_ERR_NODE_RANGE before Z
// is written), Z written in full.  Yc, counts (and r) from S1-S3.
cudaError_t launch_binned(Allocator &al, const int32_t *E, const float *w,
                          int64_t s, int64_t n, int32_t K, const uint8_t *Yc,
                          const float *r, const uint32_t *counts, float *Z,
                          DevStatus *st, cudaStream_t stream);

// ------------------------------------------------------------ autotuner
// The tuned GEE_AUTO choice for an edge-list problem (gee_tune.cu); false
// when the current device has no table.
bool tuned_choice(int64_t s, int64_t n, int32_t K, gee_strategy *strategy,
                  int32_t *block);

// ------------------------------------------------------------ runtime
// S1-S5 of L label vectors (Y[l*n + i], L >= 1) on a resident graph,
// enqueued on `stream` without waiting: *st receives the call's device
// status word (in ws).  Z is [n][L*K].  Argument checks are the caller's.
// deterministic: float sums in fixed point (bitwise reproducible); not for
// L >= kWideMinLabels with weights (GEE_ERR_UNSUPPORTED).
bool graph_weighted(const gee_graph *graph);
// Arcs of the graph's longest row (a self-loop gives its row two arcs).
uint32_t graph_max_degree(const gee_graph *graph);
gee_status graph_pass_enqueue(Workspace &ws, gee_graph *graph,
                              const int32_t *Y, int32_t L, int32_t K,
                              int32_t laplacian, float *Z, DevStatus **st,
                              cudaStream_t stream, bool host_z = false,
                              bool deterministic = false);

// ------------------------------------------------------------ tracing
// When tracing is on (gee_profile_enable), a ProfScope brackets one kernel
// launch with CUDA events on the launching stream.
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t stream);
    ~ProfScope();

  private:
    const char *name_;
    cudaStream_t stream_;
    cudaEvent_t begin_ = nullptr;
};

}  // namespace gee
