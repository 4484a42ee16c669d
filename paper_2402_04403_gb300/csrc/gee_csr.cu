// gee_csr.cu -- the row-sorted (CSR) form of GEE's edge pass on sm_103a.
//
// The paper's Ligra version runs Alg. 1's loop body inside edgeMapDense, one
// worker walking each node's edge list (Section III).  Here the same walk is
// organised for a GPU:
//
//   build_csr      edge list -> symmetric CSR (each edge (u,v,w) gives arcs
//                  u->v and v->u), rows with more than kHubDegree arcs moved
//                  to a separate hub CSR cut into chunks of kHubChunk arcs.
//   k_partition    splits rows + arcs into tiles of 1,024 (or 4,096) merged units
//                  (1 per arc, max(K,16) per row) so every tile moves about
//                  the same number of bytes.
//   k_pull_light   row tiles of the rows with at most kHubDegree arcs:
//                  coalesced arc sweep with labels through the read-only
//                  path (hub labels stay in L1) and shared atomics per
//                  (row, class), then the tile's Z rows -- contiguous in Z
//                  -- scaled by 1/n_k and written once.
//   k_pull_heavy   rows with more arcs, one warp per chunk of kHubChunk arcs;
//                  single-chunk rows write their Z row, longer rows leave
//                  per-chunk partial sums.
//   k_hub_fixup    sums those partials in chunk order and writes the rows.
//
// No global atomics touch Z: every light row is written once; a hub row
// gets zeros from k_pull_light, then its value from k_pull_heavy or
// k_hub_fixup, which run after it on the same stream.
#include <cmath>
#include <cstring>

#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int64_t kHubBit = int64_t(1) << 62;

// ------------------------------------------------------------ block scan
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v,
                                                        int64_t *warp_sums,
                                                        int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_sums[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int64_t t = warp_sums[w];
            warp_sums[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const int64_t r = warp_sums[warp] + x - v;
    __syncthreads();
    return r;
}

template <class In>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_reduce(const In *__restrict__ in, int64_t n,
                  int64_t *__restrict__ partial)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    __shared__ int64_t total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t sum = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        if (base + i < n)
            sum += (int64_t)in[base + i];
    block_exclusive_scan(sum, warp_sums, &total);
    if (threadIdx.x == 0)
        partial[blockIdx.x] = total;
}

// One CTA: exclusive scan of the per-tile sums in place; total -> *out_total.
__global__ void __launch_bounds__(1024)
    k_scan_partials(int64_t *__restrict__ partial, int64_t nb,
                    int64_t *__restrict__ out_total)
{
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t total;
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    int64_t sum = 0;
    for (int64_t i = b0; i < b0 + per && i < nb; ++i)
        sum += partial[i];
    int64_t run = block_exclusive_scan(sum, warp_sums, &total);
    for (int64_t i = b0; i < b0 + per && i < nb; ++i) {
        const int64_t t = partial[i];
        partial[i] = run;
        run += t;
    }
    if (threadIdx.x == 0)
        *out_total = total;
}

template <class In, class Out>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_apply(const In *__restrict__ in, int64_t n,
                 const int64_t *__restrict__ partial, Out *__restrict__ out)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    __shared__ int64_t total;
    const int64_t base =
        (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? (int64_t)in[base + j] : 0;
        sum += v[j];
    }
    int64_t run =
        block_exclusive_scan(sum, warp_sums, &total) + partial[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n)
            out[base + j] = (Out)run;
        run += v[j];
    }
}

// out[0..n) = exclusive prefix sums of in, out[n] = total.
template <class In, class Out>
cudaError_t exclusive_scan(const In *in, int64_t n, Out *out, Allocator &tmp,
                           cudaStream_t stream)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        return cudaMemsetAsync(out, 0, sizeof(Out), stream);
    }
    int64_t *partial = nullptr, *total = nullptr;
    cudaError_t e = tmp.alloc((void **)&partial, sizeof(int64_t) * (nb + 1));
    if (e != cudaSuccess)
        return e;
    total = partial + nb;
    k_scan_reduce<In><<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n,
                                                                partial);
    k_scan_partials<<<1, 1024, 0, stream>>>(partial, nb, total);
    k_scan_apply<In, Out>
        <<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, partial, out);
    // out[n] = total (narrowing copy for 32-bit outputs)
    if (sizeof(Out) == sizeof(int64_t))
        e = cudaMemcpyAsync(out + n, total, sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, stream);
    else
        e = cudaMemcpyAsync(out + n, total, sizeof(Out),
                            cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}

// ------------------------------------------------------------ CSR build
__device__ __forceinline__ bool node_ok(int32_t x, int64_t n)
{
    return (int64_t)(uint32_t)x < n;
}

template <class F>
__device__ __forceinline__ void for_each_edge(const int32_t *__restrict__ E,
                                              int64_t s, F &&f)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < s; i += nthreads) {
        const int2 e = __ldcs(reinterpret_cast<const int2 *>(E) + i);
        f(e.x, e.y, i);
    }
}

__global__ void k_csr_degree(const int32_t *__restrict__ E,
                             const float *__restrict__ w, int64_t s,
                             int64_t n, uint32_t *__restrict__ deg,
                             DevStatus *st)
{
    for_each_edge(E, s, [&](int32_t u, int32_t v, int64_t i) {
        if (!node_ok(u, n) || !node_ok(v, n)) {
            report(st, GEE_ERR_NODE_RANGE, (unsigned long long)i);
            return;
        }
        if (w != nullptr && !(w[i] >= 0.0f))
            atomicMax(&st->aux, 1);  // negative weight: no Laplacian
        atomicAdd(deg + u, 1u);
        atomicAdd(deg + v, 1u);
    });
}

// deg_main = deg for ordinary rows, 0 for hub rows; hub = 1 for hub rows.
__global__ void k_classify(const uint32_t *__restrict__ deg, int64_t n,
                           uint32_t *__restrict__ deg_main,
                           uint32_t *__restrict__ hub)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads) {
        const uint32_t d = deg[i];
        const bool h = d > (uint32_t)kHubDegree;
        deg_main[i] = h ? 0u : d;
        hub[i] = h ? 1u : 0u;
    }
}

__global__ void k_hub_list(const uint32_t *__restrict__ deg,
                           const uint32_t *__restrict__ hub,
                           const int64_t *__restrict__ hub_index, int64_t n,
                           int32_t *__restrict__ hub_row,
                           uint32_t *__restrict__ hub_deg,
                           uint32_t *__restrict__ hub_nchunks)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads) {
        if (!hub[i])
            continue;
        const int64_t h = hub_index[i];
        hub_row[h] = (int32_t)i;
        hub_deg[h] = deg[i];
        hub_nchunks[h] = (deg[i] + kHubChunk - 1) / kHubChunk;
    }
}

// bits[w] bit b = hub[32w + b]: one warp ballot per word.
__global__ void k_hub_bits(const uint32_t *__restrict__ hub, int64_t n,
                           uint32_t *__restrict__ bits)
{
    const int64_t words = (n + 31) >> 5;
    const int64_t lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < words; w += nwarps) {
        const int64_t i = (w << 5) + lane;
        const uint32_t b = __ballot_sync(0xffffffffu, i < n && hub[i] != 0u);
        if (lane == 0)
            bits[w] = b;
    }
}

__global__ void k_chunk_list(const int64_t *__restrict__ hub_ptr,
                             const int32_t *__restrict__ hub_chunk0,
                             int64_t hubs, int32_t *__restrict__ chunk_hub,
                             int64_t *__restrict__ chunk_begin)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t h = tid; h < hubs; h += nthreads) {
        const int32_t c0 = hub_chunk0[h], c1 = hub_chunk0[h + 1];
        for (int32_t c = c0; c < c1; ++c) {
            chunk_hub[c] = (int32_t)h;
            chunk_begin[c] = hub_ptr[h] + (int64_t)(c - c0) * kHubChunk;
        }
    }
}

// base[i] = first arc slot of row i in the main CSR, or (hub slot | kHubBit).
__global__ void k_base(const int64_t *__restrict__ rowptr,
                       const uint32_t *__restrict__ hub,
                       const int64_t *__restrict__ hub_index,
                       const int64_t *__restrict__ hub_ptr, int64_t n,
                       int64_t *__restrict__ base)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads)
        base[i] = hub[i] ? (hub_ptr[hub_index[i]] | kHubBit) : rowptr[i];
}


// ------------------------------------------------------------ degree ranks
// Nodes are ranked by decreasing degree (in buckets of a quarter octave) and
// arcs store the rank of their target instead of its id.  The labels of the
// highest-degree nodes -- the targets of most arcs in a power-law graph --
// then sit at the front of the rank-ordered label array, where the pull
// kernel keeps them in shared memory.
constexpr int kRankBuckets = 129;

__device__ __forceinline__ int rank_bucket(uint32_t d)
{
    if (d == 0u)
        return kRankBuckets - 1;
    const int oct = 31 - __clz(d);
    int frac = 0;
    if (oct >= 2)
        frac = (int)((d >> (oct - 2)) & 3u);
    else if (oct == 1)
        frac = (int)((d & 1u) << 1);
    return 127 - (4 * oct + frac);
}

// Ranks are stable within a bucket (nodes of one bucket in id order), so the
// compact labels of a pass, written in node order to their ranks, land in
// runs rather than one byte at a time (`k_labels`).  Nodes are taken in
// blocks of kRankBlock; per block and bucket a count, bucket-major
// (count[b * blocks + block]), whose exclusive scan is the rank of the
// block's first node of that bucket.
constexpr int kRankBlock = 1024;

__global__ void __launch_bounds__(kRankBlock)
    k_rank_block_count(const uint32_t *__restrict__ deg, int64_t n,
                       int64_t blocks, uint32_t *__restrict__ count)
{
    __shared__ uint32_t h[kRankBuckets];
    for (int b = threadIdx.x; b < kRankBuckets; b += blockDim.x)
        h[b] = 0u;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)kRankBlock + threadIdx.x;
    if (i < n)
        atomicAdd(&h[rank_bucket(deg[i])], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kRankBuckets; b += blockDim.x)
        count[(int64_t)b * blocks + blockIdx.x] = h[b];
}

// rank[i] = base[bucket][block] + the number of the block's nodes of the
// same bucket before i: their number in earlier warps (a per-bucket scan of
// the warps' counts) plus the lanes before it in its own warp.  Ranks form
// a permutation of [0, n).
__global__ void __launch_bounds__(kRankBlock)
    k_rank_block_assign(const uint32_t *__restrict__ deg, int64_t n,
                        int64_t blocks, const int32_t *__restrict__ base,
                        int32_t *__restrict__ rank)
{
    constexpr int kWarps = kRankBlock / 32;
    __shared__ uint32_t wcount[kWarps][kRankBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < kWarps * kRankBuckets; j += blockDim.x)
        (&wcount[0][0])[j] = 0u;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)kRankBlock + threadIdx.x;
    const int b = i < n ? rank_bucket(deg[i]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const unsigned before = __popc(peers & ((1u << lane) - 1u));
    if (b >= 0 && before == 0u)
        wcount[warp][b] = (uint32_t)__popc(peers);
    __syncthreads();
    // exclusive scan of each bucket's counts over the warps, in place
    for (int bb = threadIdx.x; bb < kRankBuckets; bb += blockDim.x) {
        uint32_t run = 0u;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wcount[w][bb];
            wcount[w][bb] = run;
            run += c;
        }
    }
    __syncthreads();
    if (b >= 0)
        rank[i] = base[(int64_t)b * blocks + blockIdx.x] +
                  (int32_t)wcount[warp][b] + (int32_t)before;
}

// Arcs u->v and v->u of every edge; the arc stores the target's rank.
__global__ void k_csr_fill(const int32_t *__restrict__ E,
                           const float *__restrict__ w, int64_t s,
                           const int64_t *__restrict__ base,
                           const int32_t *__restrict__ rank,
                           uint32_t *__restrict__ cursor,
                           int32_t *__restrict__ col,
                           float *__restrict__ val,
                           int32_t *__restrict__ col_h,
                           float *__restrict__ val_h, const DevStatus *st)
{
    if (failed(st))
        return;
    auto arc = [&](int32_t from, int32_t to, float wt) {
        const int64_t b = base[from];
        const int64_t slot = atomicAdd(cursor + from, 1u);
        const int32_t target = rank[to];
        if (b & kHubBit) {
            const int64_t p = (b & ~kHubBit) + slot;
            col_h[p] = target;
            if (val_h)
                val_h[p] = wt;
        } else {
            col[b + slot] = target;
            if (val)
                val[b + slot] = wt;
        }
    };
    for_each_edge(E, s, [&](int32_t u, int32_t v, int64_t i) {
        const float wt = (w != nullptr) ? w[i] : 1.0f;
        arc(u, v, wt);
        arc(v, u, wt);
    });
}

// ------------------------------------------------------------ Laplacian
// d_u (FP64 sum of the row's arc weights, or the arc count), r = 1/sqrt(d).
__global__ void k_row_rsqrt(const int64_t *__restrict__ rowptr,
                            const float *__restrict__ val, int64_t n,
                            float *__restrict__ r)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads) {
        const int64_t a0 = rowptr[i], a1 = rowptr[i + 1];
        double d = 0.0;
        if (val != nullptr)
            for (int64_t a = a0; a < a1; ++a)
                d += (double)val[a];
        else
            d = (double)(a1 - a0);
        r[i] = rsqrt_rn32(d);
    }
}

// Hub rows: one warp per hub, FP64 lane sums combined in a fixed tree.
__global__ void k_hub_rsqrt(const int32_t *__restrict__ hub_row,
                            const int64_t *__restrict__ hub_ptr,
                            const float *__restrict__ val_h, int64_t hubs,
                            float *__restrict__ r)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = warp; h < hubs; h += nwarps) {
        const int64_t a0 = hub_ptr[h], a1 = hub_ptr[h + 1];
        double d = 0.0;
        if (val_h != nullptr)
            for (int64_t a = a0 + lane; a < a1; a += 32)
                d += (double)val_h[a];
        else
            d = (lane == 0) ? (double)(a1 - a0) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0)
            r[hub_row[h]] = rsqrt_rn32(d);
    }
}

__global__ void k_scatter_by_rank(const float *__restrict__ r, int64_t n,
                                  const int32_t *__restrict__ rank,
                                  float *__restrict__ r_rank)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads)
        r_rank[rank[i]] = r[i];
}

// Laplacian arc value w * r(row) * r(target); targets are ranks.
__global__ void k_lap_values(const int64_t *__restrict__ rowptr,
                             const int32_t *__restrict__ col,
                             const float *__restrict__ val, int64_t n,
                             const float *__restrict__ r,
                             const float *__restrict__ r_rank,
                             float *__restrict__ out)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads) {
        const float ri = r[i];
        for (int64_t a = rowptr[i]; a < rowptr[i + 1]; ++a) {
            const float w = val ? val[a] : 1.0f;
            out[a] = w * ri * r_rank[col[a]];
        }
    }
}

__global__ void k_lap_values_hub(const int32_t *__restrict__ hub_row,
                                 const int64_t *__restrict__ hub_ptr,
                                 const int32_t *__restrict__ col_h,
                                 const float *__restrict__ val_h, int64_t hubs,
                                 const float *__restrict__ r,
                                 const float *__restrict__ r_rank,
                                 float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = warp; h < hubs; h += nwarps) {
        const float ri = r[hub_row[h]];
        for (int64_t a = hub_ptr[h] + lane; a < hub_ptr[h + 1]; a += 32) {
            const float w = val_h ? val_h[a] : 1.0f;
            out[a] = w * ri * r_rank[col_h[a]];
        }
    }
}

// ------------------------------------------------------------ partition
// Units: 1 per arc, C = max(K, 16) per row (its Z write; the floor keeps the
// rows of one tile, and so the shared-memory row table, bounded for small K).
// tile_row[t] = first row whose end unit E_r = rowptr[r+1] + r*C lies at or
// after t*units (n if none).  Tile t owns rows [tile_row[t],
// tile_row[t+1]) with all their arcs: at most ceil(units / C) rows and
// units + kHubDegree arcs.
__device__ __host__ inline int row_cost(int32_t K) { return K > 16 ? K : 16; }

__global__ void k_partition(const int64_t *__restrict__ rowptr, int64_t n,
                            int32_t K, int64_t ntiles, int32_t units,
                            int32_t *__restrict__ tile_row)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > ntiles)
        return;
    if (t == ntiles) {
        tile_row[t] = (int32_t)n;
        return;
    }
    const int64_t C = row_cost(K);
    const int64_t diag = t * units;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rowptr[mid + 1] + mid * C >= diag)
            hi = mid;
        else
            lo = mid + 1;
    }
    tile_row[t] = (int32_t)lo;
}

// ------------------------------------------------------------ pull
// Two persistent kernels, one CTA per SM.  Labels are read through the
// read-only path: with targets stored as degree ranks the most referenced
// labels are the first bytes of Yc and stay in L1.  A random byte gather
// that misses L1 costs about one SM clock in the L1 unit whatever its form,
// so the hub-row kernel, bound by those gathers, keeps the labels of the
// first kHotLabels ranks in shared memory (128 K measured best: larger
// copies shrink L1 too much; the row-tile kernel has no shared memory to
// spare).  Labels of the remaining ranks (hub rows), or of ranks from
// kLightColdFrom on (row tiles), almost never hit L1 and are read from L2
// without taking an L1 line, which leaves the lines to the loads in flight
// (hub rows 6.97 -> 6.41 ms, row tiles 5.47 -> 5.34 ms on the paper-scale
// graph).
//
// k_pull_light: rows with at most kHubDegree arcs.  Every warp of the CTA
//   is an independent group that takes row tiles of kTileUnits units from a
//   global counter; per tile: load the row starts, sweep the arcs (16-byte
//   loads, label, binary search for the row, shared atomic per (row,
//   class)), write the tile's Z rows -- contiguous in Z -- once with
//   16-byte stores.  One warp per tile needs only warp barriers, so no warp
//   waits for the slowest of several (groups of 4 warps on 4,096-unit
//   tiles: 5.22 ms on the paper-scale graph, one warp on 1,024 units:
//   4.89 ms).  The launch takes as many warps as the tiles' accumulators
//   fit in shared memory, at most 32.
//   Rows kept in the hub CSR have no arcs here and get zeros.
// k_pull_heavy: rows with more than kHubDegree arcs, cut into chunks of at
//   most kHubChunk arcs.  One warp per chunk, no block barriers; warps draw
//   kChunkGrab consecutive chunks at a time from a counter (measured faster
//   than fixed ranges of equal arc counts: no tail of idle warps).  A single-chunk row's Z row
//   is written directly, overwriting the zeros of k_pull_light (which runs
//   first); longer rows leave per-chunk partial sums for k_hub_fixup.
// Row-tile shapes: groups of GT threads on tiles of 32*GT units.  GT = 32
// (one warp per tile, warp barriers) for Z in device memory; GT = 128
// (named barriers) for page-locked host Z, whose larger tiles leave fewer
// partial 128-byte lines at tile ends for the host link.
constexpr int kDeviceGroup = 32;
constexpr int kHostGroup = 128;
template <int GT>
constexpr int tile_units() { return 32 * GT; }
static_assert(tile_units<kDeviceGroup>() == kTileUnits,
              "scratch for tile starts is sized by kTileUnits");
constexpr int kUnroll = 8;        // arcs in flight per thread (hub chunks)
constexpr int kLightUnroll = 4;   // the same for row tiles: a warp's tile of
                                  // 1,024 units holds about a quad per lane
                                  // (8: 4.89 ms, 4: 4.80 ms at paper scale)
constexpr int kTableCounts = 8;   // counts below this convert by table
constexpr int kHeavyThreads = 1024;
constexpr int kHeavyCopyCells = 128;  // float sums: copies x cols up to this
constexpr int kChunkGrab = 4;     // hub chunks a warp draws at a time
constexpr int kHotLabels = 131072; // hub-row kernel: bytes of labels in shared memory
// The same bytes as 6-bit codes: kHotWords words of five codes each, laid
// out so that rank v sits in word v mod kHotWords (no division by five)
constexpr int kHotWordsLog2 = 15;
constexpr int kHotWords = 1 << kHotWordsLog2;
static_assert(kHotWords * 4 == kHotLabels, "packed copy fills the byte copy's room");
constexpr int64_t kHotPackedFrom = int64_t(1) << 25;  // nodes (see hot_labels)
constexpr int kLightColdFrom = 1 << 18;  // row-tile kernel: ranks read past L1

struct PullArgs {
    const int64_t *rowptr;
    const int32_t *col;
    const float *val;
    const int32_t *tile_row;
    int64_t ntiles;
    const int32_t *hub_row;
    const int32_t *hub_chunk0;
    const int32_t *chunk_hub;
    const int64_t *chunk_begin;
    const int64_t *hub_ptr;
    const int32_t *col_h;
    const float *val_h;
    int64_t chunks;
    int64_t hub_arcs;
    const uint8_t *Yc;
    const uint32_t *counts;
    float *Z;
    uint32_t *hub_part;
    unsigned long long *work;
    const DevStatus *st;
    int32_t cols;         // Z columns per row: L label vectors x classes
    int32_t L;            // label vectors
    int32_t Ls;           // bytes per rank in Yc: L padded to 4 or to 16
    int32_t classes;      // classes per label vector
    uint32_t kmagic;      // floor((2^32-1) / cols) + 1: j / cols == umulhi(j, kmagic)
    int32_t max_rows;
    int32_t area_off;     // start of the per-group / per-warp areas
    int32_t group_bytes;  // per group (light) or per warp (heavy)
    int32_t acc_off, slot_off;
    int32_t hot_off, hot_n;  // heavy kernel: shared copy of the labels of
                             // ranks [0, hot_n) (as bytes: a multiple of 16)
    int32_t cold_from;       // labels of ranks >= cold_from are read past L1
    int32_t hot_packed;      // 1: the hot copy holds 6-bit codes, five per
                             // 32-bit word (63 = unknown)
    int32_t copies;          // heavy kernel: accumulator copies per warp
    double fx_scale, fx_inv; // fixed-point arc values: 2^shift, 2^-shift
    const uint32_t *hub_bits;  // light kernel: if set, hub rows' cells are
                               // left untouched (bit r: row r is a hub row)
    int32_t hub_direct;      // 1: single-chunk hub rows are written to Z by
                             // k_pull_heavy; 0: every chunk leaves partials
                             // and k_hub_fixup writes all hub rows
};

template <int GT>
__device__ __forceinline__ void group_sync(int g)
{
    if constexpr (GT == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

// Label of rank v (read-only path; the most referenced labels -- the front
// of the rank-ordered array -- stay in L1).
__device__ __forceinline__ uint32_t label_of(const PullArgs &a, int32_t v)
{
    return __ldg(a.Yc + v);
}

// Label of a rarely referenced rank: read from L2 without taking an L1 line
// (such gathers almost never hit L1, and the lines they would take are what
// keeps the other loads in flight).
__device__ __forceinline__ uint32_t cold_label_of(const PullArgs &a, int32_t v)
{
    uint32_t r;
    asm("ld.global.cg.u8 %0, [%1];" : "=r"(r) : "l"(a.Yc + v));
    return r;
}

// column of local cell j (the tile's first cell is a multiple of cols);
// the magic multiplier is exact for j < 2^32 / cols and does not exist for
// cols = 1
__device__ __forceinline__ int class_of(const PullArgs &a, int j)
{
    if (a.cols == 1)
        return 0;
    return j - a.cols * (int)__umulhi((unsigned)j, a.kmagic);
}

template <bool WEIGHTED>
__device__ __forceinline__ float cell_value(uint32_t c, int k,
                                            const uint32_t *nk,
                                            const float *table)
{
    if (WEIGHTED)
        return sum_to_z(__uint_as_float(c), nk[k]);
    return c < (uint32_t)kTableCounts ? table[k * kTableCounts + c]
                                      : count_to_z(c, nk[k]);
}

// CTA prologue of both pull kernels: n_k and the small-count table (Z
// values of counts 0..kTableCounts-1).
template <bool WEIGHTED>
__device__ __forceinline__ void load_shared(const PullArgs &a, uint32_t *nk,
                                            float *table)
{
    for (int k = threadIdx.x; k < a.cols; k += blockDim.x)
        nk[k] = a.counts[k];
    if (!WEIGHTED)
        for (int i = threadIdx.x; i < a.cols * kTableCounts; i += blockDim.x) {
            const int k = i / kTableCounts;
            table[i] = count_to_z((uint32_t)(i - k * kTableCounts),
                                  a.counts[k]);
        }
}

// Accumulator cells of a hub chunk: every arc belongs to the same row.
struct ChunkCells {
    int first;
    __device__ __forceinline__ void at(int) {}
    __device__ __forceinline__ int base(int) const { return first; }
};

// Accumulator cells of a row tile: rp[r] is the first arc of local row r
// (rp[NR] = NA).  at(i) finds the row of arc i by binary search; cell()
// then advances row by row for the following arcs.
struct TileCells {
    const int32_t *rp;
    int NR, K, off;
    int row, next;
    __device__ __forceinline__ void at(int i)
    {
        int lo = 0, hi = NR - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rp[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        row = lo;
        next = rp[lo + 1];
    }
    __device__ __forceinline__ int base(int i)
    {
        while (i >= next) {
            ++row;
            next = rp[row + 1];
        }
        return off + row * K;
    }
};

// Adds the arcs [0, NA) that start at colp[0] (any alignment) with NT
// threads, t = this thread: 16-byte loads of four arcs for the aligned body
// in rounds of kUnroll arcs per thread -- the next round's arcs are loaded
// before this round's labels are gathered, so the two latencies overlap --
// and single arcs for the head and tail.  cells maps (arc, label) to an
// accumulator index; arcs whose label is unknown go to this thread's own
// sink cell (no branch, no shared-address contention).
// SPAN (row tiles): instead of a scalar head and tail, every 16-byte group
// that overlaps the arcs is loaded and the arcs outside [0, NA) are
// skipped, so a tile runs no scalar row searches (column arrays carry 4
// entries of padding past their end).  HOT: a shared-memory copy of the
// first hot_n labels is consulted first (hub chunks), as bytes or (CODES)
// as 6-bit codes.
template <bool WEIGHTED, bool MULTI, int NT, class Cells, int UNROLL = kUnroll,
          bool FIXED = false, bool SPAN = false, bool HOT = false,
          bool CODES = false>
__device__ __forceinline__ void sweep_arcs(const PullArgs &a,
                                           const int32_t *colp,
                                           const float *valp, int NA, int t,
                                           uint32_t *acc, int sink,
                                           Cells &cells,
                                           const uint8_t *hot = nullptr,
                                           int hot_n = 0)
{
    float *accf = reinterpret_cast<float *>(acc);
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(acc);
    auto put = [&](int c, float w) {
        if (FIXED)  // 8-byte cells: the arc value in fixed point
            atomicAdd(acc64 + c, (unsigned long long)__double2ll_rn(
                                     (double)w * a.fx_scale));
        else if (WEIGHTED)
            atomicAdd(accf + c, w);
        else
            atomicAdd(acc + c, 1u);
    };
    // one label vector: y is the target's label; several: y is the target
    // rank and its L labels (adjacent bytes of Yc) are read here
    auto add = [&](int i, uint32_t y, float w) {
        if (!MULTI) {
            put(y != kNoLabel ? cells.base(i) + (int)y : sink, w);
        } else {
            // the target's labels: Ls adjacent bytes, read 16 or 4 at a time
            const int b = cells.base(i);
            const uint8_t *lab = a.Yc + (int64_t)y * a.Ls;
            auto four = [&](uint32_t word, int l0) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int l = l0 + e;
                    const uint32_t yl = (word >> (8 * e)) & 0xFFu;
                    if (l < a.L)
                        put(yl != kNoLabel ? b + l * a.classes + (int)yl : sink,
                            w);
                }
            };
            if ((a.Ls & 15) == 0) {
                for (int c = 0; c < a.Ls; c += 16) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(lab + c));
                    four(q.x, c);
                    four(q.y, c + 4);
                    four(q.z, c + 8);
                    four(q.w, c + 12);
                }
            } else {
                for (int c = 0; c < a.Ls; c += 4)
                    four(__ldg(reinterpret_cast<const uint32_t *>(lab + c)), c);
            }
        }
    };
    // the labels of the hot_n most referenced ranks come from the CTA's
    // shared-memory copy, those below cold_from through L1, the rest from L2
    auto fetch = [&](int32_t v) -> uint32_t {
        if (MULTI)
            return (uint32_t)v;
        if (HOT && v < hot_n) {
            if (!CODES)
                return (uint32_t)hot[v];
            // rank v is code v >> kHotWordsLog2 of word v mod kHotWords
            const uint32_t code =
                (reinterpret_cast<const uint32_t *>(hot)[v & (kHotWords - 1)] >>
                 (6u * ((uint32_t)v >> kHotWordsLog2))) & 63u;
            return code == 63u ? kNoLabel : code;
        }
        return v < a.cold_from ? label_of(a, v) : cold_label_of(a, v);
    };
    if constexpr (SPAN) {
        static_assert(UNROLL == 4, "one quad per thread per round");
        const int pre = (int)((reinterpret_cast<uintptr_t>(colp) >> 2) & 3);
        const int4 *col4 = reinterpret_cast<const int4 *>(colp - pre);
        const float4 *val4 = reinterpret_cast<const float4 *>(valp - pre);
        const int nq = (NA + pre + 3) >> 2;
        auto load = [&](int q, int4 &c, float4 &w) {
            const bool ok = q < nq;
            c = ok ? __ldcs(col4 + q) : make_int4(0, 0, 0, 0);
            if (WEIGHTED)
                w = ok ? __ldcs(val4 + q) : make_float4(0, 0, 0, 0);
        };
        int4 c;
        float4 w;
        load(t, c, w);
        for (int q = t; q < nq; q += NT) {
            int4 cn;
            float4 wn;
            load(q + NT, cn, wn);  // next round's arcs, in flight now
            const int i0 = 4 * q - pre;
            const int cv[4] = {c.x, c.y, c.z, c.w};
            const float wv[4] = {w.x, w.y, w.z, w.w};
            uint32_t y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                y[e] = (i0 + e >= 0 && i0 + e < NA) ? fetch(cv[e]) : kNoLabel;
            cells.at(i0 > 0 ? i0 : 0);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i0 + e >= 0 && i0 + e < NA)
                    add(i0 + e, y[e], WEIGHTED ? wv[e] : 0.0f);
            c = cn;
            w = wn;
        }
        return;
    }
    const int head =
        min((int)((4 - ((reinterpret_cast<uintptr_t>(colp) >> 2) & 3)) & 3), NA);
    if (t < head) {
        cells.at(t);
        add(t, fetch(colp[t]), WEIGHTED ? valp[t] : 0.0f);
    }
    const int nq = (NA - head) >> 2;
    const int4 *col4 = reinterpret_cast<const int4 *>(colp + head);
    const float4 *val4 = reinterpret_cast<const float4 *>(valp + head);
    constexpr int kQ = UNROLL / 4;  // quads per thread per round
    auto quads = [&](int q0, int4 (&c)[kQ], float4 (&w)[kQ]) {
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int q = q0 + u * NT;
            const bool ok = q < nq;
            c[u] = ok ? __ldcs(col4 + q) : make_int4(0, 0, 0, 0);
            if (WEIGHTED)
                w[u] = ok ? __ldcs(val4 + q) : make_float4(0, 0, 0, 0);
        }
    };
    int4 c[kQ];
    float4 w[kQ];
    if (t < nq)
        quads(t, c, w);
    for (int q0 = t; q0 < nq; q0 += kQ * NT) {
        int4 cn[kQ];
        float4 wn[kQ];
        quads(q0 + kQ * NT, cn, wn);  // next round's arcs, in flight now
        uint32_t y[UNROLL];
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            y[4 * u + 0] = fetch(c[u].x);
            y[4 * u + 1] = fetch(c[u].y);
            y[4 * u + 2] = fetch(c[u].z);
            y[4 * u + 3] = fetch(c[u].w);
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int q = q0 + u * NT;
            if (q < nq) {
                const int i0 = head + 4 * q;
                cells.at(i0);
                add(i0 + 0, y[4 * u + 0], WEIGHTED ? w[u].x : 0.0f);
                add(i0 + 1, y[4 * u + 1], WEIGHTED ? w[u].y : 0.0f);
                add(i0 + 2, y[4 * u + 2], WEIGHTED ? w[u].z : 0.0f);
                add(i0 + 3, y[4 * u + 3], WEIGHTED ? w[u].w : 0.0f);
            }
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            c[u] = cn[u];
            w[u] = wn[u];
        }
    }
    const int tail0 = head + 4 * nq;
    if (t < NA - tail0) {
        cells.at(tail0 + t);
        add(tail0 + t, fetch(colp[tail0 + t]),
            WEIGHTED ? valp[tail0 + t] : 0.0f);
    }
}

// Row starts of a tile, loaded ahead into registers: entry i = gt + j*32
// of rowptr[r0 .. r1] for the thread with group rank gt.
constexpr int kRowsAhead = 3;
static_assert(kRowsAhead * kDeviceGroup >= tile_units<kDeviceGroup>() / 16 + 1 &&
                  kRowsAhead * kHostGroup >= tile_units<kHostGroup>() / 16 + 1,
              "a tile's row starts fit in kRowsAhead per thread");
// Floats in a 128-byte line, and the float offset of p within its line.
constexpr int kLineFloats = 32;
__device__ __forceinline__ int line_offset(const float *p)
{
    return (int)((reinterpret_cast<uintptr_t>(p) >> 2) & (kLineFloats - 1));
}

struct TileRows {
    int32_t r0 = 0, r1 = 0;
    int64_t A0 = 0;
    int64_t rv[kRowsAhead];
};

template <int GT>
__device__ __forceinline__ void load_tile_rows(const PullArgs &a, int gt,
                                               TileRows &tr)
{
    tr.A0 = a.rowptr[tr.r0];
    const int NR = tr.r1 - tr.r0;
#pragma unroll
    for (int j = 0; j < kRowsAhead; ++j) {
        const int i = gt + j * GT;
        tr.rv[j] = i <= NR ? a.rowptr[tr.r0 + i] : 0;
    }
}

// One row tile (after the setup has been published by the caller's
// barrier): sweep its arcs into the accumulators, barrier, then scale and
// write its Z rows.  `before_write` runs between the barrier and the write
// phase (the caller issues the next tile's loads there).
template <bool WEIGHTED, bool MULTI, int GT, bool FIXED, class BeforeWrite>
__device__ __forceinline__ void row_tile(const PullArgs &a, int g, int gt,
                                         unsigned char *gs,
                                         const uint32_t *nk,
                                         const float *table,
                                         const TileRows &tr,
                                         BeforeWrite &&before_write)
{
    const int32_t K = a.cols;  // cells per row
    const int NR = tr.r1 - tr.r0;
    int32_t *rp = reinterpret_cast<int32_t *>(gs);  // row starts, tile-relative
    uint32_t *acc = reinterpret_cast<uint32_t *>(gs + a.acc_off);
    const int64_t g0 = (int64_t)tr.r0 * K;  // first Z cell of the tile
    // acc[off + j] holds cell g0 + j, off = the cell's float offset within
    // the unit its stores start at (any 4-byte aligned Z): a 128-byte line
    // for page-locked host Z (GT = kHostGroup), which the host link needs
    // whole; 16 bytes for device Z, where whole lines do not matter to HBM
    constexpr int kAlign = GT == kHostGroup ? kLineFloats : 4;
    const int off = line_offset(a.Z + g0) & (kAlign - 1);
    const int cells = NR * K;
    const int NA = NR > 0 ? rp[NR] : 0;

    // sweep: the row of arc i is the last row starting at or before i
    if (NA > 0) {
        TileCells tc{rp, NR, K, off, 0, 0};
        sweep_arcs<WEIGHTED, MULTI, GT, TileCells, kLightUnroll, FIXED, true>(
            a, a.col + tr.A0, WEIGHTED ? a.val + tr.A0 : nullptr, NA, gt, acc,
            a.max_rows * K + kLineFloats + 4 + (gt & 31), tc);
    }
    group_sync<GT>(g);
    before_write();

    // the tile's rows are contiguous in Z: scale once and stream out with
    // 16-byte stores between an unaligned head and tail (for host Z the
    // head runs to a 128-byte line, so each warp's stores cover whole
    // lines); all-zero quads (most of them: isolated nodes, sparse rows)
    // skip the conversion
    float *z = a.Z + g0;
    const int head = min((kAlign - off) & (kAlign - 1), cells);
    const int nq = (cells - head) >> 2;
    const int tail0 = head + 4 * nq;
    // each cell read here is cleared again, so the accumulators are zero
    // for the group's next tile
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(acc);
    auto quad_values = [&](int j0) {
        float4 o4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if constexpr (FIXED) {  // four 8-byte cells
            ulonglong2 *p2 = reinterpret_cast<ulonglong2 *>(acc64 + off + j0);
            const ulonglong2 c0 = p2[0], c1 = p2[1];
            if ((c0.x | c0.y | c1.x | c1.y) != 0ull) {
                p2[0] = make_ulonglong2(0ull, 0ull);
                p2[1] = make_ulonglong2(0ull, 0ull);
                int k = class_of(a, j0);
                const unsigned long long cs[4] = {c0.x, c0.y, c1.x, c1.y};
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    o[e] = fixed_to_z(cs[e], a.fx_inv, nk[k]);
                    if (++k == K)
                        k = 0;
                }
                o4 = make_float4(o[0], o[1], o[2], o[3]);
            }
            return o4;
        }
        uint4 *p4 = reinterpret_cast<uint4 *>(acc + off + j0);
        const uint4 c4 = *p4;
        if ((c4.x | c4.y | c4.z | c4.w) != 0u) {
            *p4 = make_uint4(0u, 0u, 0u, 0u);
            int k = class_of(a, j0);
            const uint32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                o[e] = cell_value<WEIGHTED>(cs[e], k, nk, table);
                if (++k == K)
                    k = 0;
            }
            o4 = make_float4(o[0], o[1], o[2], o[3]);
        }
        return o4;
    };
    auto scalar_value = [&](int j) {
        if constexpr (FIXED) {
            const unsigned long long c = acc64[off + j];
            acc64[off + j] = 0ull;
            return fixed_to_z(c, a.fx_inv, nk[class_of(a, j)]);
        }
        const uint32_t c = acc[off + j];
        acc[off + j] = 0u;
        return cell_value<WEIGHTED>(c, class_of(a, j), nk, table);
    };
    if (a.hub_bits == nullptr) {
        if (gt < head)
            __stcs(z + gt, scalar_value(gt));
        for (int q = gt; q < nq; q += GT) {
            const int j0 = head + 4 * q;
            __stcs(reinterpret_cast<float4 *>(z + j0), quad_values(j0));
        }
        if (gt < cells - tail0)
            __stcs(z + tail0 + gt, scalar_value(tail0 + gt));
        return;
    }
    // hub rows' cells are left to k_hub_fixup: a quad that touches one is
    // written cell by cell
    auto hub_cell = [&](int j) {
        const int64_t r = tr.r0 + (a.cols == 1 ? j : (int)__umulhi((unsigned)j, a.kmagic));
        return ((__ldg(a.hub_bits + (r >> 5)) >> (r & 31)) & 1u) != 0u;
    };
    if (gt < head) {
        const float v = scalar_value(gt);
        if (!hub_cell(gt))
            __stcs(z + gt, v);
    }
    for (int q = gt; q < nq; q += GT) {
        const int j0 = head + 4 * q;
        const float4 o4 = quad_values(j0);
        const bool h0 = hub_cell(j0), h1 = hub_cell(j0 + 1),
                   h2 = hub_cell(j0 + 2), h3 = hub_cell(j0 + 3);
        if (!(h0 | h1 | h2 | h3)) {
            __stcs(reinterpret_cast<float4 *>(z + j0), o4);
        } else {
            if (!h0)
                __stcs(z + j0, o4.x);
            if (!h1)
                __stcs(z + j0 + 1, o4.y);
            if (!h2)
                __stcs(z + j0 + 2, o4.z);
            if (!h3)
                __stcs(z + j0 + 3, o4.w);
        }
    }
    if (gt < cells - tail0) {
        const float v = scalar_value(tail0 + gt);
        if (!hub_cell(tail0 + gt))
            __stcs(z + tail0 + gt, v);
    }
}

// Each group pipelines its tiles: it draws tile t+1 before the setup
// barrier of tile t, loads t+1's row range while sweeping t and t+1's row
// starts while writing t, so a tile's setup finds its row starts in
// registers.  The accumulators are zeroed once; the write phase clears
// every cell it reads, so a tile starts on zeros.  Two group barriers per
// tile: setup published (which also orders the previous tile's writes and
// clears before this tile's sweep), accumulators complete.  The setup
// rewrites only the row starts, which no thread reads after the second
// barrier.
template <bool WEIGHTED, bool MULTI, int GT, bool FIXED>
__global__ void __launch_bounds__(1024, 1)
    k_pull_light(PullArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (failed(a.st))
        return;
    uint32_t *nk = reinterpret_cast<uint32_t *>(sm);
    float *table = reinterpret_cast<float *>(sm + ((a.cols * 4 + 15) & ~15));
    load_shared<WEIGHTED>(a, nk, table);
    __syncthreads();
    const int g = threadIdx.x / GT;
    const int gt = threadIdx.x - g * GT;
    unsigned char *gs = sm + a.area_off + (size_t)g * a.group_bytes;
    long long *slot = reinterpret_cast<long long *>(gs + a.slot_off);
    int32_t *rp = reinterpret_cast<int32_t *>(gs);
    uint32_t *acc = reinterpret_cast<uint32_t *>(gs + a.acc_off);
    const int32_t K = a.cols;
    {
        // every cell a tile can use: max_rows rows at a line offset
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        const int words = (a.max_rows * K + kLineFloats + 3) / 4 * (FIXED ? 2 : 1);
        for (int c = gt; c < words; c += GT)
            acc4[c] = make_uint4(0u, 0u, 0u, 0u);
    }

    if (gt == 0)
        slot[0] = (long long)atomicAdd(a.work, 1ull);
    group_sync<GT>(g);
    int64_t item = slot[0];
    TileRows cur;
    if (item < a.ntiles) {
        cur.r0 = a.tile_row[item];
        cur.r1 = a.tile_row[item + 1];
        load_tile_rows<GT>(a, gt, cur);
    }
    for (int it = 0; item < a.ntiles; ++it) {
        // the next tile, read by the group after the setup barrier below
        if (gt == 0)
            slot[(it + 1) & 1] = (long long)atomicAdd(a.work, 1ull);
        // setup: publish the row starts (the accumulators are zero)
        const int NR = cur.r1 - cur.r0;
#pragma unroll
        for (int j = 0; j < kRowsAhead; ++j) {
            const int i = gt + j * GT;
            if (i <= NR)
                rp[i] = (int32_t)(cur.rv[j] - cur.A0);
        }
        group_sync<GT>(g);
        const int64_t next = slot[(it + 1) & 1];
        TileRows nxt;
        if (next < a.ntiles) {  // in flight during the sweep
            nxt.r0 = a.tile_row[next];
            nxt.r1 = a.tile_row[next + 1];
        }
        row_tile<WEIGHTED, MULTI, GT, FIXED>(a, g, gt, gs, nk, table, cur, [&]() {
            if (next < a.ntiles)  // in flight during the write phase
                load_tile_rows<GT>(a, gt, nxt);
        });
        item = next;
        cur = nxt;
    }
}

template <bool WEIGHTED, bool MULTI, bool FIXED, bool CODES>
__global__ void __launch_bounds__(kHeavyThreads, 1) k_pull_heavy(PullArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (failed(a.st))
        return;
    uint32_t *nk = reinterpret_cast<uint32_t *>(sm);
    float *table = reinterpret_cast<float *>(sm + ((a.cols * 4 + 15) & ~15));
    load_shared<WEIGHTED>(a, nk, table);
    // copy of the labels of the most referenced ranks (front of Yc)
    uint8_t *hot = sm + a.hot_off;
    const int hot_n = MULTI ? 0 : a.hot_n;
    if (a.hot_packed) {
        // word w holds the codes of ranks w, w + kHotWords, ..., w + 4 kHotWords
        uint32_t *hw = reinterpret_cast<uint32_t *>(hot);
        for (int w = threadIdx.x; w < kHotWords; w += blockDim.x) {
            uint32_t word = 0u;
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int v = w + e * kHotWords;
                const uint32_t y = v < hot_n ? (uint32_t)__ldg(a.Yc + v) : kNoLabel;
                word |= (y == kNoLabel ? 63u : y) << (6 * e);
            }
            hw[w] = word;
        }
    } else {
        for (int i = threadIdx.x; i < hot_n / 16; i += blockDim.x)
            reinterpret_cast<uint4 *>(hot)[i] =
                __ldg(reinterpret_cast<const uint4 *>(a.Yc) + i);
    }
    __syncthreads();
    const int32_t K = a.cols;  // cells per row
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *acc = reinterpret_cast<uint32_t *>(sm + a.area_off +
                                                 (size_t)wib * a.group_bytes);
    float *accf = reinterpret_cast<float *>(acc);
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(acc);
    const int copies = WEIGHTED ? a.copies : 1;  // a power of two
    const int copy = (lane & (copies - 1)) * K;
    // warps draw kChunkGrab consecutive chunks at a time from a counter
    for (;;) {
        unsigned long long g0 = 0;
        if (lane == 0)
            g0 = atomicAdd(a.work, (unsigned long long)kChunkGrab);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if (g0 >= (unsigned long long)a.chunks)
            break;
        const int64_t c_lo = (int64_t)g0;
        const int64_t c_hi = min(c_lo + kChunkGrab, a.chunks);
    for (int64_t c = c_lo; c < c_hi; ++c) {
        for (int i = lane; i < copies * K; i += 32) {
            if (FIXED)
                acc64[i] = 0ull;
            else
                acc[i] = 0u;
        }
        __syncwarp();
        const int32_t h = a.chunk_hub[c];
        const int64_t b = a.chunk_begin[c];
        const int64_t hend = a.hub_ptr[h + 1];
        const int n = (int)((b + kHubChunk < hend ? b + kHubChunk : hend) - b);
        ChunkCells cells{copy};
        sweep_arcs<WEIGHTED, MULTI, 32, ChunkCells, kUnroll, FIXED, false, true,
                   CODES>(
            a, a.col_h + b, WEIGHTED ? a.val_h + b : nullptr, n, lane, acc,
            copies * K + lane, cells, hot, hot_n);
        __syncwarp();
        const bool whole =
            a.hub_direct && a.hub_chunk0[h + 1] - a.hub_chunk0[h] == 1;
        float *zrow = a.Z + (int64_t)a.hub_row[h] * K;
        for (int k = lane; k < K; k += 32) {
            if (FIXED) {  // exact integer sums: any order
                unsigned long long q = 0ull;
                for (int r = 0; r < copies; ++r)
                    q += acc64[r * K + k];
                if (whole)
                    zrow[k] = fixed_to_z(q, a.fx_inv, nk[k]);
                else
                    reinterpret_cast<unsigned long long *>(a.hub_part)[c * K + k] = q;
                continue;
            }
            uint32_t bits;
            if (WEIGHTED) {
                float s = 0.0f;
                for (int r = 0; r < copies; ++r)
                    s += accf[r * K + k];
                bits = __float_as_uint(s);
            } else {
                uint32_t s = 0;
                for (int r = 0; r < copies; ++r)
                    s += acc[r * K + k];
                bits = s;
            }
            if (whole)
                zrow[k] = cell_value<WEIGHTED>(bits, k, nk, table);
            else
                a.hub_part[c * K + k] = bits;
        }
        __syncwarp();
    }
    }
}

// One warp per hub row: its chunk partials summed in chunk order, then
// scaled.  Rows with fewer than min_chunks chunks are skipped (1: every hub
// row; 2: single-chunk rows were written by k_pull_heavy).
template <bool WEIGHTED, bool FIXED>
__global__ void k_hub_fixup(const int32_t *__restrict__ hub_row,
                            const int32_t *__restrict__ hub_chunk0,
                            int64_t hubs, const uint32_t *__restrict__ part,
                            const uint32_t *__restrict__ counts, int32_t K,
                            float *__restrict__ Z, int32_t min_chunks,
                            double fx_inv, const DevStatus *st)
{
    if (failed(st))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // 32 rows per step: each lane tests one, the warp then sums the rows
    // that need it one after another (most hub rows are a single chunk,
    // which the hub kernel wrote)
    for (int64_t h0 = warp * 32; h0 < hubs; h0 += nwarps * 32) {
        const int64_t hl = h0 + lane;
        const bool want =
            hl < hubs && hub_chunk0[hl + 1] - hub_chunk0[hl] >= min_chunks;
        for (unsigned todo = __ballot_sync(0xffffffffu, want); todo != 0u;
             todo &= todo - 1u) {
            const int64_t h = h0 + __ffs(todo) - 1;
            const int32_t c0 = hub_chunk0[h], c1 = hub_chunk0[h + 1];
            float *zrow = Z + (int64_t)hub_row[h] * K;
            for (int k = lane; k < K; k += 32) {
                if (FIXED) {
                    const unsigned long long *p64 =
                        reinterpret_cast<const unsigned long long *>(part);
                    unsigned long long q = 0ull;
                    for (int32_t c = c0; c < c1; ++c)
                        q += p64[(int64_t)c * K + k];
                    zrow[k] = fixed_to_z(q, fx_inv, counts[k]);
                } else if (WEIGHTED) {
                    float s = 0.0f;
                    for (int32_t c = c0; c < c1; ++c)
                        s += __uint_as_float(part[(int64_t)c * K + k]);
                    zrow[k] = sum_to_z(s, counts[k]);
                } else {
                    uint32_t s = 0;
                    for (int32_t c = c0; c < c1; ++c)
                        s += part[(int64_t)c * K + k];
                    zrow[k] = count_to_z(s, counts[k]);
                }
            }
        }
    }
}

inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory: [n_k (cols)][table cols x 8][per-group / per-warp areas].
// Returns the bytes to launch with.
size_t plan_shared(size_t area_bytes, PullArgs &a)
{
    const size_t fixed = align16((size_t)a.cols * 4) +
                         align16((size_t)a.cols * kTableCounts * 4);
    a.area_off = (int32_t)fixed;
    return fixed + area_bytes;
}

// ext[0] = max degree, ext[1] = bits of max |w| (non-negative floats order
// like their bit patterns).
__global__ void k_graph_extent(const uint32_t *__restrict__ deg, int64_t n,
                               const float *__restrict__ w, int64_t s,
                               uint32_t *__restrict__ ext)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    uint32_t d = 0u, m = 0u;
    for (int64_t i = tid; i < n; i += nthreads)
        d = max(d, deg[i]);
    if (w != nullptr)
        for (int64_t i = tid; i < s; i += nthreads)
            m = max(m, __float_as_uint(fabsf(w[i])));
    for (int o = 16; o > 0; o >>= 1) {
        d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(ext, d);
        atomicMax(ext + 1, m);
    }
}

}  // namespace

int fixed_shift(const Csr &g, bool laplacian)
{
    const double bound = laplacian ? 1.0
                         : g.max_abs_w > 0.0f ? (double)g.max_abs_w : 1.0;
    const double m = (g.max_deg > 0 ? (double)g.max_deg : 1.0) * bound;
    return (int)std::floor(62.0 - std::log2(m));
}

// ---------------------------------------------------------------- host side
cudaError_t build_csr(const int32_t *E, const float *w, int64_t s, int64_t n,
                      Allocator &persist, Allocator &al, Csr &g, DevStatus *st,
                      cudaStream_t stream)
{
#define GEE_TRY(x)                                                             \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess)                                                 \
            return e_;                                                         \
    } while (0)
    g.n = n;
    g.s = s;
    g.weighted = (w != nullptr);
    const int sms = sm_count();
    uint32_t *deg, *deg_main, *hub;
    int64_t *hub_index;
    GEE_TRY(al.alloc((void **)&deg, sizeof(uint32_t) * (n + 1)));
    GEE_TRY(al.alloc((void **)&deg_main, sizeof(uint32_t) * (n + 1)));
    GEE_TRY(al.alloc((void **)&hub, sizeof(uint32_t) * (n + 1)));
    GEE_TRY(al.alloc((void **)&hub_index, sizeof(int64_t) * (n + 1)));
    GEE_TRY(persist.alloc((void **)&g.rowptr, sizeof(int64_t) * (n + 1)));
    GEE_TRY(persist.alloc((void **)&g.rank, sizeof(int32_t) * (n + 1)));
    GEE_TRY(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * (n + 1), stream));
    if (s > 0)
        k_csr_degree<<<grid_for(s, 256, sms * 8), 256, 0, stream>>>(
            E, w, s, n, deg, st);
    uint32_t *ext;
    GEE_TRY(al.alloc((void **)&ext, sizeof(uint32_t) * 2));
    GEE_TRY(cudaMemsetAsync(ext, 0, sizeof(uint32_t) * 2, stream));
    if (n > 0 || w != nullptr)
        k_graph_extent<<<grid_for(n > s ? n : s, 256, sms * 4), 256, 0,
                         stream>>>(deg, n, w, w != nullptr ? s : 0, ext);
    if (n > 0)
        k_classify<<<grid_for(n, 256, sms * 8), 256, 0, stream>>>(
            deg, n, deg_main, hub);
    GEE_TRY(exclusive_scan(deg_main, n, g.rowptr, al, stream));
    GEE_TRY(exclusive_scan(hub, n, hub_index, al, stream));
    // degree ranks, stable within each bucket
    if (n > 0) {
        const int64_t blocks = (n + kRankBlock - 1) / kRankBlock;
        const int64_t cells = blocks * kRankBuckets;
        uint32_t *count;
        int32_t *base;
        GEE_TRY(al.alloc((void **)&count, sizeof(uint32_t) * (cells + 1)));
        GEE_TRY(al.alloc((void **)&base, sizeof(int32_t) * (cells + 1)));
        k_rank_block_count<<<(unsigned)blocks, kRankBlock, 0, stream>>>(
            deg, n, blocks, count);
        GEE_TRY(exclusive_scan(count, cells, base, al, stream));
        k_rank_block_assign<<<(unsigned)blocks, kRankBlock, 0, stream>>>(
            deg, n, blocks, base, g.rank);
    }
    int64_t host[2];
    GEE_TRY(cudaMemcpyAsync(&host[0], g.rowptr + n, 8, cudaMemcpyDeviceToHost,
                            stream));
    GEE_TRY(cudaMemcpyAsync(&host[1], hub_index + n, 8,
                            cudaMemcpyDeviceToHost, stream));
    DevStatus hst;
    GEE_TRY(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost,
                            stream));
    uint32_t hext[2];
    GEE_TRY(cudaMemcpyAsync(hext, ext, sizeof(hext), cudaMemcpyDeviceToHost,
                            stream));
    GEE_TRY(cudaStreamSynchronize(stream));
    g.negative_weight = hst.aux;
    g.max_deg = hext[0];
    std::memcpy(&g.max_abs_w, &hext[1], sizeof(float));
    if (hst.code != 0)
        return cudaSuccess;  // caller reports the status
    g.nnz_main = host[0];
    g.hubs = host[1];
    g.hub_arcs = 2 * s - g.nnz_main;
    // arrays are padded by 4 entries so 16-byte vector reads may overrun
    GEE_TRY(persist.alloc((void **)&g.col, sizeof(int32_t) * (g.nnz_main + 4)));
    if (g.weighted)
        GEE_TRY(persist.alloc((void **)&g.val, sizeof(float) * (g.nnz_main + 4)));
    int64_t *base;
    uint32_t *cursor;
    GEE_TRY(al.alloc((void **)&base, sizeof(int64_t) * (n + 1)));
    GEE_TRY(al.alloc((void **)&cursor, sizeof(uint32_t) * (n + 1)));
    GEE_TRY(persist.alloc((void **)&g.hub_ptr, sizeof(int64_t) * (g.hubs + 1)));
    GEE_TRY(persist.alloc((void **)&g.hub_bits,
                          sizeof(uint32_t) * ((n + 31) / 32 + 1)));
    GEE_TRY(cudaMemsetAsync(g.hub_bits, 0,
                            sizeof(uint32_t) * ((n + 31) / 32 + 1), stream));
    if (n > 0)
        k_hub_bits<<<grid_for((n + 31) / 32 * 32, 256, sms * 8), 256, 0,
                     stream>>>(hub, n, g.hub_bits);
    if (g.hubs > 0) {
        uint32_t *hub_deg, *hub_nchunks;
        GEE_TRY(persist.alloc((void **)&g.hub_row, sizeof(int32_t) * g.hubs));
        GEE_TRY(al.alloc((void **)&hub_deg, sizeof(uint32_t) * g.hubs));
        GEE_TRY(al.alloc((void **)&hub_nchunks, sizeof(uint32_t) * g.hubs));
        GEE_TRY(persist.alloc((void **)&g.hub_chunk0,
                              sizeof(int32_t) * (g.hubs + 1)));
        GEE_TRY(persist.alloc((void **)&g.col_h,
                              sizeof(int32_t) * (g.hub_arcs + 4)));
        if (g.weighted)
            GEE_TRY(persist.alloc((void **)&g.val_h,
                                  sizeof(float) * (g.hub_arcs + 4)));
        k_hub_list<<<grid_for(n, 256, sms * 8), 256, 0, stream>>>(
            deg, hub, hub_index, n, g.hub_row, hub_deg, hub_nchunks);
        GEE_TRY(exclusive_scan(hub_deg, g.hubs, g.hub_ptr, al, stream));
        GEE_TRY(exclusive_scan(hub_nchunks, g.hubs, g.hub_chunk0, al, stream));
        int32_t chunks = 0;
        GEE_TRY(cudaMemcpyAsync(&chunks, g.hub_chunk0 + g.hubs, 4,
                                cudaMemcpyDeviceToHost, stream));
        GEE_TRY(cudaStreamSynchronize(stream));
        g.chunks = chunks;
        GEE_TRY(persist.alloc((void **)&g.chunk_hub, sizeof(int32_t) * chunks));
        GEE_TRY(persist.alloc((void **)&g.chunk_begin,
                              sizeof(int64_t) * chunks));
        k_chunk_list<<<grid_for(g.hubs, 128, sms * 8), 128, 0, stream>>>(
            g.hub_ptr, g.hub_chunk0, g.hubs, g.chunk_hub, g.chunk_begin);
    } else {
        GEE_TRY(cudaMemsetAsync(g.hub_ptr, 0, sizeof(int64_t), stream));
    }
    if (n > 0)
        k_base<<<grid_for(n, 256, sms * 8), 256, 0, stream>>>(
            g.rowptr, hub, hub_index, g.hub_ptr, n, base);
    GEE_TRY(cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * (n + 1), stream));
    if (s > 0)
        k_csr_fill<<<grid_for(s, 256, sms * 8), 256, 0, stream>>>(
            E, w, s, base, g.rank, cursor, g.col, g.val, g.col_h, g.val_h, st);
    return cudaGetLastError();
#undef GEE_TRY
}

namespace {

// Arcs [0, m) of col whose target rank is below `below`.
__global__ void k_count_below(const int32_t *__restrict__ col, int64_t m,
                              int32_t below, unsigned long long *out)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0ull;
    for (int64_t i = tid; i < m; i += nth)
        c += col[i] < below ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c != 0ull)
        atomicAdd(out, c);
}

}  // namespace

int32_t hot_labels(int64_t n, int32_t L, int32_t classes, int32_t *packed)
{
    // 6-bit codes while the classes and the unknown code fit, on graphs
    // large enough that the extra labels pay for the decoding: five labels
    // per word, so the same kHotLabels bytes hold 25 % more of them.  Hub
    // kernel, packed against bytes: 65.6 M nodes (the paper-scale graph)
    // 6.17 against 6.38 ms, the same with 90 % unknown labels 6.15 against
    // 6.37; 16.7 M nodes (R-MAT-24) 1.32 against 1.28; 8.2 M nodes 0.70
    // against 0.64 (96 or 160 KB of codes at paper scale: 6.41 / 6.54 ms)
    *packed = (L == 1 && classes <= 63 && n >= kHotPackedFrom) ? 1 : 0;
    if (L > 1)
        return 0;
    if (*packed)
        return (int32_t)std::min<int64_t>((int64_t)kHotWords * 5, n);
    return (int32_t)(std::min<int64_t>((int64_t)kHotLabels, n) & ~int64_t(15));
}

cudaError_t count_hub_shared_arcs(const Csr &g, int32_t K,
                                  unsigned long long *d_out,
                                  cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess || g.hub_arcs == 0)
        return e;
    int32_t packed = 0;
    const int32_t hot = hot_labels(g.n, 1, K, &packed);
    k_count_below<<<grid_for(g.hub_arcs, 256, sm_count() * 8), 256, 0, stream>>>(
        g.col_h, g.hub_arcs, hot, d_out);
    return cudaGetLastError();
}

cudaError_t build_laplacian_values(Csr &g, Allocator &persist, Allocator &tmp,
                                   cudaStream_t stream)
{
    const int sms = sm_count();
    float *r, *r_rank;
    cudaError_t e = tmp.alloc((void **)&r, sizeof(float) * (g.n + 1));
    if (e != cudaSuccess)
        return e;
    e = tmp.alloc((void **)&r_rank, sizeof(float) * (g.n + 1));
    if (e != cudaSuccess)
        return e;
    e = persist.alloc((void **)&g.lap_val, sizeof(float) * (g.nnz_main + 4));
    if (e != cudaSuccess)
        return e;
    if (g.hubs > 0) {
        e = persist.alloc((void **)&g.lap_val_h,
                          sizeof(float) * (g.hub_arcs + 4));
        if (e != cudaSuccess)
            return e;
    }
    if (g.n > 0) {
        k_row_rsqrt<<<grid_for(g.n, 256, sms * 8), 256, 0, stream>>>(
            g.rowptr, g.val, g.n, r);
        if (g.hubs > 0)
            k_hub_rsqrt<<<grid_for(g.hubs * 32, 256, sms * 8), 256, 0,
                          stream>>>(g.hub_row, g.hub_ptr, g.val_h, g.hubs, r);
        k_scatter_by_rank<<<grid_for(g.n, 256, sms * 8), 256, 0, stream>>>(
            r, g.n, g.rank, r_rank);
        k_lap_values<<<grid_for(g.n, 256, sms * 8), 256, 0, stream>>>(
            g.rowptr, g.col, g.val, g.n, r, r_rank, g.lap_val);
        if (g.hubs > 0)
            k_lap_values_hub<<<grid_for(g.hubs * 32, 256, sms * 8), 256, 0,
                               stream>>>(g.hub_row, g.hub_ptr, g.col_h,
                                         g.val_h, g.hubs, r, r_rank,
                                         g.lap_val_h);
    }
    return cudaGetLastError();
}

int64_t pull_tiles(const Csr &g, int32_t K, bool host_z)
{
    const int64_t units = g.nnz_main + g.n * (int64_t)row_cost(K);
    const int64_t tu = host_z ? tile_units<kHostGroup>() : tile_units<kDeviceGroup>();
    return (units + tu - 1) / tu;
}

cudaError_t launch_partition(const Csr &g, int32_t K, int32_t *tile_row,
                             int64_t ntiles, bool host_z, cudaStream_t stream)
{
    k_partition<<<grid_for(ntiles + 1, 256, 1 << 30), 256, 0, stream>>>(
        g.rowptr, g.n, K, ntiles,
        host_z ? tile_units<kHostGroup>() : tile_units<kDeviceGroup>(),
        tile_row);
    return cudaGetLastError();
}

template <class Kern>
static cudaError_t launch_persistent(Kern kernel, int threads, size_t smem,
                                     const PullArgs &a, cudaStream_t stream,
                                     int ctas = 0)
{
    cudaError_t e = cudaFuncSetAttribute(
        kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kernel<<<ctas > 0 ? ctas : sm_count(), threads, smem, stream>>>(a);
    return cudaGetLastError();
}

static PullArgs pull_args(const Csr &g, int32_t L, int32_t classes,
                          bool laplacian,
                          const int32_t *tile_row, int64_t ntiles,
                          const uint8_t *Yc, const uint32_t *counts, float *Z,
                          void *hub_part, unsigned long long *work,
                          const DevStatus *st)
{
    PullArgs a = {};
    a.cold_from = INT32_MAX;
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.val = laplacian ? g.lap_val : g.val;
    a.tile_row = tile_row;
    a.ntiles = ntiles;
    a.hub_row = g.hub_row;
    a.hub_chunk0 = g.hub_chunk0;
    a.chunk_hub = g.chunk_hub;
    a.chunk_begin = g.chunk_begin;
    a.hub_ptr = g.hub_ptr;
    a.col_h = g.col_h;
    a.val_h = laplacian ? g.lap_val_h : g.val_h;
    a.chunks = g.chunks;
    a.hub_arcs = g.hub_arcs;
    a.Yc = Yc;
    a.counts = counts;
    a.Z = Z;
    a.hub_part = static_cast<uint32_t *>(hub_part);
    a.work = work;
    a.st = st;
    a.L = L;
    a.Ls = label_stride(L);
    a.classes = classes;
    a.cols = L * classes;
    a.kmagic = a.cols > 1 ? (uint32_t)(0xFFFFFFFFull / (uint32_t)a.cols + 1ull)
                          : 0u;
    return a;
}

cudaError_t launch_pull_light(const Csr &g, int32_t L, int32_t classes,
                              bool weighted, bool laplacian,
                              const int32_t *tile_row,
                              int64_t ntiles, const uint8_t *Yc,
                              const uint32_t *counts, float *Z,
                              unsigned long long *work, const DevStatus *st,
                              cudaStream_t stream, int ctas, bool host_z,
                              bool fixed, int shift)
{
    if (ntiles == 0)
        return cudaSuccess;
    PullArgs a = pull_args(g, L, classes, laplacian, tile_row, ntiles, Yc,
                           counts, Z, nullptr, work, st);
    a.hub_bits = host_z && g.chunks > 0 ? g.hub_bits : nullptr;
    const int K = a.cols;
    const int C = row_cost(K);
    const int GT = host_z ? kHostGroup : kDeviceGroup;
    const int units = 32 * GT;
    a.max_rows = (units + C - 1) / C;
    const size_t rpb = align16((size_t)(a.max_rows + 2) * 4);
    // + kLineFloats + 4 cells: the offset (< kLineFloats) and the 16-byte
    // rounding of the zeroing; then 32 sink cells (one per lane) for arcs of
    // unknown label
    const size_t accb = align16((size_t)(a.max_rows * K + kLineFloats + 4 + 32) *
                                (fixed ? 8 : 4));
    a.fx_scale = std::ldexp(1.0, shift);
    a.fx_inv = std::ldexp(1.0, -shift);
    a.acc_off = (int32_t)rpb;
    a.slot_off = (int32_t)(rpb + accb);
    a.group_bytes = (int32_t)(a.slot_off + 16);
    // as many groups as their areas fit (wide rows take more), at most
    // 1,024 threads
    const size_t base = plan_shared(0, a);
    const size_t room = (size_t)max_block_smem();
    int groups = room > base ? (int)((room - base) / a.group_bytes) : 0;
    if (groups > 1024 / GT)
        groups = 1024 / GT;
    if (groups < 1)
        return cudaErrorInvalidConfiguration;
    const size_t smem = plan_shared((size_t)groups * a.group_bytes, a);
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess)
        return e;
    a.cold_from = kLightColdFrom;
    const int threads = groups * GT;
    const bool w = weighted || laplacian;
#define GEE_LIGHT(W, M, F)                                                     \
    (host_z ? launch_persistent(k_pull_light<W, M, kHostGroup, F>, threads,    \
                                smem, a, stream, ctas)                         \
            : launch_persistent(k_pull_light<W, M, kDeviceGroup, F>, threads,  \
                                smem, a, stream, ctas))
    if (fixed)
        return L > 1 ? GEE_LIGHT(true, true, true) : GEE_LIGHT(true, false, true);
    if (L > 1)
        return w ? GEE_LIGHT(true, true, false) : GEE_LIGHT(false, true, false);
    return w ? GEE_LIGHT(true, false, false) : GEE_LIGHT(false, false, false);
#undef GEE_LIGHT
}

cudaError_t launch_pull_heavy(const Csr &g, int32_t L, int32_t classes,
                              bool weighted, bool laplacian, const uint8_t *Yc,
                              const uint32_t *counts, float *Z,
                              void *hub_part, bool partials_only,
                              unsigned long long *work, const DevStatus *st,
                              cudaStream_t stream, int ctas, bool fixed,
                              int shift)
{
    if (g.chunks == 0)
        return cudaSuccess;
    PullArgs a = pull_args(g, L, classes, laplacian, nullptr, 0, Yc, counts, Z,
                           hub_part, work, st);
    a.hub_direct = partials_only ? 0 : 1;
    cudaError_t e0 = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (e0 != cudaSuccess)
        return e0;
    // `copies` accumulators of cols cells per warp, then 32 sink cells, then
    // the hot labels (at most the first n ranks, a multiple of 16 bytes).
    // Integer counts use one copy; float sums spread the lanes over up to
    // four (lane l adds into copy l mod copies): shared-memory float adds
    // from several lanes to one cell serialise, and a few classes take all
    // of a warp's adds
    const bool w = weighted || laplacian;
    a.copies = 1;
    while (w && a.copies < 4 && 2 * a.copies * a.cols <= kHeavyCopyCells)
        a.copies *= 2;
    a.group_bytes =
        (int32_t)align16((size_t)(a.copies * a.cols + 32) * (fixed ? 8 : 4));
    a.fx_scale = std::ldexp(1.0, shift);
    a.fx_inv = std::ldexp(1.0, -shift);
    a.hot_n = hot_labels(g.n, L, a.classes, &a.hot_packed);
    a.cold_from = a.hot_n;
    const size_t hot_bytes =
        a.hot_packed ? (size_t)kHotWords * 4 : (size_t)a.hot_n;
    // as many warps as their accumulators fit next to the hot labels (wide
    // rows of 8-byte cells take more than 32 would have)
    const size_t base = plan_shared(hot_bytes, a);
    const size_t room = (size_t)max_block_smem();
    int warps = room > base ? (int)((room - base) / a.group_bytes) : 0;
    if (warps > kHeavyThreads / 32)
        warps = kHeavyThreads / 32;
    if (warps < 1)
        return cudaErrorInvalidConfiguration;
    const size_t area = (size_t)warps * a.group_bytes;
    const size_t smem = plan_shared(area + hot_bytes, a);
    a.hot_off = a.area_off + (int32_t)area;
    const int threads = warps * 32;
#define GEE_HEAVY(W, M, F, C)                                                  \
    launch_persistent(k_pull_heavy<W, M, F, C>, threads, smem, a, stream, ctas)
    const bool codes = a.hot_packed != 0;  // only for one label vector
    if (fixed)
        return L > 1 ? GEE_HEAVY(true, true, true, false)
                     : (codes ? GEE_HEAVY(true, false, true, true)
                              : GEE_HEAVY(true, false, true, false));
    if (L > 1)
        return w ? GEE_HEAVY(true, true, false, false)
                 : GEE_HEAVY(false, true, false, false);
    if (codes)
        return w ? GEE_HEAVY(true, false, false, true)
                 : GEE_HEAVY(false, false, false, true);
    return w ? GEE_HEAVY(true, false, false, false)
             : GEE_HEAVY(false, false, false, false);
#undef GEE_HEAVY
}

cudaError_t launch_hub_fixup(const Csr &g, int32_t K, bool weighted,
                             bool laplacian, const uint32_t *counts, float *Z,
                             const void *hub_part, bool all_rows,
                             const DevStatus *st, cudaStream_t stream,
                             bool fixed, int shift)
{
    if (g.hubs == 0)
        return cudaSuccess;
    const uint32_t *part = static_cast<const uint32_t *>(hub_part);
    const int fb = grid_for(g.hubs, 256, sm_count() * 8);
    const int32_t min_chunks = all_rows ? 1 : 2;
    const double inv = std::ldexp(1.0, -shift);
    if (fixed)
        k_hub_fixup<true, true><<<fb, 256, 0, stream>>>(
            g.hub_row, g.hub_chunk0, g.hubs, part, counts, K, Z, min_chunks,
            inv, st);
    else if (weighted || laplacian)
        k_hub_fixup<true, false><<<fb, 256, 0, stream>>>(
            g.hub_row, g.hub_chunk0, g.hubs, part, counts, K, Z, min_chunks,
            inv, st);
    else
        k_hub_fixup<false, false><<<fb, 256, 0, stream>>>(
            g.hub_row, g.hub_chunk0, g.hubs, part, counts, K, Z, min_chunks,
            inv, st);
    return cudaGetLastError();
}

}  // namespace gee
