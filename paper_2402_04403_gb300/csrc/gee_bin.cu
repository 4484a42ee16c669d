// gee_bin.cu -- GEE_BINNED: the edge-list pass with its updates grouped by
// destination row tile and summed in shared memory.
//
// Alg. 1's loop body sends each edge's two updates to rows u and v of Z.
// Pushed one at a time into a Z larger than L2 (GEE_ATOMIC), every update
// is an L2 reduction that misses: a DRAM read-modify-write per update.
// Here the updates are first written out as 4-byte records grouped by the
// tile of Z rows they land in -- propagation blocking (Beamer, Asanovic and
// Patterson, "Reducing PageRank communication via propagation blocking",
// IPDPS 2017), in two levels like the two digit passes of a radix
// partition -- and every tile is then summed in shared memory and its rows
// of Z written once, scaled by 1/n_k:
//
//   k_bin_count   checks the endpoints; per coarse bin (a group of row
//                 tiles), how many updates its rows can receive
//   k_bin_scan    capacities -> record offsets (one CTA)
//   k_bin_edges   per edge: both labels gathered, one record per update
//                 whose sender has a known label, appended to the coarse
//                 bin of its row (staged in shared memory by bin, then
//                 written out as contiguous runs)
//   k_bin_fine    per coarse bin, the records of each of its row tiles
//   k_bin_split   coarse records -> 16-bit records (the cell within the
//                 tile), grouped by row tile the same way
//   k_bin_tiles   per row tile: shared-memory accumulators -- uint32
//                 counts, or float sums with their rounding errors kept
//                 beside them -- then the tile's rows of Z, written once
//
// Up to 65,536 tiles the tile records are laid out by tile pair instead:
// k_bin_count_pairs counts both endpoints of every edge per pair of tiles
// (2i, 2i+1) -- 32 K counters, one shared-memory array per CTA -- and each
// pair gets one region of that size, which tile 2i fills from its start and
// tile 2i+1 from its end.  The regions' sizes are then known before any
// record is written, the coarse bins' regions are unions of whole pairs, and
// k_bin_fine (a read of every coarse record to count them per tile) and its
// scan drop out.
//
// The kernels take a table of problems so that several edge lists can share
// one sequence of launches; global row tiles number every problem's tiles
// in problem order.
#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kEdgeThreads = 512;  // k_bin_count / k_bin_edges
constexpr int kEdgeChunk = 4096;   // edges per chunk of those kernels
constexpr int kEdgesPerThread = kEdgeChunk / kEdgeThreads;
constexpr int kRecThreads = 512;   // k_bin_fine / k_bin_split
constexpr int kRecChunk = 8192;    // records per chunk of those kernels
constexpr int kSplitBlocks = 2;    // resident split CTAs per SM (64 registers)
constexpr int kRecsPerThread = kRecChunk / kRecThreads;
constexpr int kMaxBins = 1024;     // coarse bins; row tiles per coarse bin
constexpr int kTileThreads = 1024;
constexpr int kTileBytes = 200 * 1024;   // accumulators of one row tile
constexpr int kTablePerClass = 8;        // counts below this convert by table
static_assert(kEdgesPerThread * kEdgeThreads == kEdgeChunk, "edge chunk");
static_assert(kRecsPerThread * kRecThreads == kRecChunk, "record chunk");
static_assert(kTileBytes / 4 < 65536, "a cell within a tile fits 16 bits");

// A label gathered by the edge kernel: these gathers almost never hit L1,
// so they take no L1 line (leaving L1 to the loads in flight; 21.9 ->
// 20.5 ms on the paper-scale graph), and keep the evict-last L2 hint.
__device__ __forceinline__ uint32_t edge_label(const uint8_t *p, uint64_t pol)
{
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u8 %0, [%1], %2;"
        : "=r"(r)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ bool node_in(int32_t x, int64_t n)
{
    return (int64_t)(uint32_t)x < n;
}

// Problem owning global edge chunk c / global row tile t: the last one
// whose first chunk / tile is at or before it.
__device__ __forceinline__ int problem_of_chunk(const BinProblem *P, int count,
                                                int64_t c)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid].chunk0 <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int problem_of_tile(const BinProblem *P, int count,
                                               int64_t t)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P[mid].tile0 <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Coarse bin whose record chunks include chunk j: the last c with
// chunk1[c] <= j (empty bins share their successor's start).
__device__ __forceinline__ int coarse_of_chunk(const unsigned long long *chunk1,
                                               int coarse,
                                               unsigned long long j)
{
    int lo = 0, hi = coarse - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk1[mid] <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Exclusive scan of h[0..B) into start[0..B) by a block of NT threads
// (B <= kMaxBins, kMaxBins / NT consecutive entries per thread); *total =
// the sum.  Ends with a block barrier.
template <int NT>
__device__ __forceinline__ void scan_bins(const uint32_t *h, uint32_t *start,
                                          int B, uint32_t *warp_tot,
                                          uint32_t *total)
{
    constexpr int kScanPer = kMaxBins / NT;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t v[kScanPer];
    uint32_t mine = 0u;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int b = kScanPer * t + i;
        v[i] = b < B ? h[b] : 0u;
        mine += v[i];
    }
    uint32_t x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        constexpr int kWarps = NT / 32;
        const uint32_t w = lane < kWarps ? warp_tot[lane] : 0u;
        uint32_t u = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o)
                u += y;
        }
        if (lane < kWarps)
            warp_tot[lane] = u - w;  // exclusive prefix of the warps
        if (lane == kWarps - 1)
            *total = u;
    }
    __syncthreads();
    uint32_t ex = warp_tot[warp] + x - mine;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int b = kScanPer * t + i;
        if (b < B)
            start[b] = ex;
        ex += v[i];
    }
    __syncthreads();
}

// Ranks within a bin come from plain shared-memory atomics (one per
// record): lanes that share a bin are serialised by the hardware, which
// costs less than grouping them first (match.any runs at about one lane per
// two SM clocks on GB300, shared-memory atomics at six or more).

// ---------------------------------------------------------------- counts
// Per coarse bin, an upper bound of its records: both endpoints of every
// edge (the update is skipped later if the sender's label is unknown).
// Endpoints outside [0, n) are reported here, before anything is written.
__global__ void __launch_bounds__(kEdgeThreads)
    k_bin_count(BinPlan pl, const BinProblem *P)
{
    extern __shared__ uint32_t hist[];
    for (int b = threadIdx.x; b < pl.coarse; b += blockDim.x)
        hist[b] = 0u;
    __syncthreads();
    // consecutive endpoints of one thread often share a bin (small
    // problems of a table): count runs, one shared add per run
    uint32_t last = 0u, run = 0u;
    auto bump = [&](uint32_t c) {
        if (c == last && run != 0u) {
            ++run;
            return;
        }
        if (run != 0u)
            atomicAdd(hist + last, run);
        last = c;
        run = 1u;
    };
    for (int64_t chunk = blockIdx.x; chunk < pl.edge_chunks;
         chunk += gridDim.x) {
        const BinProblem &p = P[problem_of_chunk(P, pl.problems, chunk)];
        const int64_t e0 = (chunk - p.chunk0) * kEdgeChunk;
        const int64_t e1 = min(e0 + (int64_t)kEdgeChunk, p.s);
        const int2 *E = reinterpret_cast<const int2 *>(p.E);
        // every edge of the chunk loaded before any is counted, so each
        // thread keeps kEdgesPerThread loads in flight
        int2 uv[kEdgesPerThread];
#pragma unroll
        for (int j = 0; j < kEdgesPerThread; ++j) {
            const int64_t e = e0 + threadIdx.x + (int64_t)j * kEdgeThreads;
            uv[j] = e < e1 ? __ldcs(E + e) : make_int2(0, 0);
        }
#pragma unroll
        for (int j = 0; j < kEdgesPerThread; ++j) {
            const int64_t e = e0 + threadIdx.x + (int64_t)j * kEdgeThreads;
            if (e >= e1)
                continue;
            if (!node_in(uv[j].x, p.n) || !node_in(uv[j].y, p.n)) {
                report(p.st, GEE_ERR_NODE_RANGE, (unsigned long long)e);
                continue;
            }
            bump(((uint32_t)p.tile0 + ((uint32_t)uv[j].x >> p.row_shift)) >>
                 pl.group_shift);
            bump(((uint32_t)p.tile0 + ((uint32_t)uv[j].y >> p.row_shift)) >>
                 pl.group_shift);
        }
    }
    if (run != 0u)
        atomicAdd(hist + last, run);
    __syncthreads();
    for (int b = threadIdx.x; b < pl.coarse; b += blockDim.x)
        if (hist[b] != 0u)
            atomicAdd(pl.cnt1 + b, (unsigned long long)hist[b]);
}

// Paired layout: per pair of row tiles, how many updates its rows can
// receive (both endpoints of every edge), in a shared-memory counter per
// pair; endpoints outside [0, n) are reported here.  One CTA per SM.
constexpr int kPairThreads = 1024;
constexpr int kMaxPairs = 32768;

__global__ void __launch_bounds__(kPairThreads, 1)
    k_bin_count_pairs(BinPlan pl, const BinProblem *P)
{
    extern __shared__ uint32_t pc[];  // [pairs]
    const int pairs = (int)((pl.tiles + 1) >> 1);
    for (int i = threadIdx.x; i < pairs; i += blockDim.x)
        pc[i] = 0u;
    __syncthreads();
    // two chunks per round, every edge of both loaded before any is
    // counted (eight loads in flight per thread)
    constexpr int kPer = kEdgeChunk / kPairThreads;
    constexpr int kChunks = 2;
    for (int64_t c0 = (int64_t)blockIdx.x * kChunks; c0 < pl.edge_chunks;
         c0 += (int64_t)gridDim.x * kChunks) {
        const BinProblem *pp[kChunks];
        int64_t e0[kChunks], e1[kChunks];
        int2 uv[kChunks][kPer];
#pragma unroll
        for (int h = 0; h < kChunks; ++h) {
            const int64_t chunk = c0 + h;
            pp[h] = chunk < pl.edge_chunks
                        ? P + problem_of_chunk(P, pl.problems, chunk)
                        : P;
            e0[h] = (chunk - pp[h]->chunk0) * kEdgeChunk;
            e1[h] = chunk < pl.edge_chunks
                        ? min(e0[h] + (int64_t)kEdgeChunk, pp[h]->s)
                        : e0[h];
            const int2 *E = reinterpret_cast<const int2 *>(pp[h]->E);
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int64_t e = e0[h] + threadIdx.x + (int64_t)j * kPairThreads;
                uv[h][j] = e < e1[h] ? __ldcs(E + e) : make_int2(0, 0);
            }
        }
#pragma unroll
        for (int h = 0; h < kChunks; ++h) {
            const BinProblem &p = *pp[h];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int64_t e = e0[h] + threadIdx.x + (int64_t)j * kPairThreads;
                if (e >= e1[h])
                    continue;
                if (!node_in(uv[h][j].x, p.n) || !node_in(uv[h][j].y, p.n)) {
                    report(p.st, GEE_ERR_NODE_RANGE, (unsigned long long)e);
                    continue;
                }
                atomicAdd(pc + (((uint32_t)p.tile0 +
                                 ((uint32_t)uv[h][j].x >> p.row_shift)) >> 1), 1u);
                atomicAdd(pc + (((uint32_t)p.tile0 +
                                 ((uint32_t)uv[h][j].y >> p.row_shift)) >> 1), 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pairs; i += blockDim.x)
        if (pc[i] != 0u)
            atomicAdd(pl.cnt2 + i, (unsigned long long)pc[i]);
}

// Paired layout: the coarse bins' record offsets from the pairs' (a coarse
// bin is a run of whole pairs; one bin of one tile when there is one tile).
__global__ void k_bin_pair_coarse(BinPlan pl)
{
    const int64_t pairs = (pl.tiles + 1) >> 1;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= pl.coarse;
         c += gridDim.x * blockDim.x)
        pl.off1[c] = pl.off2[min(((int64_t)c * pl.group + 1) >> 1, pairs)];
}

// First record of tile t's region among the tile records: its pair's
// region, from the start for an even tile, from the end for an odd one
// (fill2 holds the records the tile received).
__device__ __forceinline__ unsigned long long tile_records_start(const BinPlan &pl,
                                                                 int64_t t)
{
    if (!pl.paired)
        return pl.off2[t];
    const int64_t q = t >> 1;
    return (t & 1) ? pl.off2[q + 1] - pl.fill2[t] : pl.off2[q];
}

// out[i] = sum of x(j) for j < i, i in [0, m]; x(j) = in[j], or with
// per_chunk the number of kRecChunk-record chunks of in[j] records.
__global__ void __launch_bounds__(1024)
    k_bin_scan(const unsigned long long *__restrict__ in, int64_t m,
               int per_chunk, unsigned long long *__restrict__ out)
{
    __shared__ unsigned long long warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    auto x = [&](int64_t j) -> unsigned long long {
        const unsigned long long v = in[j];
        return per_chunk ? (v + kRecChunk - 1) / kRecChunk : v;
    };
    const int64_t per = (m + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)t * per;
    const int64_t b1 = min(b0 + per, m);
    unsigned long long sum = 0ull;
    for (int64_t j = b0; j < b1; ++j)
        sum += x(j);
    unsigned long long v = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += y;
    }
    if (lane == 31)
        warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const unsigned long long w = lane < nw ? warp_tot[lane] : 0ull;
        unsigned long long u = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o)
                u += y;
        }
        if (lane < nw)
            warp_tot[lane] = u - w;
        if (lane == nw - 1)
            out[m] = u;
    }
    __syncthreads();
    unsigned long long run = warp_tot[warp] + v - sum;
    for (int64_t j = b0; j < b1; ++j) {
        out[j] = run;
        run += x(j);
    }
}

// ---------------------------------------------------------------- records
// Alg. 1 loop body, as records: edge (u, v, w) gives (row u, class Y[v],
// w [* r_v]) and (row v, class Y[u], w [* r_u]) where the class is known.
// A record is its row tile within the coarse bin (high 16 bits) and its
// cell within the tile (low 16 bits); the weighted form keeps the value in
// a parallel float array.
template <bool WEIGHTED, bool LAP, bool WIDE>
__global__ void __launch_bounds__(kEdgeThreads, 2)
    k_bin_edges(BinPlan pl, const BinProblem *P)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint32_t warp_tot[kEdgeThreads / 32];
    __shared__ uint32_t s_total;
    constexpr int kRec = 2 * kEdgeChunk;
    uint32_t *hist = reinterpret_cast<uint32_t *>(sm);  // counts, then cursors
    uint32_t *start = hist + kMaxBins;
    // dst0[b] + i: where staged record i of bin b goes in the coarse records
    unsigned long long *dst0 =
        reinterpret_cast<unsigned long long *>(start + kMaxBins);
    uint32_t *skey = reinterpret_cast<uint32_t *>(dst0 + kMaxBins);
    float *sval = reinterpret_cast<float *>(skey + kRec);
    uint16_t *sbin =
        reinterpret_cast<uint16_t *>(sval + (WEIGHTED ? kRec : 0));
    const int B = pl.coarse;
    const uint32_t G = (uint32_t)pl.group;
    for (int b = threadIdx.x; b < B; b += blockDim.x)
        hist[b] = 0u;
    __syncthreads();
    const uint64_t keep = policy_evict_last();
    for (int64_t chunk = blockIdx.x; chunk < pl.edge_chunks;
         chunk += gridDim.x) {
        const BinProblem &p = P[problem_of_chunk(P, pl.problems, chunk)];
        if (failed(p.st))
            continue;  // the same for every thread: no kernel writes st now
        const int64_t e0 = (chunk - p.chunk0) * kEdgeChunk;
        const int64_t e1 = min(e0 + (int64_t)kEdgeChunk, p.s);
        const int2 *E = reinterpret_cast<const int2 *>(p.E);
        const uint32_t rs = p.row_shift, gs = pl.group_shift;
        const uint32_t rows = (uint32_t)p.rows, K = (uint32_t)p.K,
                       tile0 = (uint32_t)p.tile0;
        int2 uv[kEdgesPerThread];
        float wt[kEdgesPerThread];
#pragma unroll
        for (int j = 0; j < kEdgesPerThread; ++j) {
            const int64_t e = e0 + threadIdx.x + (int64_t)j * kEdgeThreads;
            const bool ok = e < e1;
            uv[j] = ok ? __ldcs(E + e) : make_int2(-1, -1);
            if (WEIGHTED)
                wt[j] = (ok && p.w != nullptr) ? __ldcs(p.w + e) : 1.0f;
        }
        // both labels of edge j in one word: Y[u] | Y[v] << 8
        uint32_t y2[kEdgesPerThread];
        float ru[kEdgesPerThread], rv[kEdgesPerThread];
#pragma unroll
        for (int j = 0; j < kEdgesPerThread; ++j) {
            const bool ok = uv[j].x >= 0;
            const uint32_t a = ok ? edge_label(p.Yc + uv[j].x, keep) : kNoLabel;
            const uint32_t b = ok ? edge_label(p.Yc + uv[j].y, keep) : kNoLabel;
            y2[j] = a | (b << 8);
            if (LAP) {
                ru[j] = ok ? __ldg(p.r + uv[j].x) : 0.0f;
                rv[j] = ok ? __ldg(p.r + uv[j].y) : 0.0f;
            }
        }
        // record i: row u with v's class (even i), row v with u's (odd i);
        // key 0xFFFFFFFF where that class is unknown.  The key holds the
        // whole tile number while it fits 16 bits (the bin is then
        // key >> (16 + gs)), else the tile within the bin, with the bin
        // kept beside it (16-bit halves of cw).  Each record's place among
        // this chunk's records of its bin comes from one shared-memory
        // atomic (16-bit halves of rk).
        uint32_t key[2 * kEdgesPerThread], rk[kEdgesPerThread];
        uint32_t cw[WIDE ? kEdgesPerThread : 1];
        float val[(WEIGHTED && LAP) ? 2 * kEdgesPerThread : 1];
#pragma unroll
        for (int i = 0; i < 2 * kEdgesPerThread; ++i) {
            const int j = i >> 1;
            const uint32_t row = (uint32_t)((i & 1) ? uv[j].y : uv[j].x);
            const uint32_t y = (i & 1) ? (y2[j] & 0xFFu) : (y2[j] >> 8);
            const uint32_t g = tile0 + (row >> rs);  // global row tile
            const uint32_t c = g >> gs;
            const bool valid = y != kNoLabel;
            key[i] = valid ? (((WIDE ? (g & (G - 1u)) : g) << 16) |
                              ((row & (rows - 1u)) * K + y))
                           : 0xFFFFFFFFu;
            if (WIDE) {
                if (i & 1)
                    cw[j] |= c << 16;
                else
                    cw[j] = c;
            }
            if (WEIGHTED && LAP)
                val[i] = __fmul_rn(wt[j], (i & 1) ? ru[j] : rv[j]);
            const uint32_t r = valid ? atomicAdd(hist + c, 1u) : 0u;
            if (i & 1)
                rk[j] |= r << 16;
            else
                rk[j] = r;
        }
        auto bin_of = [&](int i) -> uint32_t {
            return WIDE ? ((cw[i >> 1] >> (16 * (i & 1))) & 0xFFFFu)
                        : (key[i] >> (16 + gs));
        };
        __syncthreads();
        scan_bins<kEdgeThreads>(hist, start, B, warp_tot, &s_total);
        // reserve each bin's run in its coarse bin; the atomics' results
        // are needed only by the write-out, so they stay in flight while
        // the records are staged
        constexpr int kResv = kMaxBins / kEdgeThreads;
        unsigned long long resv[kResv];
#pragma unroll
        for (int i = 0; i < kResv; ++i) {
            const int b = threadIdx.x + i * kEdgeThreads;
            resv[i] = 0ull;
            if (b < B) {
                const uint32_t h = hist[b];
                if (h != 0u)
                    resv[i] = atomicAdd(pl.fill1 + b, (unsigned long long)h);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * kEdgesPerThread; ++i) {
            if (key[i] != 0xFFFFFFFFu) {
                const uint32_t c = bin_of(i);
                const uint32_t pos =
                    start[c] + ((rk[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
                skey[pos] = key[i];
                if (WIDE)
                    sbin[pos] = (uint16_t)c;
                if (WEIGHTED)
                    sval[pos] = LAP ? val[i] : wt[i >> 1];
            }
        }
#pragma unroll
        for (int i = 0; i < kResv; ++i) {
            const int b = threadIdx.x + i * kEdgeThreads;
            if (b < B)  // unsigned wrap-around cancels when i is added
                dst0[b] = pl.off1[b] + resv[i] - start[b];
        }
        __syncthreads();
        const uint32_t total = s_total;
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
            const uint32_t k1 = skey[i];
            const unsigned long long dst =
                dst0[WIDE ? (uint32_t)sbin[i] : (k1 >> (16 + gs))] + i;
            __stcs(pl.key1 + dst, k1);
            if (WEIGHTED)
                __stcs(pl.val1 + dst, sval[i]);
        }
        for (int b = threadIdx.x; b < B; b += blockDim.x)
            hist[b] = 0u;
        __syncthreads();
    }
}

// Per coarse bin: records per row tile (exact counts of what k_bin_split
// will write).
__global__ void __launch_bounds__(kRecThreads) k_bin_fine(BinPlan pl)
{
    extern __shared__ uint32_t hist[];
    __shared__ int s_c;
    __shared__ unsigned long long s_r0, s_r1;
    const int G = pl.group;
    for (int f = threadIdx.x; f < G; f += blockDim.x)
        hist[f] = 0u;
    const unsigned long long chunks = pl.chunk1[pl.coarse];
    for (unsigned long long j = blockIdx.x; j < chunks; j += gridDim.x) {
        if (threadIdx.x == 0) {
            const int c = coarse_of_chunk(pl.chunk1, pl.coarse, j);
            const unsigned long long r0 =
                pl.off1[c] + (j - pl.chunk1[c]) * kRecChunk;
            s_c = c;
            s_r0 = r0;
            s_r1 = min(r0 + kRecChunk, pl.off1[c] + pl.fill1[c]);
        }
        __syncthreads();
        const int c = s_c;
        const unsigned long long r1 = s_r1;
        const unsigned long long r0 = s_r0;
        uint32_t key[kRecsPerThread];
#pragma unroll
        for (int q = 0; q < kRecsPerThread; ++q) {
            const unsigned long long r =
                r0 + threadIdx.x + (unsigned long long)q * kRecThreads;
            key[q] = r < r1 ? __ldcs(pl.key1 + r) : 0xFFFFFFFFu;
        }
        uint32_t last = 0u, run = 0u;
#pragma unroll
        for (int q = 0; q < kRecsPerThread; ++q) {
            if (key[q] == 0xFFFFFFFFu)
                continue;
            const uint32_t f = (key[q] >> 16) & (uint32_t)(G - 1);
            if (f == last && run != 0u) {
                ++run;
                continue;
            }
            if (run != 0u)
                atomicAdd(hist + last, run);
            last = f;
            run = 1u;
        }
        if (run != 0u)
            atomicAdd(hist + last, run);
        __syncthreads();
        for (int f = threadIdx.x; f < G; f += blockDim.x) {
            const uint32_t h = hist[f];
            if (h != 0u) {
                atomicAdd(pl.cnt2 + (int64_t)c * G + f, (unsigned long long)h);
                hist[f] = 0u;
            }
        }
        __syncthreads();
    }
}

// Coarse records -> tile records (the low 16 bits), grouped by row tile.
template <bool WEIGHTED>
__global__ void __launch_bounds__(kRecThreads, kSplitBlocks) k_bin_split(BinPlan pl)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint32_t warp_tot[kRecThreads / 32];
    __shared__ uint32_t s_total;
    __shared__ int s_c;
    __shared__ unsigned long long s_r0, s_r1;
    uint32_t *hist = reinterpret_cast<uint32_t *>(sm);  // counts, then cursors
    uint32_t *start = hist + kMaxBins;
    // dst0[f] + i: where staged record i of tile f goes in the tile records
    unsigned long long *dst0 =
        reinterpret_cast<unsigned long long *>(start + kMaxBins);
    float *sval = reinterpret_cast<float *>(dst0 + kMaxBins);
    // staged record: cell | tile << 16
    uint32_t *sent =
        reinterpret_cast<uint32_t *>(sval + (WEIGHTED ? kRecChunk : 0));
    const int G = pl.group;
    for (int f = threadIdx.x; f < G; f += blockDim.x)
        hist[f] = 0u;
    const unsigned long long chunks = pl.chunk1[pl.coarse];
    for (unsigned long long j = blockIdx.x; j < chunks; j += gridDim.x) {
        if (threadIdx.x == 0) {
            const int c = coarse_of_chunk(pl.chunk1, pl.coarse, j);
            const unsigned long long r0 =
                pl.off1[c] + (j - pl.chunk1[c]) * kRecChunk;
            s_c = c;
            s_r0 = r0;
            s_r1 = min(r0 + kRecChunk, pl.off1[c] + pl.fill1[c]);
        }
        __syncthreads();
        const int c = s_c;
        const unsigned long long r0 = s_r0, r1 = s_r1;
        uint32_t key[kRecsPerThread];
        float val[kRecsPerThread];
#pragma unroll
        for (int q = 0; q < kRecsPerThread; ++q) {
            const unsigned long long r =
                r0 + threadIdx.x + (unsigned long long)q * kRecThreads;
            const bool ok = r < r1;
            key[q] = ok ? __ldcs(pl.key1 + r) : 0xFFFFFFFFu;
            if (WEIGHTED)
                val[q] = ok ? __ldcs(pl.val1 + r) : 0.0f;
        }
        // each record's place among this chunk's records of its tile, kept
        // as 16-bit halves; the record's tile within the coarse bin is
        // (key >> 16) & (G - 1) for both coarse key forms
        const uint32_t gm = (uint32_t)(G - 1);
        uint32_t rk[kRecsPerThread / 2];
#pragma unroll
        for (int q = 0; q < kRecsPerThread; ++q) {
            const bool ok = key[q] != 0xFFFFFFFFu;
            const uint32_t r = ok ? atomicAdd(hist + ((key[q] >> 16) & gm), 1u) : 0u;
            if (q & 1)
                rk[q >> 1] |= r << 16;
            else
                rk[q >> 1] = r;
        }
        __syncthreads();
        scan_bins<kRecThreads>(hist, start, G, warp_tot, &s_total);
        constexpr int kResv = kMaxBins / kRecThreads;
        unsigned long long resv[kResv];
#pragma unroll
        for (int i = 0; i < kResv; ++i) {
            const int f = threadIdx.x + i * kRecThreads;
            resv[i] = 0ull;
            if (f < G) {
                const uint32_t h = hist[f];
                if (h != 0u)
                    resv[i] = atomicAdd(pl.fill2 + (int64_t)c * G + f,
                                        (unsigned long long)h);
            }
        }
#pragma unroll
        for (int q = 0; q < kRecsPerThread; ++q) {
            const bool ok = key[q] != 0xFFFFFFFFu;
            if (ok) {
                const uint32_t f = (key[q] >> 16) & gm;
                const uint32_t pos =
                    start[f] + ((rk[q >> 1] >> (16 * (q & 1))) & 0xFFFFu);
                sent[pos] = (f << 16) | (key[q] & 0xFFFFu);
                if (WEIGHTED)
                    sval[pos] = val[q];
            }
        }
#pragma unroll
        for (int i = 0; i < kResv; ++i) {
            const int f = threadIdx.x + i * kRecThreads;
            if (f >= G)
                continue;
            // unsigned wrap-around cancels when i is added.  Paired: an even
            // tile fills its pair's region from the start, an odd one from
            // the end (this run ends where the tile's previous run began)
            const int64_t g = (int64_t)c * G + f;
            const bool odd = pl.paired && (g & 1);
            const unsigned long long base =
                pl.off2[pl.paired ? (g >> 1) + (odd ? 1 : 0) : g];
            dst0[f] = odd ? base - resv[i] - hist[f] - start[f]
                          : base + resv[i] - start[f];
        }
        __syncthreads();
        const uint32_t total = s_total;
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
            const uint32_t e = sent[i];
            const unsigned long long dst = dst0[e >> 16] + i;
            pl.key2[dst] = (uint16_t)(e & 0xFFFFu);
            if (WEIGHTED)
                __stcs(pl.val2 + dst, sval[i]);
        }
        for (int f = threadIdx.x; f < G; f += blockDim.x)
            hist[f] = 0u;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- tiles
// Weighted cell: the float sum `hi` and the sum of the rounding errors of
// the additions made to it.  atomicAdd returns the value it added to, so
// the thread recomputes that one rounded addition and its exact error
// (TwoSum: Knuth, TAOCP vol. 2, 4.2.2) and adds the error to `lo`: hi + lo
// then carries the sum to about one float rounding, whatever the number
// and order of the additions.
__device__ __forceinline__ void compensated_add(float2 *cell, float x)
{
    const float old = atomicAdd(&cell->x, x);
    const float s = __fadd_rn(old, x);
    const float xp = __fsub_rn(s, old);
    const float op = __fsub_rn(s, xp);
    const float err = __fadd_rn(__fsub_rn(old, op), __fsub_rn(x, xp));
    if (err != 0.0f)
        atomicAdd(&cell->y, err);
}

// One CTA per SM; tiles drawn from a counter.  Per tile: add its records
// into the accumulators (cell j of the tile at acc[off + j], off = Z's
// float offset within 16 bytes, so that accumulator quads line up with
// 16-byte stores of Z), then convert and store its Z rows, clearing every
// accumulator read.  Two barriers per tile.
template <bool WEIGHTED, bool LAP>
__global__ void __launch_bounds__(kTileThreads, 1)
    k_bin_tiles(BinPlan pl, const BinProblem *P)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ long long s_tile[2];
    uint32_t *nk = reinterpret_cast<uint32_t *>(sm);
    float *table = reinterpret_cast<float *>(sm + 1024);
    unsigned char *accb =
        sm + 1024 + (WEIGHTED ? 0 : kMaxClasses * kTablePerClass * 4 + 32);
    uint32_t *acc = reinterpret_cast<uint32_t *>(accb);
    float2 *accw = reinterpret_cast<float2 *>(accb);
    constexpr int kCells = WEIGHTED ? kTileBytes / 8 : kTileBytes / 4;
    if (WEIGHTED)
        for (int j = threadIdx.x; j < kCells + 4; j += blockDim.x)
            accw[j] = make_float2(0.0f, 0.0f);
    else
        for (int j = threadIdx.x; j < kCells + 4; j += blockDim.x)
            acc[j] = 0u;
    int cur = -1;
    for (int it = 0;; ++it) {
        if (threadIdx.x == 0)
            s_tile[it & 1] = (long long)atomicAdd(pl.work, 1ull);
        __syncthreads();  // also ends the previous tile's write phase
        const long long t = s_tile[it & 1];
        if (t >= pl.tiles)
            break;
        const int pi = problem_of_tile(P, pl.problems, t);
        const BinProblem &p = P[pi];
        if (failed(p.st))
            continue;
        const int32_t K = p.K;
        if (pi != cur) {  // the problem's n_k (and small-count table)
            for (int k = threadIdx.x; k < K; k += blockDim.x)
                nk[k] = p.counts[k];
            if (!WEIGHTED)
                for (int i = threadIdx.x; i < K * kTablePerClass;
                     i += blockDim.x) {
                    const int k = i / kTablePerClass;
                    table[i] = count_to_z((uint32_t)(i - k * kTablePerClass),
                                          p.counts[k]);
                }
            cur = pi;
        }
        const int64_t r0 = (t - p.tile0) * (int64_t)p.rows;
        const int64_t r1 = min(r0 + (int64_t)p.rows, p.n);
        const int cells = (int)((r1 - r0) * K);
        float *z = p.Z + r0 * K;
        const int off = (int)((reinterpret_cast<uintptr_t>(z) >> 2) & 3);
        const unsigned long long rec0 = tile_records_start(pl, t);
        const long long nrec = (long long)pl.fill2[t];
        // -- accumulate: keys 8 at a time from a 16-byte boundary
        const uint16_t *k2 = pl.key2 + rec0;
        const float *v2 = pl.val2 + rec0;
        const int head = (int)min((long long)((8 - (rec0 & 7)) & 7), nrec);
        const long long nq = (nrec - head) >> 3;
        auto add1 = [&](uint32_t key, float x) {
            if (WEIGHTED)
                compensated_add(accw + off + key, x);
            else
                atomicAdd(acc + off + key, 1u);
        };
        if ((int)threadIdx.x < head)
            add1(k2[threadIdx.x], WEIGHTED ? v2[threadIdx.x] : 0.0f);
        const uint4 *k8 = reinterpret_cast<const uint4 *>(k2 + head);
        const float4 *v8 = reinterpret_cast<const float4 *>(v2 + head);
        // two groups of 8 records per thread per round, both loaded first
        auto add8 = [&](uint4 kk, float4 a, float4 b) {
            const uint32_t ks[8] = {kk.x & 0xFFFFu, kk.x >> 16,
                                    kk.y & 0xFFFFu, kk.y >> 16,
                                    kk.z & 0xFFFFu, kk.z >> 16,
                                    kk.w & 0xFFFFu, kk.w >> 16};
            const float xs[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                add1(ks[e], xs[e]);
        };
        const float4 f0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (long long q = threadIdx.x; q < nq; q += 2 * (long long)blockDim.x) {
            const long long q1 = q + blockDim.x;
            const bool two = q1 < nq;
            const uint4 k0 = __ldcs(k8 + q);
            const uint4 k1 = two ? __ldcs(k8 + q1) : make_uint4(0u, 0u, 0u, 0u);
            float4 a0 = f0, b0 = f0, a1 = f0, b1 = f0;
            if (WEIGHTED) {
                a0 = __ldcs(v8 + 2 * q);
                b0 = __ldcs(v8 + 2 * q + 1);
                if (two) {
                    a1 = __ldcs(v8 + 2 * q1);
                    b1 = __ldcs(v8 + 2 * q1 + 1);
                }
            }
            add8(k0, a0, b0);
            if (two)
                add8(k1, a1, b1);
        }
        {
            const long long t0 = head + 8 * nq;
            if ((long long)threadIdx.x < nrec - t0)
                add1(k2[t0 + threadIdx.x],
                     WEIGHTED ? v2[t0 + threadIdx.x] : 0.0f);
        }
        __syncthreads();
        // -- write the tile's rows: cell j of row r0 + j / K, class j % K
        const uint32_t kmagic = p.kmagic;
        auto class_of = [&](int j) -> int {
            return K == 1 ? 0 : j - K * (int)__umulhi((unsigned)j, kmagic);
        };
        auto row_of = [&](int j) -> int {
            return K == 1 ? j : (int)__umulhi((unsigned)j, kmagic);
        };
        auto value = [&](int j, int k) -> float {
            if (WEIGHTED) {
                const float2 c = accw[off + j];
                accw[off + j] = make_float2(0.0f, 0.0f);
                float v = sum_to_z(__fadd_rn(c.x, c.y), nk[k]);
                if (LAP)
                    v = __fmul_rn(v, __ldg(p.r + r0 + row_of(j)));
                return v;
            }
            const uint32_t c = acc[off + j];
            acc[off + j] = 0u;
            return c < (uint32_t)kTablePerClass ? table[k * kTablePerClass + c]
                                                : count_to_z(c, nk[k]);
        };
        const int zh = min((4 - off) & 3, cells);
        const int zq = (cells - zh) >> 2;
        if ((int)threadIdx.x < zh)
            __stcs(z + threadIdx.x, value(threadIdx.x, class_of(threadIdx.x)));
        // quads of cells: acc[off + j0] is 16-byte aligned (off + zh is a
        // multiple of 4); read and cleared whole, all-zero quads (isolated
        // rows, classes a row never sees) skip the conversion
        for (int q = threadIdx.x; q < zq; q += blockDim.x) {
            const int j0 = zh + 4 * q;
            float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (WEIGHTED) {
                float4 *a4 = reinterpret_cast<float4 *>(accw + off + j0);
                const float4 c01 = a4[0], c23 = a4[1];
                const float hi[4] = {c01.x, c01.z, c23.x, c23.z};
                const float lo[4] = {c01.y, c01.w, c23.y, c23.w};
                if ((hi[0] != 0.0f) | (hi[1] != 0.0f) | (hi[2] != 0.0f) |
                    (hi[3] != 0.0f) | (lo[0] != 0.0f) | (lo[1] != 0.0f) |
                    (lo[2] != 0.0f) | (lo[3] != 0.0f)) {
                    a4[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    a4[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    int k = class_of(j0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float v = sum_to_z(__fadd_rn(hi[e], lo[e]), nk[k]);
                        if (LAP)
                            v = __fmul_rn(v, __ldg(p.r + r0 + row_of(j0 + e)));
                        o[e] = v;
                        if (++k == K)
                            k = 0;
                    }
                }
            } else {
                uint4 *a4 = reinterpret_cast<uint4 *>(acc + off + j0);
                const uint4 c4 = *a4;
                if ((c4.x | c4.y | c4.z | c4.w) != 0u) {
                    *a4 = make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
                    int k = class_of(j0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t c = cs[e];
                        o[e] = c == 0u ? 0.0f
                               : c < (uint32_t)kTablePerClass
                                   ? table[k * kTablePerClass + c]
                                   : count_to_z(c, nk[k]);
                        if (++k == K)
                            k = 0;
                    }
                }
            }
            __stcs(reinterpret_cast<float4 *>(z + j0),
                   make_float4(o[0], o[1], o[2], o[3]));
        }
        {
            const int j = zh + 4 * zq + (int)threadIdx.x;
            if (j < cells)
                __stcs(z + j, value(j, class_of(j)));
        }
    }
}

template <class Kern>
cudaError_t with_smem(Kern k, size_t bytes)
{
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

size_t edges_smem(bool weighted)
{
    const size_t rec = 2 * kEdgeChunk;
    return kMaxBins * (4 + 4 + 8) + rec * (4 + 2 + (weighted ? 4 : 0));
}

size_t split_smem(bool weighted)
{
    return kMaxBins * (4 + 4 + 8) + (size_t)kRecChunk * (4 + (weighted ? 4 : 0));
}

size_t tiles_smem(bool weighted)
{
    const size_t cells = (weighted ? kTileBytes / 8 : kTileBytes / 4) + 4;
    return 1024 + (weighted ? 0 : kMaxClasses * kTablePerClass * 4 + 32) +
           cells * (weighted ? 8 : 4);
}

}  // namespace

// ---------------------------------------------------------------- host side
int32_t bin_rows(int32_t K, bool weighted)
{
    const int cells = weighted ? kTileBytes / 8 : kTileBytes / 4;
    int32_t r = 1;
    while (2 * r * K <= cells)
        r *= 2;
    return r;
}

bool bin_layout(int64_t tiles, int32_t *coarse, int32_t *group)
{
    if (tiles < 1)
        tiles = 1;
    if (tiles > (int64_t)kMaxBins * kMaxBins)
        return false;
    int64_t g = 1;
    while (g * g < tiles)
        g *= 2;
    const int64_t c = (tiles + g - 1) / g;
    *group = (int32_t)g;
    *coarse = (int32_t)c;
    return g <= kMaxBins && c <= kMaxBins;
}

size_t bin_scratch_bytes(int64_t records, int64_t tiles, bool weighted)
{
    int32_t coarse = 1, group = 1;
    bin_layout(tiles, &coarse, &group);
    const size_t fine = (size_t)coarse * group;
    size_t b = (size_t)records * (4 + 2) + 2 * 256;
    if (weighted)
        b += (size_t)records * 8 + 2 * 256;
    b += 8 * (4 * ((size_t)coarse + 1) + 3 * (fine + 1) + 1) + 4 * 256;
    return b;
}

cudaError_t bin_enqueue(Allocator &al, BinPlan &pl, const BinProblem *dP,
                        bool weighted, bool laplacian, cudaStream_t stream)
{
    const size_t fine = (size_t)pl.coarse * pl.group;
    unsigned long long *ctr = nullptr;
    // counters: cnt1, fill1, cnt2, fill2, work (zeroed together), then
    // off1, chunk1, off2
    const size_t zeroed = 2 * ((size_t)pl.coarse + 1) + 2 * (fine + 1) + 1;
    const size_t words = zeroed + 2 * ((size_t)pl.coarse + 1) + (fine + 1);
    cudaError_t e = al.alloc((void **)&ctr, 8 * words);
    if (e != cudaSuccess)
        return e;
    pl.cnt1 = ctr;
    pl.fill1 = pl.cnt1 + pl.coarse + 1;
    pl.cnt2 = pl.fill1 + pl.coarse + 1;
    pl.fill2 = pl.cnt2 + fine + 1;
    pl.work = pl.fill2 + fine + 1;
    pl.off1 = pl.work + 1;
    pl.chunk1 = pl.off1 + pl.coarse + 1;
    pl.off2 = pl.chunk1 + pl.coarse + 1;
    const size_t recs = (size_t)(pl.records > 0 ? pl.records : 1);
    if ((e = al.alloc((void **)&pl.key1, recs * 4)) != cudaSuccess ||
        (e = al.alloc((void **)&pl.key2, recs * 2 + 16)) != cudaSuccess)
        return e;
    pl.val1 = nullptr;
    pl.val2 = nullptr;
    if (weighted &&
        ((e = al.alloc((void **)&pl.val1, recs * 4)) != cudaSuccess ||
         (e = al.alloc((void **)&pl.val2, recs * 4 + 32)) != cudaSuccess))
        return e;
    if ((e = cudaMemsetAsync(ctr, 0, 8 * zeroed, stream)) != cudaSuccess)
        return e;
    const int sms = sm_count();
    auto grid = [&](int64_t work, int per_sm) {
        return (int)std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)sms * per_sm));
    };
    // tile records by pair while the pairs' counters fit one CTA's shared
    // memory (and the coarse keys hold whole tile numbers)
    const int64_t pairs = (pl.tiles + 1) >> 1;
    pl.paired = pl.tiles <= 65536 && pairs <= kMaxPairs ? 1 : 0;
    if (pl.paired) {
        if (pl.edge_chunks > 0) {
            ProfScope p("k_bin_count_pairs", stream);
            const size_t sm_b = (size_t)pairs * 4;
            if ((e = with_smem(k_bin_count_pairs, sm_b)) != cudaSuccess)
                return e;
            k_bin_count_pairs<<<grid((pl.edge_chunks + 1) / 2, 1), kPairThreads,
                                sm_b, stream>>>(pl, dP);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return e;
        }
        {
            ProfScope p("k_bin_scan", stream);
            k_bin_scan<<<1, 1024, 0, stream>>>(pl.cnt2, pairs, 0, pl.off2);
        }
        {
            ProfScope p("k_bin_pair_coarse", stream);
            k_bin_pair_coarse<<<(pl.coarse + 256) / 256, 256, 0, stream>>>(pl);
        }
    } else {
        if (pl.edge_chunks > 0) {
            ProfScope p("k_bin_count", stream);
            k_bin_count<<<grid(pl.edge_chunks, 4), kEdgeThreads,
                          (size_t)pl.coarse * 4, stream>>>(pl, dP);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return e;
        }
        {
            ProfScope p("k_bin_scan", stream);
            k_bin_scan<<<1, 1024, 0, stream>>>(pl.cnt1, pl.coarse, 0, pl.off1);
        }
    }
    if (pl.edge_chunks > 0) {
        ProfScope p("k_bin_edges", stream);
        const size_t sm_b = edges_smem(weighted);
        const int blocks = grid(pl.edge_chunks, 2);
        // record keys hold the whole tile number up to 2^16 tiles
        const bool wide = pl.tiles > 65536;
        auto go = [&](auto kern) -> cudaError_t {
            cudaError_t r = with_smem(kern, sm_b);
            if (r == cudaSuccess)
                kern<<<blocks, kEdgeThreads, sm_b, stream>>>(pl, dP);
            return r;
        };
        if (!weighted)
            e = wide ? go(k_bin_edges<false, false, true>)
                     : go(k_bin_edges<false, false, false>);
        else if (!laplacian)
            e = wide ? go(k_bin_edges<true, false, true>)
                     : go(k_bin_edges<true, false, false>);
        else
            e = wide ? go(k_bin_edges<true, true, true>)
                     : go(k_bin_edges<true, true, false>);
        if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    {
        ProfScope p("k_bin_scan", stream);
        k_bin_scan<<<1, 1024, 0, stream>>>(pl.fill1, pl.coarse, 1, pl.chunk1);
    }
    const int64_t chunk_bound = pl.records / kRecChunk + pl.coarse;
    if (!pl.paired) {
        {
            ProfScope p("k_bin_fine", stream);
            k_bin_fine<<<grid(chunk_bound, 8), kRecThreads, (size_t)pl.group * 4,
                         stream>>>(pl);
        }
        {
            ProfScope p("k_bin_scan", stream);
            k_bin_scan<<<1, 1024, 0, stream>>>(pl.cnt2, (int64_t)fine, 0, pl.off2);
        }
    }
    {
        ProfScope p("k_bin_split", stream);
        const size_t sm_b = split_smem(weighted);
        if (weighted) {
            if ((e = with_smem(k_bin_split<true>, sm_b)) != cudaSuccess)
                return e;
            k_bin_split<true>
                <<<grid(chunk_bound, kSplitBlocks), kRecThreads, sm_b, stream>>>(pl);
        } else {
            if ((e = with_smem(k_bin_split<false>, sm_b)) != cudaSuccess)
                return e;
            k_bin_split<false>
                <<<grid(chunk_bound, kSplitBlocks), kRecThreads, sm_b, stream>>>(pl);
        }
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    if (pl.tiles > 0) {
        ProfScope p("k_bin_tiles", stream);
        const size_t sm_b = tiles_smem(weighted);
        const int blocks = grid(pl.tiles, 1);
        if (!weighted) {
            if ((e = with_smem(k_bin_tiles<false, false>, sm_b)) != cudaSuccess)
                return e;
            k_bin_tiles<false, false><<<blocks, kTileThreads, sm_b, stream>>>(pl, dP);
        } else if (!laplacian) {
            if ((e = with_smem(k_bin_tiles<true, false>, sm_b)) != cudaSuccess)
                return e;
            k_bin_tiles<true, false><<<blocks, kTileThreads, sm_b, stream>>>(pl, dP);
        } else {
            if ((e = with_smem(k_bin_tiles<true, true>, sm_b)) != cudaSuccess)
                return e;
            k_bin_tiles<true, true><<<blocks, kTileThreads, sm_b, stream>>>(pl, dP);
        }
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_binned(Allocator &al, const int32_t *E, const float *w,
                          int64_t s, int64_t n, int32_t K, const uint8_t *Yc,
                          const float *r, const uint32_t *counts, float *Z,
                          DevStatus *st, cudaStream_t stream)
{
    const bool weighted = (w != nullptr) || (r != nullptr);
    BinProblem hp{};
    hp.E = E;
    hp.w = w;
    hp.s = s;
    hp.n = n;
    hp.Yc = Yc;
    hp.r = r;
    hp.Z = Z;
    hp.counts = counts;
    hp.st = st;
    hp.K = K;
    hp.rows = bin_rows(K, weighted);
    hp.row_shift = (uint32_t)__builtin_ctz((unsigned)hp.rows);
    hp.kmagic = K > 1 ? (uint32_t)(0xFFFFFFFFull / (uint32_t)K + 1ull) : 0u;
    hp.tile0 = 0;
    hp.tiles = (n + hp.rows - 1) / hp.rows;
    hp.chunk0 = 0;
    BinPlan pl{};
    pl.problems = 1;
    pl.tiles = hp.tiles;
    pl.edge_chunks = (s + kEdgeChunk - 1) / kEdgeChunk;
    pl.records = 2 * s;
    if (!bin_layout(pl.tiles, &pl.coarse, &pl.group))
        return cudaErrorInvalidValue;
    pl.group_shift = (uint32_t)__builtin_ctz((unsigned)pl.group);
    BinProblem *dP = nullptr;
    cudaError_t e = al.alloc((void **)&dP, sizeof(BinProblem));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dP, &hp, sizeof(hp), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
        return e;
    return bin_enqueue(al, pl, dP, weighted, r != nullptr, stream);
}

int64_t binned_batch_tiles(const BatchProblem *P, int count)
{
    bool weighted = false;
    for (int i = 0; i < count; ++i)
        weighted |= P[i].w != nullptr;
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t rows = bin_rows(P[i].K, weighted);
        tiles += (P[i].n + rows - 1) / rows;
    }
    int32_t coarse = 0, group = 0;
    return bin_layout(tiles, &coarse, &group) ? tiles : 0;
}

cudaError_t launch_binned_batch(Allocator &al, const BatchProblem *P,
                                int count, cudaStream_t stream)
{
    bool weighted = false;
    for (int i = 0; i < count; ++i)
        weighted |= P[i].w != nullptr;
    std::vector<BinProblem> hp((size_t)count);
    int64_t tiles = 0, chunks = 0, records = 0;
    for (int i = 0; i < count; ++i) {
        const BatchProblem &q = P[i];
        BinProblem &b = hp[(size_t)i];
        b = BinProblem{};
        b.E = q.E;
        b.w = q.w;
        b.s = q.s;
        b.n = q.n;
        b.Yc = q.Yc;
        b.r = nullptr;
        b.Z = q.Z;
        b.counts = q.counts;
        b.st = q.st;
        b.K = q.K;
        b.rows = bin_rows(q.K, weighted);
        b.row_shift = (uint32_t)__builtin_ctz((unsigned)b.rows);
        b.kmagic = q.K > 1 ? (uint32_t)(0xFFFFFFFFull / (uint32_t)q.K + 1ull) : 0u;
        b.tile0 = tiles;
        b.tiles = (q.n + b.rows - 1) / b.rows;
        b.chunk0 = chunks;
        tiles += b.tiles;
        chunks += (q.s + kEdgeChunk - 1) / kEdgeChunk;
        records += 2 * q.s;
    }
    BinPlan pl{};
    pl.problems = count;
    pl.tiles = tiles;
    pl.edge_chunks = chunks;
    pl.records = records;
    if (count < 1 || !bin_layout(tiles, &pl.coarse, &pl.group))
        return cudaErrorInvalidValue;
    pl.group_shift = (uint32_t)__builtin_ctz((unsigned)pl.group);
    BinProblem *dP = nullptr;
    cudaError_t e = al.alloc((void **)&dP, sizeof(BinProblem) * count);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dP, hp.data(), sizeof(BinProblem) * count,
                            cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
        return e;
    return bin_enqueue(al, pl, dP, weighted, false, stream);
}

}  // namespace gee
