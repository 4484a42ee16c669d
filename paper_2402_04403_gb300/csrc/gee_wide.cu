// gee_wide.cu -- the pull pass for many label vectors at once.
//
// With L label vectors the widened W has L*K columns (one block of K per
// vector) and every arc (u -> v) adds to L cells of row u: cell (l, Y_l[v])
// for each l.  Here the lanes of a warp take the L labels of one arc instead
// of 32 different arcs: lane l reads byte l of the target's label record
// (Yc[v*Ls + l], one 32-byte sector per arc for L <= 32) and adds to its
// own accumulator column.  No two lanes ever touch the same cell, so the
// accumulation needs neither atomics nor a fixed summation order to be
// exact: it is deterministic for float weights too.
//
// Accumulators of a warp are class-major, acc[(j*K + k)*32 + lane] for label
// l = 32*j + lane, so every update of a warp hits 32 different banks.  A Z
// row is node-major (column l*K + k); it is transposed through a per-warp
// stage buffer with an odd row pitch (conflict-free on both sides) and
// written with coalesced stores.
//
// k_wide_rows:   rows with at most kHubDegree arcs; warps take batches of
//                rows from a global counter; rows without arcs (isolated
//                nodes and hub rows) get zeros.
// k_wide_chunks: hub rows in chunks of kHubChunk arcs, one warp per chunk,
//                warps take contiguous chunk ranges of equal arc counts;
//                single-chunk rows are written directly (after the zeros of
//                k_wide_rows), longer rows leave raw partial sums for
//                k_hub_fixup, in Z's column order.
#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kRowBatch = 32;   // rows a warp takes per grab
constexpr int kUnrollArcs = 8;  // label loads in flight per lane (4 arcs each)
constexpr int kMaxWarps = 32;
constexpr int kSmallCounts = 8;  // counts below this convert by table

struct WideArgs {
    const int64_t *rowptr;
    const int32_t *col;
    const float *val;
    int64_t n;
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
    const uint32_t *counts;  // [L*K], column order
    float *Z;
    uint32_t *hub_part;      // [chunks * cols]
    unsigned long long *work;
    const DevStatus *st;
    int32_t L, Ls, K, cols;
    int32_t Lb;              // label blocks of 32 lanes: ceil(L / 32)
    int32_t Kp;              // stage row pitch: K rounded up to odd
    int32_t vec;             // K % 4 == 0 and Z 16-byte aligned: lanes
                             // write their own cells, tables class-major
    int32_t table_off;       // shared memory: [nk][table][per-warp areas]
    int32_t area_off;
    int32_t acc_bytes;       // per warp: accumulators (K + 1 rows per block
                             // of 32 labels, the last a sink), then stage
    int32_t warp_bytes;
};

// Position of this lane's first Z column (c = lane) in the stage buffer and
// how it moves when c advances by 32.
struct StageWalk {
    int k, s;       // class of column c, stage index l*Kp + k
    int dk, ds;     // per step of 32 columns, before the carry
};

__device__ __forceinline__ StageWalk stage_walk(const WideArgs &a, int lane)
{
    StageWalk w;
    const int l = lane / a.K;
    w.k = lane - l * a.K;
    w.s = l * a.Kp + w.k;
    w.dk = 32 % a.K;
    w.ds = (32 / a.K) * a.Kp + w.dk;
    return w;
}

// Adds the arcs [0, NA) at colp/valp.  32 arcs are loaded at a time (one
// per lane); their label records are then fetched cooperatively -- eight
// lanes per 32-byte block of a record, one word each, so one load
// instruction covers four arcs and all 32 arcs' labels are in flight at
// once -- and every lane takes its own byte of each record by a shuffle.
// Labels are below K or 255 (unknown, and the padding bytes of a record):
// min(y, K) sends the latter to the block's sink row K, which is never read.
template <bool WEIGHTED>
__device__ __forceinline__ void wide_sweep(const WideArgs &a,
                                           const int32_t *colp,
                                           const float *valp, int64_t NA,
                                           int lane, uint32_t *acc)
{
    constexpr unsigned kAll = 0xffffffffu;
    uint32_t *accl = acc + lane;         // this lane's accumulator column
    float *accf = reinterpret_cast<float *>(accl);
    const int slot = lane >> 3;          // arc slot of this lane's loads
    const int word_off = (lane & 7) * 4; // its word within a 32-byte block
    const int holder = lane >> 2;        // lane (of an arc's 8) with my byte
    const uint32_t pick = 0x4440u | (lane & 3);  // byte_perm: my byte, zeros
    for (int64_t base = 0; base < NA; base += 32) {
        const int m = (int)min((int64_t)32, NA - base);
        int32_t c = 0;
        float w = 0.0f;
        if (lane < m) {
            c = __ldcs(colp + base + lane);
            if (WEIGHTED)
                w = __ldcs(valp + base + lane);
        }
        // record of arc 4u + slot, or none past the end
        const uint8_t *rec[kUnrollArcs];
#pragma unroll
        for (int u = 0; u < kUnrollArcs; ++u) {
            const int32_t v = __shfl_sync(kAll, c, 4 * u + slot);
            rec[u] = 4 * u + slot < m ? a.Yc + (int64_t)v * a.Ls + word_off
                                      : nullptr;
        }
        for (int j = 0; j < a.Lb; ++j) {
            uint32_t word[kUnrollArcs];
#pragma unroll
            for (int u = 0; u < kUnrollArcs; ++u)
                word[u] = rec[u] != nullptr
                              ? __ldg(reinterpret_cast<const uint32_t *>(
                                    rec[u] + 32 * j))
                              : 0xffffffffu;
            // block j's rows: classes j*(K+1) + k, then its sink row
            const int row0 = j * (a.K + 1);
#pragma unroll
            for (int u = 0; u < kUnrollArcs; ++u) {
                if (4 * u < m) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t wd =
                            __shfl_sync(kAll, word[u], (e << 3) | holder);
                        const int r =
                            row0 + min((int)__byte_perm(wd, 0u, pick), a.K);
                        if (WEIGHTED)
                            accf[r * 32] += __shfl_sync(kAll, w, 4 * u + e);
                        else
                            accl[r * 32] += 1u;
                    }
                }
            }
        }
    }
}

// Z value of a cell.  Count path: RN32(C / n_k), by table below
// kSmallCounts.  Weighted path: nk holds the bits of RN32(1/n_k) (0 for an
// empty class) and the weight sum is multiplied by it -- the per-class
// factor 1/n_k of W (Alg. 1), applied once per cell.
template <bool WEIGHTED>
__device__ __forceinline__ float wide_value(uint32_t x, int c,
                                            const uint32_t *nk,
                                            const float *table)
{
    if (WEIGHTED)
        return __fmul_rn(__uint_as_float(x), __uint_as_float(nk[c]));
    return x < (uint32_t)kSmallCounts ? table[c * kSmallCounts + x]
                                      : count_to_z(x, nk[c]);
}

// Moves the warp's accumulators into node-major order (zeroing them for the
// next row) and writes the row: Z values (TO_Z) or the raw sums.
template <bool WEIGHTED, bool TO_Z>
__device__ __forceinline__ void wide_emit(const WideArgs &a, uint32_t *acc,
                                          uint32_t *stage,
                                          const uint32_t *nk,
                                          const float *table, float *out,
                                          int lane, const StageWalk &sw)
{
    for (int j = 0; j < a.Lb; ++j) {
        const int l = 32 * j + lane;
        uint32_t *col = acc + j * (a.K + 1) * 32 + lane;
        uint32_t *srow = stage + l * a.Kp;
        for (int k = 0; k < a.K; ++k) {
            const uint32_t x = col[k * 32];
            col[k * 32] = 0u;
            if (l < a.L)
                srow[k] = x;
        }
    }
    __syncwarp();
    int k = sw.k, s = sw.s;
    for (int c = lane; c < a.cols; c += 32) {
        const uint32_t x = stage[s];
        if (TO_Z)
            __stcs(out + c, wide_value<WEIGHTED>(x, c, nk, table));
        else
            reinterpret_cast<uint32_t *>(out)[c] = x;
        k += sw.dk;
        s += sw.ds;
        if (k >= a.K) {
            k -= a.K;
            s += a.Kp - a.K;
        }
    }
    __syncwarp();
}

// The same when a lane's K cells are 16-byte aligned in Z (K % 4 == 0):
// lane l writes cells l*K .. l*K+K-1 straight from its accumulator column
// with 16-byte stores, no transposition.  n_k and the small-count table are
// class-major here (entry (j*K + k)*32 + lane), so lookups are conflict-free.
template <bool WEIGHTED, bool TO_Z>
__device__ __forceinline__ void wide_emit_vec(const WideArgs &a, uint32_t *acc,
                                              const uint32_t *nk,
                                              const float *table, float *out,
                                              int lane)
{
    for (int j = 0; j < a.Lb; ++j) {
        const int l = 32 * j + lane;
        uint32_t *col = acc + j * (a.K + 1) * 32 + lane;
        const uint32_t *nkc = nk + j * a.K * 32 + lane;
        const float *tc = table + j * a.K * 32 * kSmallCounts + lane;
        float4 *o = reinterpret_cast<float4 *>(out + (int64_t)l * a.K);
        for (int k = 0; k < a.K; k += 4) {
            uint32_t x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                x[e] = col[(k + e) * 32];
                col[(k + e) * 32] = 0u;
            }
            if (l < a.L) {
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (!TO_Z)
                        v[e] = __uint_as_float(x[e]);
                    else if (WEIGHTED)
                        v[e] = __fmul_rn(__uint_as_float(x[e]),
                                         __uint_as_float(nkc[(k + e) * 32]));
                    else
                        v[e] = x[e] < (uint32_t)kSmallCounts
                                   ? tc[((k + e) * kSmallCounts + x[e]) * 32]
                                   : count_to_z(x[e], nkc[(k + e) * 32]);
                }
                const float4 q = make_float4(v[0], v[1], v[2], v[3]);
                if (TO_Z)
                    __stcs(o + k / 4, q);
                else
                    o[k / 4] = q;
            }
        }
    }
}

// CTA prologue: n_k and the Z values of small counts in shared memory, all
// accumulators zero.
template <bool WEIGHTED>
__device__ __forceinline__ void wide_prologue(const WideArgs &a,
                                              unsigned char *sm)
{
    uint32_t *nk = reinterpret_cast<uint32_t *>(sm);
    float *table = reinterpret_cast<float *>(sm + a.table_off);
    // n_k, or for weights the bits of RN32(1/n_k) (a single rounding: the
    // double quotient is rounded again to float, innocuous since 53 >= 2*24+2)
    auto entry = [&](int c) -> uint32_t {
        const uint32_t n = a.counts[c];
        if (!WEIGHTED)
            return n;
        return n == 0u ? 0u
                       : __float_as_uint(__double2float_rn(1.0 / (double)n));
    };
    if (a.vec) {
        // entry (j*K + k)*32 + lane belongs to column (32j + lane)*K + k
        const int cells = a.Lb * a.K * 32;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int l = (i / (a.K * 32)) * 32 + (i & 31);
            const int k = (i >> 5) % a.K;
            nk[i] = l < a.L ? entry(l * a.K + k) : 0u;
        }
        if (!WEIGHTED)
            for (int i = threadIdx.x; i < cells * kSmallCounts; i += blockDim.x) {
                const int lane = i & 31;
                const int x = (i >> 5) % kSmallCounts;
                const int jk = (i >> 5) / kSmallCounts;  // j*K + k
                const int l = (jk / a.K) * 32 + lane;
                table[i] = l < a.L ? count_to_z((uint32_t)x,
                                                a.counts[l * a.K + jk % a.K])
                                   : 0.0f;
            }
    } else {
        for (int c = threadIdx.x; c < a.cols; c += blockDim.x)
            nk[c] = entry(c);
        if (!WEIGHTED)
            for (int i = threadIdx.x; i < a.cols * kSmallCounts; i += blockDim.x) {
                const int c = i / kSmallCounts;
                table[i] = count_to_z((uint32_t)(i - c * kSmallCounts), a.counts[c]);
            }
    }
    const int warps = blockDim.x >> 5;
    const int words = a.acc_bytes / 4;
    for (int i = threadIdx.x; i < warps * words; i += blockDim.x) {
        const int w = i / words;
        reinterpret_cast<uint32_t *>(sm + a.area_off +
                                     (size_t)w * a.warp_bytes)[i - w * words] =
            0u;
    }
    __syncthreads();
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kMaxWarps * 32, 1) k_wide_rows(WideArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (failed(a.st))
        return;
    wide_prologue<WEIGHTED>(a, sm);
    const uint32_t *nk = reinterpret_cast<const uint32_t *>(sm);
    const float *table = reinterpret_cast<const float *>(sm + a.table_off);
    const int lane = threadIdx.x & 31;
    unsigned char *ws = sm + a.area_off + (size_t)(threadIdx.x >> 5) * a.warp_bytes;
    uint32_t *acc = reinterpret_cast<uint32_t *>(ws);
    uint32_t *stage = reinterpret_cast<uint32_t *>(ws + a.acc_bytes);
    const StageWalk sw = stage_walk(a, lane);
    for (;;) {
        unsigned long long r0 = 0;
        if (lane == 0)
            r0 = atomicAdd(a.work, (unsigned long long)kRowBatch);
        r0 = __shfl_sync(0xffffffffu, r0, 0);
        if (r0 >= (unsigned long long)a.n)
            break;
        const int nr = (int)min((int64_t)kRowBatch, a.n - (int64_t)r0);
        // the batch's row starts, one per lane, and the end of its last row
        int64_t rp = 0;
        if (lane < nr)
            rp = a.rowptr[r0 + lane];
        const int64_t last = a.rowptr[r0 + nr];
        for (int i = 0; i < nr; ++i) {
            const int64_t b = __shfl_sync(0xffffffffu, rp, i);
            const int64_t next = __shfl_sync(0xffffffffu, rp, (i + 1) & 31);
            const int64_t e = i + 1 < nr ? next : last;
            float *z = a.Z + (int64_t)(r0 + i) * a.cols;
            if (b == e) {
                if (a.vec)
                    for (int c = lane; c < a.cols / 4; c += 32)
                        __stcs(reinterpret_cast<float4 *>(z) + c,
                               make_float4(0.0f, 0.0f, 0.0f, 0.0f));
                else
                    for (int c = lane; c < a.cols; c += 32)
                        __stcs(z + c, 0.0f);
                continue;
            }
            wide_sweep<WEIGHTED>(a, a.col + b, WEIGHTED ? a.val + b : nullptr,
                                 e - b, lane, acc);
            if (a.vec)
                wide_emit_vec<WEIGHTED, true>(a, acc, nk, table, z, lane);
            else
                wide_emit<WEIGHTED, true>(a, acc, stage, nk, table, z, lane, sw);
        }
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kMaxWarps * 32, 1) k_wide_chunks(WideArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (failed(a.st))
        return;
    wide_prologue<WEIGHTED>(a, sm);
    const uint32_t *nk = reinterpret_cast<const uint32_t *>(sm);
    const float *table = reinterpret_cast<const float *>(sm + a.table_off);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *ws = sm + a.area_off + (size_t)wib * a.warp_bytes;
    uint32_t *acc = reinterpret_cast<uint32_t *>(ws);
    uint32_t *stage = reinterpret_cast<uint32_t *>(ws + a.acc_bytes);
    const StageWalk sw = stage_walk(a, lane);
    // this warp's chunks: those whose first arc lies in its equal share of
    // the hub arcs (chunk_begin is increasing)
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    auto first_chunk_at = [&](int64_t arc) {
        int64_t lo = 0, hi = a.chunks;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (a.chunk_begin[mid] < arc)
                lo = mid + 1;
            else
                hi = mid;
        }
        return lo;
    };
    const int64_t c_lo = first_chunk_at(a.hub_arcs * w / nw);
    const int64_t c_hi = first_chunk_at(a.hub_arcs * (w + 1) / nw);
    for (int64_t c = c_lo; c < c_hi; ++c) {
        const int32_t h = a.chunk_hub[c];
        const int64_t b = a.chunk_begin[c];
        const int64_t hend = a.hub_ptr[h + 1];
        const int64_t NA = (b + kHubChunk < hend ? b + kHubChunk : hend) - b;
        wide_sweep<WEIGHTED>(a, a.col_h + b, WEIGHTED ? a.val_h + b : nullptr,
                             NA, lane, acc);
        const bool whole = a.hub_chunk0[h + 1] - a.hub_chunk0[h] == 1;
        float *out = whole ? a.Z + (int64_t)a.hub_row[h] * a.cols
                           : reinterpret_cast<float *>(a.hub_part + c * a.cols);
        if (a.vec) {
            if (whole)
                wide_emit_vec<WEIGHTED, true>(a, acc, nk, table, out, lane);
            else
                wide_emit_vec<WEIGHTED, false>(a, acc, nk, table, out, lane);
        } else {
            if (whole)
                wide_emit<WEIGHTED, true>(a, acc, stage, nk, table, out, lane, sw);
            else
                wide_emit<WEIGHTED, false>(a, acc, stage, nk, table, out, lane, sw);
        }
    }
}

inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

int max_shared_optin()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               dev) != cudaSuccess ||
        v <= 0)
        return 48 * 1024;
    return v;
}

// Fills the argument block and returns the shared-memory bytes and warps
// per CTA (as many as fit, at most kMaxWarps); 0 warps if none fits.
size_t wide_plan(const Csr &g, int32_t L, int32_t K, bool weighted,
                 bool laplacian, const uint8_t *Yc, const uint32_t *counts,
                 float *Z, void *hub_part, unsigned long long *work,
                 const DevStatus *st, WideArgs &a, int &warps)
{
    a = WideArgs{};
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.val = laplacian ? g.lap_val : g.val;
    a.n = g.n;
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
    a.K = K;
    a.cols = L * K;
    a.Lb = (L + 31) / 32;
    a.Kp = K | 1;
    a.vec = (K % 4 == 0) && (reinterpret_cast<uintptr_t>(Z) & 15) == 0;
    const bool w = weighted || laplacian;
    const size_t tcells = a.vec ? (size_t)a.Lb * K * 32 : (size_t)a.cols;
    a.table_off = (int32_t)align16(tcells * 4);
    a.area_off = a.table_off +
                 (int32_t)(w ? 0 : align16(tcells * kSmallCounts * 4));
    a.acc_bytes = (int32_t)((size_t)a.Lb * (K + 1) * 32 * 4);
    a.warp_bytes = a.acc_bytes + (int32_t)align16((size_t)L * a.Kp * 4);
    const int64_t room = (int64_t)max_shared_optin() - a.area_off;
    int64_t fit = room > 0 ? room / a.warp_bytes : 0;
    warps = (int)(fit < kMaxWarps ? fit : kMaxWarps);
    return (size_t)a.area_off + (size_t)warps * a.warp_bytes;
}

template <class Kern>
cudaError_t launch_wide(Kern kernel, int warps, size_t smem, const WideArgs &a,
                        cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(
        kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kernel<<<sm_count(), warps * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wide_rows(const Csr &g, int32_t L, int32_t K,
                             bool weighted, bool laplacian, const uint8_t *Yc,
                             const uint32_t *counts, float *Z,
                             unsigned long long *work, const DevStatus *st,
                             cudaStream_t stream)
{
    if (g.n == 0)
        return cudaSuccess;
    WideArgs a;
    int warps = 0;
    const size_t smem = wide_plan(g, L, K, weighted, laplacian, Yc, counts, Z,
                                  nullptr, work, st, a, warps);
    if (warps == 0)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess)
        return e;
    return (weighted || laplacian)
               ? launch_wide(k_wide_rows<true>, warps, smem, a, stream)
               : launch_wide(k_wide_rows<false>, warps, smem, a, stream);
}

cudaError_t launch_wide_chunks(const Csr &g, int32_t L, int32_t K,
                               bool weighted, bool laplacian,
                               const uint8_t *Yc, const uint32_t *counts,
                               float *Z, void *hub_part, const DevStatus *st,
                               cudaStream_t stream)
{
    if (g.chunks == 0)
        return cudaSuccess;
    WideArgs a;
    int warps = 0;
    const size_t smem = wide_plan(g, L, K, weighted, laplacian, Yc, counts, Z,
                                  hub_part, nullptr, st, a, warps);
    if (warps == 0)
        return cudaErrorInvalidConfiguration;
    return (weighted || laplacian)
               ? launch_wide(k_wide_chunks<true>, warps, smem, a, stream)
               : launch_wide(k_wide_chunks<false>, warps, smem, a, stream);
}

}  // namespace gee
