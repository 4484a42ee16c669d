// gee_batch.cu -- many independent embeddings in one sequence of persistent
// launches.
//
// A batch is a list of problems, each an edge list with its own n, K, label
// vector, optional weights and output Z -- the edge-list form of S1-S5
// (Alg. 1) applied to every problem.  Small graphs cannot fill the GPU one
// call at a time and would pay a handful of launches and a host round trip
// each; here every phase is one persistent launch over the chunks of all
// problems:
//
//   k_batch_init      status words and class counts of every problem
//   k_batch_labels    S1+S2: validate Y, compact labels, histogram n_k
//   k_batch_validate  endpoints in [0, n) (optional)
//   k_batch_zero      Z = 0
//   k_batch_scatter   S4: red.global adds into Z (uint32 counts in Z's bytes
//                     for unit weights, FP32 weight sums otherwise)
//   k_batch_finalize  S5: Z = RN32(C / n_k), or sum / n_k
//
// Warps take fixed-size chunks from one counter per phase, in problem
// order, so the few problems in flight at any time keep their Z in L2 while
// the atomics land.  The scatter's chunks are small (kBatchEdgeChunk = 1,024
// edges) because its working set is the Z rows of every chunk in flight,
// one per warp: 4,096 graphs of 1e3-1e5 nodes took 31.9 ms in the scatter
// with 4,096-edge chunks, 21.4 ms with 1,024.  Its bound is then the L2's
// tag lookups (74.7 % busy: two reductions and two label reads per edge);
// chunks dealt to warps statically (78 ms), drawn from 16 counters (39 ms),
// whole-CTA spans with the labels in shared memory (60 ms), or one launch
// that clears, adds and finishes each problem in turn under bounded waits
// (38.6 ms against 27 ms for the three launches) were all slower.  A
// problem whose labels or endpoints fail validation is skipped by the later
// phases and its Z is left untouched.  The launch
// arguments are only the device addresses of the header and the problem
// table, so one CUDA graph of the sequence serves every batch that reuses
// those two buffers.
#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kBatchThreads = 512;
constexpr int kUnroll = 4;  // independent elements per lane in flight
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int64_t kValidateSpan =
    kBatchEdgeChunk >= 4096 ? 1 : 4096 / kBatchEdgeChunk;

__device__ __forceinline__ int64_t chunk0_of(const BatchProblem &p, int kind)
{
    return kind == kChunkNodes ? p.node_chunk0
                               : (kind == kChunkEdges ? p.edge_chunk0
                                                      : p.cell_chunk0);
}

// Problem owning global chunk c of a kind: the last with chunk0 <= c.
__device__ __forceinline__ int find_problem(const BatchProblem *P, int count,
                                            int kind, int64_t c)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk0_of(P[mid], kind) <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Next chunk of a phase for this warp (lane 0 draws, all lanes get it).
__device__ __forceinline__ int64_t next_chunk(BatchHeader *h, int counter)
{
    unsigned long long c = 0;
    if ((threadIdx.x & 31) == 0)
        c = atomicAdd(&h->work[counter], 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, c, 0);
}

__global__ void k_batch_init(BatchHeader *h, const BatchProblem *P)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    if (tid < kWorkCounters)
        h->work[tid] = 0ull;
    for (int64_t p = tid; p < h->count; p += nth) {
        DevStatus *st = P[p].st;
        st->code = 0;
        st->aux = 0;
        st->index = ~0ull;
    }
    for (int64_t i = tid; i < h->count_cells; i += nth)
        h->counts[i] = 0u;
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_labels(BatchHeader *h, const BatchProblem *P)
{
    __shared__ uint32_t hist_all[kBatchWarps][256];
    const int lane = threadIdx.x & 31;
    uint32_t *hist = hist_all[threadIdx.x >> 5];
    for (int k = lane; k < 256; k += 32)
        hist[k] = 0u;
    __syncwarp();
    for (;;) {
        const int64_t c = next_chunk(h, kWorkLabels);
        if (c >= h->node_chunks)
            break;
        const BatchProblem &p = P[find_problem(P, (int)h->count, kChunkNodes, c)];
        const int64_t i0 = (c - p.node_chunk0) * kBatchNodeChunk;
        const int64_t i1 = min(i0 + kBatchNodeChunk, p.n);
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const int32_t y = __ldcs(p.Y + i);
            uint32_t code = kNoLabel;
            if ((uint32_t)y < (uint32_t)p.K) {
                atomicAdd(&hist[y], 1u);
                code = (uint32_t)y;
            } else if (y != -1) {
                report(p.st, GEE_ERR_LABEL_RANGE, (unsigned long long)i);
            }
            p.Yc[i] = (uint8_t)code;
        }
        __syncwarp();
        for (int k = lane; k < p.K; k += 32) {
            if (hist[k] != 0u) {
                atomicAdd(p.counts + k, hist[k]);
                hist[k] = 0u;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_validate(BatchHeader *h, const BatchProblem *P)
{
    const int lane = threadIdx.x & 31;
    int64_t c = 0, last = 0;  // this warp's next chunk and the end of its draw
    for (;;) {
        if (c == last) {
            // no locality to keep here: kValidateSpan chunks per draw
            c = next_chunk(h, kWorkValidate) * kValidateSpan;
            last = c + kValidateSpan;
        }
        if (c >= h->edge_chunks)
            break;
        const BatchProblem &p = P[find_problem(P, (int)h->count, kChunkEdges, c)];
        ++c;
        const int64_t e0 = (c - 1 - p.edge_chunk0) * kBatchEdgeChunk;
        const int64_t e1 = min(e0 + kBatchEdgeChunk, p.s);
        const int2 *E = reinterpret_cast<const int2 *>(p.E);
        for (int64_t b = e0 + lane; b < e1; b += 32 * kUnroll) {
            int2 uv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                uv[u] = b + 32 * u < e1 ? __ldcs(E + b + 32 * u) : make_int2(0, 0);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if ((uint64_t)(uint32_t)uv[u].x >= (uint64_t)p.n ||
                    (uint64_t)(uint32_t)uv[u].y >= (uint64_t)p.n)
                    report(p.st, GEE_ERR_NODE_RANGE,
                           (unsigned long long)(b + 32 * u));
        }
    }
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_zero(BatchHeader *h, const BatchProblem *P)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int64_t c = next_chunk(h, kWorkZero);
        if (c >= h->cell_chunks)
            break;
        const BatchProblem &p = P[find_problem(P, (int)h->count, kChunkCells, c)];
        if (failed(p.st))
            continue;
        const int64_t cells = p.n * p.K;
        const int64_t j0 = (c - p.cell_chunk0) * kBatchCellChunk;
        const int64_t j1 = min(j0 + kBatchCellChunk, cells);
        for (int64_t j = j0 + lane; j < j1; j += 32)
            p.Z[j] = 0.0f;
    }
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_scatter(BatchHeader *h, const BatchProblem *P)
{
    const int lane = threadIdx.x & 31;
    const uint64_t keep = policy_evict_last();
    for (;;) {
        const int64_t c = next_chunk(h, kWorkScatter);
        if (c >= h->edge_chunks)
            break;
        const BatchProblem &p = P[find_problem(P, (int)h->count, kChunkEdges, c)];
        if (failed(p.st))
            continue;
        const int64_t e0 = (c - p.edge_chunk0) * kBatchEdgeChunk;
        const int64_t e1 = min(e0 + kBatchEdgeChunk, p.s);
        const int2 *E = reinterpret_cast<const int2 *>(p.E);
        uint32_t *C = reinterpret_cast<uint32_t *>(p.Z);
        const int64_t K = p.K;
        // kUnroll edges per lane in flight: their pairs and weights, then
        // their labels, then the adds
        for (int64_t b = e0 + lane; b < e1; b += 32 * kUnroll) {
            int2 uv[kUnroll];
            float wt[kUnroll];
            bool ok[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t e = b + 32 * u;
                uv[u] = e < e1 ? __ldcs(E + e) : make_int2(0, 0);
                wt[u] = (e < e1 && p.w != nullptr) ? __ldcs(p.w + e) : 1.0f;
                ok[u] = e < e1;
            }
            uint32_t yu[kUnroll], yv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (ok[u] && ((uint64_t)(uint32_t)uv[u].x >= (uint64_t)p.n ||
                              (uint64_t)(uint32_t)uv[u].y >= (uint64_t)p.n)) {
                    report(p.st, GEE_ERR_NODE_RANGE,
                           (unsigned long long)(b + 32 * u));
                    ok[u] = false;
                }
                yu[u] = ok[u] ? load_label(p.Yc + uv[u].x, keep) : kNoLabel;
                yv[u] = ok[u] ? load_label(p.Yc + uv[u].y, keep) : kNoLabel;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (p.w == nullptr) {
                    if (yv[u] != kNoLabel)
                        atomicAdd(C + uv[u].x * K + yv[u], 1u);
                    if (yu[u] != kNoLabel)
                        atomicAdd(C + uv[u].y * K + yu[u], 1u);
                } else {
                    if (yv[u] != kNoLabel)
                        atomicAdd(p.Z + uv[u].x * K + yv[u], wt[u]);
                    if (yu[u] != kNoLabel)
                        atomicAdd(p.Z + uv[u].y * K + yu[u], wt[u]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kBatchThreads)
    k_batch_finalize(BatchHeader *h, const BatchProblem *P)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int64_t c = next_chunk(h, kWorkFinalize);
        if (c >= h->cell_chunks)
            break;
        const BatchProblem &p = P[find_problem(P, (int)h->count, kChunkCells, c)];
        if (failed(p.st))
            continue;
        const int64_t cells = p.n * p.K;
        const int64_t j0 = (c - p.cell_chunk0) * kBatchCellChunk;
        const int64_t j1 = min(j0 + kBatchCellChunk, cells);
        const int K = p.K;
        uint32_t *C = reinterpret_cast<uint32_t *>(p.Z);
        auto value = [&](uint32_t x, int k) {
            return p.w == nullptr ? count_to_z(x, p.counts[k])
                                  : sum_to_z(__uint_as_float(x), p.counts[k]);
        };
        // 16-byte loads and stores between a scalar head (up to the first
        // 16-byte boundary of Z) and tail: kUnroll quads per lane in flight
        const int64_t head =
            min((int64_t)(((16u - (reinterpret_cast<uintptr_t>(p.Z + j0) & 15u)) &
                           15u) >> 2),
                j1 - j0);
        const int64_t jb = j0 + head;
        const int64_t nq = (j1 - jb) >> 2;
        const int64_t jt = jb + 4 * nq;
        if (lane < head)
            p.Z[j0 + lane] = value(C[j0 + lane], (int)((j0 + lane) % K));
        if (lane < j1 - jt)
            p.Z[jt + lane] = value(C[jt + lane], (int)((jt + lane) % K));
        const uint4 *C4 = reinterpret_cast<const uint4 *>(C + jb);
        float4 *Z4 = reinterpret_cast<float4 *>(p.Z + jb);
        // class of this lane's quad's first cell, advanced by 128 cells per
        // step
        int k = (int)((jb + 4 * (int64_t)lane) % K);
        const int dk = 128 % K;
        for (int64_t q = lane; q < nq; q += 32 * kUnroll) {
            uint4 x[kUnroll];
            int kk[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                x[u] = q + 32 * u < nq ? C4[q + 32 * u] : make_uint4(0u, 0u, 0u, 0u);
                kk[u] = k;
                k += dk;
                if (k >= K)
                    k -= K;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (q + 32 * u >= nq)
                    continue;
                const uint32_t xs[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
                float o[4];
                int ke = kk[u];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    o[e] = value(xs[e], ke);
                    if (++ke == K)
                        ke = 0;
                }
                Z4[q + 32 * u] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

}  // namespace

int64_t batch_layout(BatchProblem *P, int count, BatchHeader &h)
{
    int64_t nodes = 0, edges = 0, cells = 0, counts = 0, yc = 0;
    for (int i = 0; i < count; ++i) {
        BatchProblem &p = P[i];
        p.node_chunk0 = nodes;
        p.edge_chunk0 = edges;
        p.cell_chunk0 = cells;
        nodes += (p.n + kBatchNodeChunk - 1) / kBatchNodeChunk;
        edges += (p.s + kBatchEdgeChunk - 1) / kBatchEdgeChunk;
        cells += (p.n * p.K + kBatchCellChunk - 1) / kBatchCellChunk;
        p.counts_off = counts;
        p.yc_off = yc;
        counts += p.K;
        yc += (p.n + 15) & ~int64_t(15);
    }
    h.count = count;
    h.node_chunks = nodes;
    h.edge_chunks = edges;
    h.cell_chunks = cells;
    h.count_cells = counts;
    h.yc_bytes = yc;
    return yc;
}

cudaError_t batch_enqueue(BatchHeader *dh, const BatchProblem *dP,
                          const BatchHeader &hh, bool validate,
                          cudaStream_t stream)
{
    (void)hh;
    const int sms = sm_count();
    {
        // a fixed grid (grid-stride loops) so the sequence's launch
        // parameters do not depend on the batch
        ProfScope p("k_batch_init", stream);
        k_batch_init<<<sms * 4, 256, 0, stream>>>(dh, dP);
    }
    // two CTAs of 512 threads per SM, persistent
    const int blocks = 2 * sms;
    {
        ProfScope p("k_batch_labels", stream);
        k_batch_labels<<<blocks, kBatchThreads, 0, stream>>>(dh, dP);
    }
    if (validate) {
        ProfScope p("k_batch_validate", stream);
        k_batch_validate<<<blocks, kBatchThreads, 0, stream>>>(dh, dP);
    }
    {
        ProfScope p("k_batch_zero", stream);
        k_batch_zero<<<blocks, kBatchThreads, 0, stream>>>(dh, dP);
    }
    {
        ProfScope p("k_batch_scatter", stream);
        k_batch_scatter<<<blocks, kBatchThreads, 0, stream>>>(dh, dP);
    }
    {
        ProfScope p("k_batch_finalize", stream);
        k_batch_finalize<<<blocks, kBatchThreads, 0, stream>>>(dh, dP);
    }
    return cudaGetLastError();
}

cudaError_t batch_labels_enqueue(BatchHeader *dh, const BatchProblem *dP,
                                 cudaStream_t stream)
{
    const int sms = sm_count();
    {
        ProfScope p("k_batch_init", stream);
        k_batch_init<<<sms * 4, 256, 0, stream>>>(dh, dP);
    }
    {
        ProfScope p("k_batch_labels", stream);
        k_batch_labels<<<2 * sms, kBatchThreads, 0, stream>>>(dh, dP);
    }
    return cudaGetLastError();
}

cudaError_t batch_graph_create(BatchHeader *dh, const BatchProblem *dP,
                               bool validate, cudaStream_t stream,
                               cudaGraphExec_t *exec)
{
    *exec = nullptr;
    sm_count();  // cached before the capture
    cudaError_t e =
        cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return e;
    BatchHeader unused{};
    cudaError_t el = batch_enqueue(dh, dP, unused, validate, stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(stream, &graph);
    if (el != cudaSuccess)
        e = el;
    if (e == cudaSuccess)
        e = cudaGraphInstantiate(exec, graph, 0);
    if (graph != nullptr)
        cudaGraphDestroy(graph);
    return e;
}

}  // namespace gee
