// gee_coo.cu -- label pass and edge-list (COO) passes of GEE on sm_103a.
//
//   k_labels         S1 + S2: label check, compact uint8 labels, n_k
//   k_degree/rsqrt   S3 for the Laplacian variant (edge-list form)
//   k_scatter_*      S4: both updates of Alg. 1's loop body per edge, as
//                    red.global atomics (ATOMIC) or into a per-CTA copy of Z
//                    in shared memory (PRIVATE)
//   k_finalize_*     S5: Z = C / n_k (count path) or acc / n_k (weighted)
//
// Edges are streamed two per 16-byte load when the edge array is 16-byte
// aligned; labels are gathered through L2 with an evict-last policy so the
// n-byte label array stays resident while edges stream past.
#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kLabelThreads = 256;

__global__ void k_status_init(DevStatus *st)
{
    st->code = 0;
    st->aux = 0;
    st->index = ~0ull;
}

// ---------------------------------------------------------------- S1 + S2
// Alg. 1 W initialisation: n_k = count(Y = k).  W itself is never stored:
// W(i, Y(i)) = 1 / n_{Y(i)} is applied once per Z cell at the end.
__global__ void __launch_bounds__(kLabelThreads)
    k_labels(const int32_t *__restrict__ Y, int64_t n, int32_t K,
             const int32_t *__restrict__ rank, uint8_t *__restrict__ Yc,
             uint32_t *__restrict__ counts, DevStatus *st)
{
    __shared__ uint32_t hist[kMaxClasses];
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        hist[k] = 0;
    __syncthreads();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    auto one = [&](int32_t y, int64_t i) -> uint32_t {
        if (y == -1)
            return kNoLabel;
        if ((uint32_t)y < (uint32_t)K) {
            atomicAdd(&hist[y], 1u);
            return (uint32_t)y;
        }
        report(st, GEE_ERR_LABEL_RANGE, (unsigned long long)i);
        return kNoLabel;
    };
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(Y) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(Yc) & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(rank) & 15) == 0) {
        const int64_t n4 = n >> 2;
        const int4 *Y4 = reinterpret_cast<const int4 *>(Y);
        for (int64_t i = tid; i < n4; i += nthreads) {
            const int4 y = __ldcs(Y4 + i);
            const uint32_t a = one(y.x, 4 * i), b = one(y.y, 4 * i + 1);
            const uint32_t c = one(y.z, 4 * i + 2), d = one(y.w, 4 * i + 3);
            if (rank == nullptr) {
                reinterpret_cast<uint32_t *>(Yc)[i] =
                    a | (b << 8) | (c << 16) | (d << 24);
            } else {
                const int4 r = __ldcs(reinterpret_cast<const int4 *>(rank) + i);
                Yc[r.x] = (uint8_t)a;
                Yc[r.y] = (uint8_t)b;
                Yc[r.z] = (uint8_t)c;
                Yc[r.w] = (uint8_t)d;
            }
        }
        head = n4 << 2;
    }
    for (int64_t i = head + tid; i < n; i += nthreads) {
        const uint8_t code = (uint8_t)one(__ldcs(Y + i), i);
        Yc[rank == nullptr ? i : (int64_t)rank[i]] = code;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (hist[k] != 0u)
            atomicAdd(&counts[k], hist[k]);
}

// L label vectors at once (Y[l*n + i]): the compact label of node i for
// vector l goes to Yc[rank[i]*Ls + l] (Ls = label_stride(L); padding bytes
// get 255), so one gather of adjacent bytes serves all vectors;
// counts[l*K + k] = n_k of vector l.  One thread per node reads its L
// labels (coalesced across the warp for each l) and writes its record with
// whole-word stores: 4, 8 or 16 bytes at a time.
__global__ void k_labels_multi(const int32_t *__restrict__ Y, int64_t n,
                               int32_t L, int32_t Ls, int32_t K,
                               const int32_t *__restrict__ rank,
                               uint8_t *__restrict__ Yc,
                               uint32_t *__restrict__ counts, DevStatus *st)
{
    __shared__ uint32_t hist[GEE_MAX_COLUMNS];
    for (int k = threadIdx.x; k < L * K; k += blockDim.x)
        hist[k] = 0;
    __syncthreads();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    // codes of labels l0 .. l0+15 of node i (255 beyond L) packed in four
    // words; all loads are issued before the histogram updates
    auto codes16 = [&](int l0, int64_t i, uint32_t (&word)[4]) {
        int32_t y[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
            y[e] = l0 + e < L ? __ldcs(Y + (int64_t)(l0 + e) * n + i) : -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            word[q] = 0u;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            uint32_t code = kNoLabel;
            if ((uint32_t)y[e] < (uint32_t)K) {
                atomicAdd(&hist[(l0 + e) * K + y[e]], 1u);
                code = (uint32_t)y[e];
            } else if (y[e] != -1) {
                report(st, GEE_ERR_LABEL_RANGE,
                       (unsigned long long)((l0 + e) * n + i));
            }
            word[e >> 2] |= code << (8 * (e & 3));
        }
    };
    for (int64_t i = tid; i < n; i += nthreads) {
        const int64_t r = rank == nullptr ? i : (int64_t)rank[i];
        uint8_t *rec = Yc + r * Ls;
        uint32_t word[4];
        if (Ls <= 8) {
            codes16(0, i, word);
            *reinterpret_cast<uint32_t *>(rec) = word[0];
            if (Ls == 8)
                *reinterpret_cast<uint32_t *>(rec + 4) = word[1];
        } else {
            for (int c = 0; c < Ls; c += 16) {
                codes16(c, i, word);
                *reinterpret_cast<uint4 *>(rec + c) =
                    make_uint4(word[0], word[1], word[2], word[3]);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < L * K; k += blockDim.x)
        if (hist[k] != 0u)
            atomicAdd(&counts[k], hist[k]);
}

// Calls f(u, v, edge_index) for every edge; two edges per 16-byte load when
// E is 16-byte aligned.
template <class F>
__device__ __forceinline__ void for_each_edge(const int32_t *__restrict__ E,
                                              int64_t s, int64_t tid,
                                              int64_t nthreads, F &&f)
{
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(E) & 15) == 0) {
        const int64_t s2 = s >> 1;
        const int4 *E4 = reinterpret_cast<const int4 *>(E);
        for (int64_t i = tid; i < s2; i += nthreads) {
            const int4 e = __ldcs(E4 + i);
            f(e.x, e.y, 2 * i);
            f(e.z, e.w, 2 * i + 1);
        }
        head = s2 << 1;
    }
    for (int64_t i = head + tid; i < s; i += nthreads) {
        const int2 e = __ldcs(reinterpret_cast<const int2 *>(E) + i);
        f(e.x, e.y, i);
    }
}

__device__ __forceinline__ bool node_ok(int32_t x, int64_t n)
{
    return (int64_t)(uint32_t)x < n;
}

__global__ void __launch_bounds__(256)
    k_validate_edges(const int32_t *__restrict__ E, int64_t s, int64_t n,
                     DevStatus *st)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for_each_edge(E, s, tid, nthreads, [&](int32_t u, int32_t v, int64_t i) {
        if (!node_ok(u, n) || !node_ok(v, n))
            report(st, GEE_ERR_NODE_RANGE, (unsigned long long)i);
    });
}

// ---------------------------------------------------------------- S3
// Laplacian reading: d_u = sum of the weights of u's edges (self-loop twice),
// accumulated in FP64 (L2 double atomics) so hub degrees keep full precision.
__global__ void __launch_bounds__(256)
    k_degree(const int32_t *__restrict__ E, const float *__restrict__ w,
             int64_t s, int64_t n, double *__restrict__ d, DevStatus *st)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for_each_edge(E, s, tid, nthreads, [&](int32_t u, int32_t v, int64_t i) {
        if (!node_ok(u, n) || !node_ok(v, n)) {
            report(st, GEE_ERR_NODE_RANGE, (unsigned long long)i);
            return;
        }
        float wt = 1.0f;
        if (w != nullptr) {
            wt = __ldcs(w + i);
            if (!(wt >= 0.0f)) {
                report(st, GEE_ERR_INVALID_ARG, (unsigned long long)i);
                return;
            }
        }
        atomicAdd(d + u, (double)wt);
        atomicAdd(d + v, (double)wt);
    });
}

__global__ void k_rsqrt(const double *__restrict__ d, int64_t n,
                        float *__restrict__ r, const DevStatus *st)
{
    if (failed(st))
        return;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads) {
        const double x = d[i];
        r[i] = rsqrt_rn32(x);
    }
}

__global__ void k_zero(uint32_t *__restrict__ p, int64_t words,
                       const DevStatus *st)
{
    if (failed(st))
        return;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const int64_t w4 = words >> 2;
        uint4 *p4 = reinterpret_cast<uint4 *>(p);
        for (int64_t i = tid; i < w4; i += nthreads)
            p4[i] = make_uint4(0u, 0u, 0u, 0u);
        head = w4 << 2;
    }
    for (int64_t i = head + tid; i < words; i += nthreads)
        p[i] = 0u;
}

// ---------------------------------------------------------------- S4 ATOMIC
// Alg. 1 loop body, as red.global.add: count path (unit weights) adds 1 to
// the uint32 count; weighted path adds w (Laplacian: w * r of the sender).
template <bool WEIGHTED, bool LAP, bool CHECK>
__global__ void __launch_bounds__(256)
    k_scatter_atomic(const int32_t *__restrict__ E,
                     const float *__restrict__ w, const float *__restrict__ r,
                     int64_t s, int64_t n, int32_t K,
                     const uint8_t *__restrict__ Yc, void *__restrict__ Zv,
                     DevStatus *st)
{
    if (failed(st))
        return;
    const uint64_t keep = policy_evict_last();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    uint32_t *C = static_cast<uint32_t *>(Zv);
    float *Z = static_cast<float *>(Zv);
    for_each_edge(E, s, tid, nthreads, [&](int32_t u, int32_t v, int64_t i) {
        if (CHECK && (!node_ok(u, n) || !node_ok(v, n))) {
            report(st, GEE_ERR_NODE_RANGE, (unsigned long long)i);
            return;
        }
        const uint32_t yu = load_label(Yc + u, keep);
        const uint32_t yv = load_label(Yc + v, keep);
        if (!WEIGHTED) {
            if (yv != kNoLabel)
                atomicAdd(C + (int64_t)u * K + yv, 1u);
            if (yu != kNoLabel)
                atomicAdd(C + (int64_t)v * K + yu, 1u);
        } else {
            const float wt = (w != nullptr) ? __ldcs(w + i) : 1.0f;
            if (yv != kNoLabel)
                atomicAdd(Z + (int64_t)u * K + yv, LAP ? wt * r[v] : wt);
            if (yu != kNoLabel)
                atomicAdd(Z + (int64_t)v * K + yu, LAP ? wt * r[u] : wt);
        }
    });
}

// ---------------------------------------------------------------- S4 PRIVATE
// Small n*K: each CTA accumulates a private copy of Z in shared memory (no
// global atomics per edge), then adds its non-zero cells to global Z.
template <bool WEIGHTED, bool LAP, bool CHECK>
__global__ void k_scatter_private(const int32_t *__restrict__ E,
                                  const float *__restrict__ w,
                                  const float *__restrict__ r, int64_t s,
                                  int64_t n, int32_t K,
                                  const uint8_t *__restrict__ Yc,
                                  void *__restrict__ Zv, DevStatus *st)
{
    extern __shared__ uint32_t zs[];
    if (failed(st))
        return;
    const int cells = (int)(n * K);
    for (int c = threadIdx.x; c < cells; c += blockDim.x)
        zs[c] = 0u;
    __syncthreads();
    float *zf = reinterpret_cast<float *>(zs);
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for_each_edge(E, s, tid, nthreads, [&](int32_t u, int32_t v, int64_t i) {
        if (CHECK && (!node_ok(u, n) || !node_ok(v, n))) {
            report(st, GEE_ERR_NODE_RANGE, (unsigned long long)i);
            return;
        }
        const uint32_t yu = __ldg(Yc + u), yv = __ldg(Yc + v);
        if (!WEIGHTED) {
            if (yv != kNoLabel)
                atomicAdd(zs + u * K + yv, 1u);
            if (yu != kNoLabel)
                atomicAdd(zs + v * K + yu, 1u);
        } else {
            const float wt = (w != nullptr) ? __ldcs(w + i) : 1.0f;
            if (yv != kNoLabel)
                atomicAdd(zf + u * K + yv, LAP ? wt * r[v] : wt);
            if (yu != kNoLabel)
                atomicAdd(zf + v * K + yu, LAP ? wt * r[u] : wt);
        }
    });
    __syncthreads();
    uint32_t *C = static_cast<uint32_t *>(Zv);
    float *Z = static_cast<float *>(Zv);
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
        if (zs[c] == 0u)
            continue;
        if (!WEIGHTED)
            atomicAdd(C + c, zs[c]);
        else
            atomicAdd(Z + c, zf[c]);
    }
}

// ---------------------------------------------------------------- S5
// Walks cells i = 4j..4j+3 with a running (row, class) position, so no
// division by K happens per cell.
struct CellCursor {
    int64_t row;
    int32_t k;
    __device__ CellCursor(int64_t cell, int32_t K)
        : row(cell / K), k((int32_t)(cell - (cell / K) * K)) {}
    __device__ void advance(int64_t step_rows, int32_t step_k, int32_t K)
    {
        row += step_rows;
        k += step_k;
        if (k >= K) {
            k -= K;
            ++row;
        }
    }
};

template <bool WEIGHTED, bool LAP>
__global__ void __launch_bounds__(256)
    k_finalize(void *__restrict__ Zv, const float *__restrict__ r, int64_t n,
               int32_t K, const uint32_t *__restrict__ counts,
               const DevStatus *st)
{
    __shared__ uint32_t nk[kMaxClasses];
    if (failed(st))
        return;
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        nk[k] = counts[k];
    __syncthreads();
    const int64_t cells = n * K;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    uint32_t *C = static_cast<uint32_t *>(Zv);
    float *Z = static_cast<float *>(Zv);
    auto cell = [&](uint32_t bits, int64_t row, int32_t k) -> float {
        if (!WEIGHTED)
            return count_to_z(bits, nk[k]);
        float z = sum_to_z(__uint_as_float(bits), nk[k]);
        if (LAP)
            z = z * r[row];
        return z;
    };
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(Zv) & 15) == 0) {
        const int64_t c4 = cells >> 2;
        const int64_t step = 4 * nthreads;
        CellCursor cur(4 * tid, K);
        const int64_t srow = step / K;
        const int32_t sk = (int32_t)(step - srow * K);
        uint4 *C4 = reinterpret_cast<uint4 *>(C);
        float4 *Z4 = reinterpret_cast<float4 *>(Z);
        for (int64_t j = tid; j < c4; j += nthreads) {
            const uint4 c = C4[j];
            float out[4];
            const uint32_t in[4] = {c.x, c.y, c.z, c.w};
            int64_t row = cur.row;
            int32_t k = cur.k;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                out[e] = cell(in[e], row, k);
                if (++k == K) {
                    k = 0;
                    ++row;
                }
            }
            __stcs(Z4 + j, make_float4(out[0], out[1], out[2], out[3]));
            cur.advance(srow, sk, K);
        }
        head = c4 << 2;
    }
    for (int64_t i = head + tid; i < cells; i += nthreads) {
        const int64_t row = i / K;
        Z[i] = cell(C[i], row, (int32_t)(i - row * K));
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_status_init(DevStatus *st, cudaStream_t stream)
{
    k_status_init<<<1, 1, 0, stream>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_labels(const int32_t *Y, int64_t n, int32_t K,
                          const int32_t *rank, uint8_t *Yc, uint32_t *counts,
                          DevStatus *st, cudaStream_t stream)
{
    if (n == 0)
        return cudaSuccess;
    const int blocks = grid_for((n + 3) / 4, kLabelThreads, sm_count() * 8);
    k_labels<<<blocks, kLabelThreads, 0, stream>>>(Y, n, K, rank, Yc, counts,
                                                   st);
    return cudaGetLastError();
}

cudaError_t launch_labels_multi(const int32_t *Y, int64_t n, int32_t L,
                                int32_t K, const int32_t *rank, uint8_t *Yc,
                                uint32_t *counts, DevStatus *st,
                                cudaStream_t stream)
{
    if (n == 0)
        return cudaSuccess;
    const int blocks = grid_for(n, kLabelThreads, sm_count() * 8);
    k_labels_multi<<<blocks, kLabelThreads, 0, stream>>>(
        Y, n, L, label_stride(L), K, rank, Yc, counts, st);
    return cudaGetLastError();
}

cudaError_t launch_validate_edges(const int32_t *E, int64_t s, int64_t n,
                                  DevStatus *st, cudaStream_t stream)
{
    if (s == 0)
        return cudaSuccess;
    const int blocks = grid_for((s + 1) / 2, 256, sm_count() * 8);
    k_validate_edges<<<blocks, 256, 0, stream>>>(E, s, n, st);
    return cudaGetLastError();
}

cudaError_t launch_degree(const int32_t *E, const float *w, int64_t s,
                          int64_t n, double *d, DevStatus *st,
                          cudaStream_t stream)
{
    if (s == 0)
        return cudaSuccess;
    const int blocks = grid_for((s + 1) / 2, 256, sm_count() * 8);
    k_degree<<<blocks, 256, 0, stream>>>(E, w, s, n, d, st);
    return cudaGetLastError();
}

cudaError_t launch_rsqrt(const double *d, int64_t n, float *r,
                         const DevStatus *st, cudaStream_t stream)
{
    if (n == 0)
        return cudaSuccess;
    k_rsqrt<<<grid_for(n, 256, sm_count() * 8), 256, 0, stream>>>(d, n, r, st);
    return cudaGetLastError();
}

cudaError_t launch_zero(void *p, int64_t words, const DevStatus *st,
                        cudaStream_t stream)
{
    if (words == 0)
        return cudaSuccess;
    k_zero<<<grid_for((words + 3) / 4, 256, sm_count() * 8), 256, 0,
             stream>>>(static_cast<uint32_t *>(p), words, st);
    return cudaGetLastError();
}

template <bool W, bool L, bool C>
static void scatter_atomic_t(int blocks, int threads, cudaStream_t stream,
                             const int32_t *E, const float *w, const float *r,
                             int64_t s, int64_t n, int32_t K,
                             const uint8_t *Yc, void *Z, DevStatus *st)
{
    k_scatter_atomic<W, L, C>
        <<<blocks, threads, 0, stream>>>(E, w, r, s, n, K, Yc, Z, st);
}

cudaError_t launch_scatter_atomic(const int32_t *E, const float *w,
                                  const float *r, int64_t s, int64_t n,
                                  int32_t K, const uint8_t *Yc, void *Z,
                                  bool check, int threads, DevStatus *st,
                                  cudaStream_t stream)
{
    if (s == 0)
        return cudaSuccess;
    const int blocks = grid_for((s + 1) / 2, threads, sm_count() * 8);
    const bool weighted = (w != nullptr) || (r != nullptr);
    const bool lap = (r != nullptr);
    if (!weighted) {
        if (check)
            scatter_atomic_t<false, false, true>(blocks, threads, stream, E, w,
                                                 r, s, n, K, Yc, Z, st);
        else
            scatter_atomic_t<false, false, false>(blocks, threads, stream, E,
                                                  w, r, s, n, K, Yc, Z, st);
    } else if (lap) {
        if (check)
            scatter_atomic_t<true, true, true>(blocks, threads, stream, E, w,
                                               r, s, n, K, Yc, Z, st);
        else
            scatter_atomic_t<true, true, false>(blocks, threads, stream, E, w,
                                                r, s, n, K, Yc, Z, st);
    } else {
        if (check)
            scatter_atomic_t<true, false, true>(blocks, threads, stream, E, w,
                                                r, s, n, K, Yc, Z, st);
        else
            scatter_atomic_t<true, false, false>(blocks, threads, stream, E, w,
                                                 r, s, n, K, Yc, Z, st);
    }
    return cudaGetLastError();
}

int64_t private_cells_limit()
{
    // 227 KB of opt-in shared memory per CTA, minus a little headroom.
    return (int64_t)(220 * 1024) / 4;
}

template <bool W, bool L, bool C>
static cudaError_t scatter_private_t(int blocks, int threads, size_t smem,
                                     cudaStream_t stream, const int32_t *E,
                                     const float *w, const float *r,
                                     int64_t s, int64_t n, int32_t K,
                                     const uint8_t *Yc, void *Z, DevStatus *st)
{
    cudaError_t e = cudaFuncSetAttribute(
        k_scatter_private<W, L, C>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_scatter_private<W, L, C>
        <<<blocks, threads, smem, stream>>>(E, w, r, s, n, K, Yc, Z, st);
    return cudaGetLastError();
}

cudaError_t launch_scatter_private(const int32_t *E, const float *w,
                                   const float *r, int64_t s, int64_t n,
                                   int32_t K, const uint8_t *Yc, void *Z,
                                   bool check, int threads, DevStatus *st,
                                   cudaStream_t stream)
{
    if (s == 0)
        return cudaSuccess;
    const size_t smem = (size_t)(n * K) * 4;
    // one CTA per SM when the copy is large, more when it is small
    int per_sm = (int)((220 * 1024) / (smem > 0 ? smem : 1));
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    // enough edges per CTA that zeroing and merging the copy pays off
    int64_t max_blocks = (s * 2) / (8 * (n * K) + 1) + 1;
    int64_t limit = (int64_t)sm_count() * per_sm;
    int blocks = (int)(max_blocks < limit ? max_blocks : limit);
    const bool weighted = (w != nullptr) || (r != nullptr);
    const bool lap = (r != nullptr);
    if (!weighted)
        return check ? scatter_private_t<false, false, true>(
                           blocks, threads, smem, stream, E, w, r, s, n, K, Yc,
                           Z, st)
                     : scatter_private_t<false, false, false>(
                           blocks, threads, smem, stream, E, w, r, s, n, K, Yc,
                           Z, st);
    if (lap)
        return check ? scatter_private_t<true, true, true>(
                           blocks, threads, smem, stream, E, w, r, s, n, K, Yc,
                           Z, st)
                     : scatter_private_t<true, true, false>(
                           blocks, threads, smem, stream, E, w, r, s, n, K, Yc,
                           Z, st);
    return check ? scatter_private_t<true, false, true>(
                       blocks, threads, smem, stream, E, w, r, s, n, K, Yc, Z,
                       st)
                 : scatter_private_t<true, false, false>(
                       blocks, threads, smem, stream, E, w, r, s, n, K, Yc, Z,
                       st);
}

cudaError_t launch_finalize_count(void *Z, int64_t n, int32_t K,
                                  const uint32_t *counts, const DevStatus *st,
                                  cudaStream_t stream)
{
    const int64_t cells = n * K;
    if (cells == 0)
        return cudaSuccess;
    k_finalize<false, false><<<grid_for((cells + 3) / 4, 256, sm_count() * 8),
                               256, 0, stream>>>(Z, nullptr, n, K, counts, st);
    return cudaGetLastError();
}

cudaError_t launch_finalize_weighted(float *Z, const float *r, int64_t n,
                                     int32_t K, const uint32_t *counts,
                                     const DevStatus *st, cudaStream_t stream)
{
    const int64_t cells = n * K;
    if (cells == 0)
        return cudaSuccess;
    const int blocks = grid_for((cells + 3) / 4, 256, sm_count() * 8);
    if (r != nullptr)
        k_finalize<true, true><<<blocks, 256, 0, stream>>>(Z, r, n, K, counts,
                                                           st);
    else
        k_finalize<true, false><<<blocks, 256, 0, stream>>>(Z, r, n, K, counts,
                                                            st);
    return cudaGetLastError();
}

}  // namespace gee
