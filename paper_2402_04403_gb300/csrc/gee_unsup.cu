// gee_unsup.cu -- unsupervised GEE on a resident graph (gee_unsupervised).
//
// Section II allows the label vector to come from unsupervised clustering
// instead of known labels.  Here the clustering is k-means on the
// embedding (Lloyd's assignment step), alternated with the unit-weight
// pass: every round embeds the current labels (S1-S5 on the resident
// graph) and moves each node to the nearest class mean of that embedding,
// until a round moves nothing.  The arithmetic is fixed so that every run
// takes the same decisions (the paper fixes no precision for this step; an
// exact evaluation can differ only on near-ties, by the FP32 bound the
// header states):
//   Z[i,j]  = RN32(C[i,j] / m_j), the pass's bit-exact count-path output
//   C[i,j]  = the exact neighbour count, recovered from Z as rint(Z * m_j)
//             in FP64 (exact while C < 2^23)
//   S[k,j]  = sum of C[i,j] over the nodes of class k (uint64, exact)
//   c[k,j]  = RN32(S[k,j] / (m_k * m_j)), the quotient formed in FP64
//   d(i,k)  = sum over j = 0..K-1 in order of (Z[i,j] - c[k,j])^2 in FP32,
//             every operation rounded on its own (no contraction)
//   node i -> the k with the smallest d among non-empty classes, lowest k
//   on ties.
// Kernels: k_unsup_hist (class sizes), k_unsup_sums (class sums in shared
// memory, flushed with 64-bit atomics), k_unsup_centroids, k_unsup_assign
// (one warp per node, one lane per class).
#include "gee_internal.cuh"

namespace gee {

namespace {

constexpr int kUnsupMaxK = 64;
constexpr int kThreads = 256;

__device__ __forceinline__ double exact_count(float z, uint64_t m)
{
    return rint(__dmul_rn((double)z, (double)m));
}

__global__ void k_unsup_hist(const int32_t *__restrict__ Y, int64_t n,
                             int32_t K, unsigned long long *m, DevStatus *st)
{
    __shared__ unsigned int h[kUnsupMaxK];
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        h[k] = 0u;
    __syncthreads();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nth) {
        const int32_t y = Y[i];
        if ((uint32_t)y < (uint32_t)K)
            atomicAdd(&h[y], 1u);
        else
            report(st, GEE_ERR_LABEL_RANGE, (unsigned long long)i);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (h[k] != 0u)
            atomicAdd(m + k, (unsigned long long)h[k]);
}

__global__ void k_unsup_sums(const int32_t *__restrict__ Y,
                             const float *__restrict__ Z, int64_t n, int32_t K,
                             const unsigned long long *__restrict__ m,
                             unsigned long long *S, const DevStatus *st)
{
    __shared__ unsigned long long s[kUnsupMaxK * kUnsupMaxK];
    __shared__ unsigned long long ms[kUnsupMaxK];
    if (failed(st))
        return;
    for (int c = threadIdx.x; c < K * K; c += blockDim.x)
        s[c] = 0ull;
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        ms[k] = m[k];
    __syncthreads();
    // thread t takes cell j = t % K of rows t / K, t / K + rows_per_step, ...
    const int rows_per_block = blockDim.x / K;
    const int j = threadIdx.x % K;
    const int r = threadIdx.x / K;
    if (r < rows_per_block) {
        for (int64_t i = (int64_t)blockIdx.x * rows_per_block + r; i < n;
             i += (int64_t)gridDim.x * rows_per_block) {
            const double c = exact_count(Z[i * K + j], ms[j]);
            if (c != 0.0)
                atomicAdd(&s[Y[i] * K + j], (unsigned long long)c);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < K * K; c += blockDim.x)
        if (s[c] != 0ull)
            atomicAdd(S + c, s[c]);
}

// cenT[j*K + k] = c[k, j] (transposed for the assignment's lane-per-class
// reads); 0 where a class is empty.
__global__ void k_unsup_centroids(const unsigned long long *__restrict__ S,
                                  const unsigned long long *__restrict__ m,
                                  int32_t K, float *cenT)
{
    for (int c = threadIdx.x; c < K * K; c += blockDim.x) {
        const int k = c / K, j = c - k * K;
        const double den = __dmul_rn((double)m[k], (double)m[j]);
        cenT[j * K + k] =
            den > 0.0 ? __double2float_rn(__ddiv_rn((double)S[c], den)) : 0.0f;
    }
}

__global__ void k_unsup_assign(const float *__restrict__ Z, int64_t n,
                               int32_t K,
                               const unsigned long long *__restrict__ m,
                               const float *__restrict__ cenT,
                               const int32_t *__restrict__ Y, int32_t *Ynext,
                               unsigned long long *moved, const DevStatus *st)
{
    __shared__ float cs[kUnsupMaxK * kUnsupMaxK];
    __shared__ unsigned long long ms[kUnsupMaxK];
    __shared__ unsigned long long block_moved;
    if (failed(st))
        return;
    for (int c = threadIdx.x; c < K * K; c += blockDim.x)
        cs[c] = cenT[c];
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        ms[k] = m[k];
    if (threadIdx.x == 0)
        block_moved = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int ka = lane, kb = lane + 32;
    unsigned long long my_moved = 0ull;
    for (int64_t i = warp; i < n; i += nwarps) {
        // Z[i, j] for j = lane and lane + 32, handed round by shuffles
        const float za = ka < K ? Z[i * K + ka] : 0.0f;
        const float zb = kb < K ? Z[i * K + kb] : 0.0f;
        float da = 0.0f, db = 0.0f;
        for (int j = 0; j < K; ++j) {
            const float zj = __shfl_sync(0xffffffffu, j < 32 ? za : zb, j & 31);
            if (ka < K) {
                const float d = __fsub_rn(zj, cs[j * K + ka]);
                da = __fadd_rn(da, __fmul_rn(d, d));
            }
            if (kb < K) {
                const float d = __fsub_rn(zj, cs[j * K + kb]);
                db = __fadd_rn(db, __fmul_rn(d, d));
            }
        }
        // this lane's best non-empty class, then the warp's (lowest k on ties)
        int bk = -1;
        float bd = 0.0f;
        if (ka < K && ms[ka] != 0ull) {
            bk = ka;
            bd = da;
        }
        if (kb < K && ms[kb] != 0ull && (bk < 0 || db < bd)) {
            bk = kb;
            bd = db;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const int ok = __shfl_down_sync(0xffffffffu, bk, off);
            const float od = __shfl_down_sync(0xffffffffu, bd, off);
            if (ok >= 0 && (bk < 0 || od < bd || (od == bd && ok < bk))) {
                bk = ok;
                bd = od;
            }
        }
        if (lane == 0) {
            const int32_t old = Y[i];
            Ynext[i] = bk;
            my_moved += (bk != old);
        }
    }
    if (lane == 0 && my_moved != 0ull)
        atomicAdd(&block_moved, my_moved);
    __syncthreads();
    if (threadIdx.x == 0 && block_moved != 0ull)
        atomicAdd(moved, block_moved);
}

}  // namespace

}  // namespace gee

using namespace gee;

extern "C" gee_status gee_unsupervised(gee_graph *graph, int32_t *Y, int32_t K,
                                       int32_t max_iter, float *Z,
                                       int32_t *rounds, int64_t *moved,
                                       gee_stream_t stream_)
{
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (graph == nullptr || rounds == nullptr || max_iter < 0 || K < 1)
        return GEE_ERR_INVALID_ARG;
    *rounds = 0;
    if (K > kUnsupMaxK)
        return GEE_ERR_UNSUPPORTED;
    int64_t n = 0, bytes = 0;
    gee_status rc = gee_graph_info(graph, &n, nullptr, nullptr, nullptr, &bytes);
    if (rc != GEE_OK)
        return rc;
    if (graph_weighted(graph))
        return GEE_ERR_UNSUPPORTED;
    // every count is at most its row's arcs; rint(Z * m_j) recovers counts
    // below 2^23 exactly (|Z m_j - C| <= C 2^-24 < 1/2), larger ones not
    if (graph_max_degree(graph) >= (1u << 23))
        return GEE_ERR_OVERFLOW;
    if (n > 0 && (Y == nullptr || Z == nullptr))
        return GEE_ERR_INVALID_ARG;
    if (((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(Z)) & 3) != 0)
        return GEE_ERR_INVALID_ARG;
    Workspace ws(stream);
    unsigned long long *m = nullptr, *S = nullptr, *mv = nullptr;
    float *cenT = nullptr;
    int32_t *Ynext = nullptr;
    DevStatus *st = nullptr;
    cudaError_t e = ws.alloc((void **)&m, sizeof(unsigned long long) * K);
    if (e == cudaSuccess)
        e = ws.alloc((void **)&S, sizeof(unsigned long long) * K * K);
    if (e == cudaSuccess)
        e = ws.alloc((void **)&mv, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = ws.alloc((void **)&cenT, sizeof(float) * K * K);
    if (e == cudaSuccess)
        e = ws.alloc((void **)&Ynext, sizeof(int32_t) * (n + 1));
    if (e == cudaSuccess)
        e = ws.alloc((void **)&st, sizeof(DevStatus));
    if (e != cudaSuccess)
        return from_cuda(e);
    const int sms = sm_count();
    const int nb = grid_for(n, kThreads, sms * 8);
    bool stale = true;  // Z not yet the embedding of the current Y
    for (int32_t r = 0; r < max_iter; ++r) {
        {
            Workspace pass(stream);
            DevStatus *pst = nullptr;
            rc = graph_pass_enqueue(pass, graph, Y, 1, K, 0, Z, &pst, stream);
            if (rc != GEE_OK)
                return rc;
            e = cudaMemcpyAsync(st, pst, sizeof(DevStatus),
                                cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess)
                return from_cuda(e);
        }
        if ((e = cudaMemsetAsync(m, 0, sizeof(unsigned long long) * K, stream)) !=
                cudaSuccess ||
            (e = cudaMemsetAsync(S, 0, sizeof(unsigned long long) * K * K,
                                 stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(mv, 0, sizeof(unsigned long long), stream)) !=
                cudaSuccess)
            return from_cuda(e);
        if (n > 0) {
            {
                ProfScope p("k_unsup_hist", stream);
                k_unsup_hist<<<nb, kThreads, 0, stream>>>(Y, n, K, m, st);
            }
            {
                ProfScope p("k_unsup_sums", stream);
                k_unsup_sums<<<nb, kThreads, 0, stream>>>(Y, Z, n, K, m, S, st);
            }
            {
                ProfScope p("k_unsup_centroids", stream);
                k_unsup_centroids<<<1, 1024, 0, stream>>>(S, m, K, cenT);
            }
            {
                ProfScope p("k_unsup_assign", stream);
                k_unsup_assign<<<grid_for(n * 32, kThreads, sms * 16), kThreads, 0,
                                 stream>>>(Z, n, K, m, cenT, Y, Ynext, mv, st);
            }
            if ((e = cudaGetLastError()) != cudaSuccess)
                return from_cuda(e);
        }
        DevStatus hs;
        unsigned long long hm = 0;
        if ((e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost,
                                 stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&hm, mv, sizeof(hm), cudaMemcpyDeviceToHost,
                                 stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(stream)) != cudaSuccess)
            return from_cuda(e);
        if (hs.code != GEE_OK)
            return static_cast<gee_status>(hs.code);
        if (moved != nullptr)
            moved[r] = (int64_t)hm;
        *rounds = r + 1;
        if (hm == 0ull) {
            stale = false;
            break;
        }
        if ((e = cudaMemcpyAsync(Y, Ynext, sizeof(int32_t) * n,
                                 cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
            return from_cuda(e);
    }
    if (stale) {
        // max_iter ended the loop (or was 0): embed the final labels
        Workspace pass(stream);
        DevStatus *pst = nullptr;
        rc = graph_pass_enqueue(pass, graph, Y, 1, K, 0, Z, &pst, stream);
        if (rc != GEE_OK)
            return rc;
        DevStatus hs;
        if ((e = cudaMemcpyAsync(&hs, pst, sizeof(hs), cudaMemcpyDeviceToHost,
                                 stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(stream)) != cudaSuccess)
            return from_cuda(e);
        if (hs.code != GEE_OK)
            return static_cast<gee_status>(hs.code);
    }
    return GEE_OK;
}
