// graphgen.cu -- device side of the seeded input generators (graphgen/).
//
// Same definitions as the numpy implementation in graphgen/__init__.py:
// Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed with counter
// (index_lo, index_hi, word2, tag); R-MAT with 16-bit quadrant draws, a keyed
// bijection of [0, 2^scale) for node ids and redraws of out-of-range edges;
// uniform labels with a fraction set to -1; weights in (0, 1].  This library
// draws inputs only and holds none of the embedding's arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#define GG_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr uint32_t kTagRmat = 0x524D4154u;
constexpr uint32_t kTagPerm = 0x5045524Du;
constexpr uint32_t kTagLabel = 0x4C41424Cu;
constexpr uint32_t kTagWeight = 0x57474854u;
constexpr uint32_t kTagPlanted = 0x504C4E54u;
constexpr int kMaxAttempts = 64;
constexpr uint64_t kPermMul1 = 0x2545F491ull;
constexpr uint64_t kPermMul2 = 0x9E3779B1ull;

struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                     uint32_t c3, uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        if (r != 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    return U4{c0, c1, c2, c3};
}

struct RmatParams {
    int64_t start, count, n;
    uint64_t seed;
    uint32_t A, AB, ABC;
    uint32_t ka, kb;
    int scale;
};

__device__ inline uint64_t permute(uint64_t x, const RmatParams &p)
{
    const uint64_t mask = (p.scale >= 64) ? ~0ull : ((1ull << p.scale) - 1);
    const int h = p.scale / 2 > 1 ? p.scale / 2 : 1;
    x = (x ^ p.ka) & mask;
    x = (x * kPermMul1) & mask;
    x ^= x >> h;
    x = (x * kPermMul2) & mask;
    x ^= x >> h;
    x = (x ^ p.kb) & mask;
    return x;
}

__global__ void k_rmat(int2 *__restrict__ out, RmatParams p)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    for (int64_t i = tid; i < p.count; i += nthreads) {
        const uint64_t idx = (uint64_t)(p.start + i);
        uint64_t u = 0, v = 0;
        for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
            u = 0;
            v = 0;
            const int ncalls = (p.scale + 7) / 8;
            for (int call = 0; call < ncalls; ++call) {
                const U4 w = philox((uint32_t)idx, (uint32_t)(idx >> 32),
                                    (uint32_t)(attempt * 8 + call), kTagRmat,
                                    k0, k1);
                const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int level = call * 8 + j;
                    if (level < p.scale) {
                        const uint32_t r = (words[j / 2] >> (16 * (j % 2))) & 0xFFFFu;
                        const uint64_t ub = r >= p.AB;
                        const uint64_t vb = (r >= p.A && r < p.AB) || r >= p.ABC;
                        u = (u << 1) | ub;
                        v = (v << 1) | vb;
                    }
                }
            }
            u = permute(u, p);
            v = permute(v, p);
            if ((int64_t)u < p.n && (int64_t)v < p.n)
                break;
            if (attempt == kMaxAttempts - 1) {
                u %= (uint64_t)p.n;
                v %= (uint64_t)p.n;
            }
        }
        out[i] = make_int2((int)u, (int)v);
    }
}

__global__ void k_labels(int32_t *__restrict__ out, int64_t start,
                         int64_t count, int32_t K, uint64_t thr, uint64_t seed)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t i = tid; i < count; i += nthreads) {
        const uint64_t idx = (uint64_t)(start + i);
        const U4 w = philox((uint32_t)idx, (uint32_t)(idx >> 32), 0u,
                            kTagLabel, k0, k1);
        int32_t cls = (int32_t)(((uint64_t)w.y * (uint64_t)K) >> 32);
        if ((uint64_t)w.x < thr)
            cls = -1;
        out[i] = cls;
    }
}

__global__ void k_weights(float *__restrict__ out, int64_t start,
                          int64_t count, uint64_t seed)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t i = tid; i < count; i += nthreads) {
        const uint64_t idx = (uint64_t)(start + i);
        const U4 w = philox((uint32_t)idx, (uint32_t)(idx >> 32), 0u,
                            kTagWeight, k0, k1);
        out[i] = (float)((w.x >> 8) + 1u) * (1.0f / 16777216.0f);
    }
}

// Planted partition drawn edge by edge (see planted_edges in Python).
__global__ void k_planted(int2 *__restrict__ out, int64_t start, int64_t count,
                          uint64_t n, uint64_t K, uint64_t thr, uint64_t seed)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t i = tid; i < count; i += nthreads) {
        const uint64_t idx = (uint64_t)(start + i);
        const U4 w = philox((uint32_t)idx, (uint32_t)(idx >> 32), 0u,
                            kTagPlanted, k0, k1);
        const uint64_t u = ((uint64_t)w.x * n) >> 32;
        const uint64_t g = (u * K) / n;
        const uint64_t b0 = (g * n + K - 1) / K;
        const uint64_t b1 = ((g + 1) * n + K - 1) / K;
        const uint64_t size = b1 - b0;
        uint64_t v;
        if ((uint64_t)w.y < thr) {
            v = b0 + (((uint64_t)w.z * size) >> 32);
        } else {
            const uint64_t r = ((uint64_t)w.z * (n - size)) >> 32;
            v = r < b0 ? r : r + size;
        }
        out[i] = make_int2((int)u, (int)v);
    }
}

__global__ void k_planted_labels(int32_t *__restrict__ out, int64_t n,
                                 int64_t K)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nthreads)
        out[i] = (int32_t)((i * K) / n);
}

int blocks_for(int64_t count)
{
    int64_t b = (count + 255) / 256;
    if (b < 1)
        b = 1;
    if (b > 152 * 32)
        b = 152 * 32;
    return (int)b;
}

}  // namespace

// Edges [start, start+count) of the R-MAT graph into out (int32 pairs).
GG_API int graphgen_rmat(void *out, int64_t start, int64_t count, int scale,
                         int64_t n, uint32_t A, uint32_t AB, uint32_t ABC,
                         uint64_t seed, void *stream)
{
    if (count <= 0)
        return 0;
    if (scale < 1 || scale > 31 || n < 1 || n > (1ll << scale))
        return 1;
    RmatParams p;
    p.start = start;
    p.count = count;
    p.n = n;
    p.seed = seed;
    p.A = A;
    p.AB = AB;
    p.ABC = ABC;
    p.scale = scale;
    const U4 keys = philox(0u, 0u, 0u, kTagPerm, (uint32_t)seed,
                           (uint32_t)(seed >> 32));
    p.ka = keys.x;
    p.kb = keys.y;
    k_rmat<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(
        static_cast<int2 *>(out), p);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

GG_API int graphgen_labels(void *out, int64_t start, int64_t count, int32_t K,
                           uint64_t thr, uint64_t seed, void *stream)
{
    if (count <= 0)
        return 0;
    k_labels<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(
        static_cast<int32_t *>(out), start, count, K, thr, seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

GG_API int graphgen_weights(void *out, int64_t start, int64_t count,
                            uint64_t seed, void *stream)
{
    if (count <= 0)
        return 0;
    k_weights<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(
        static_cast<float *>(out), start, count, seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

GG_API int graphgen_planted(void *out, int64_t start, int64_t count, int64_t n,
                            int32_t K, uint64_t thr, uint64_t seed,
                            void *stream)
{
    if (count <= 0)
        return 0;
    if (n < 1 || n > 2147483647ll || K < 1 || K > n)
        return 1;
    k_planted<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(
        static_cast<int2 *>(out), start, count, (uint64_t)n, (uint64_t)K, thr,
        seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

GG_API int graphgen_planted_labels(void *out, int64_t n, int32_t K,
                                   void *stream)
{
    if (n <= 0)
        return 0;
    if (K < 1)
        return 1;
    k_planted_labels<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
        static_cast<int32_t *>(out), n, K);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
