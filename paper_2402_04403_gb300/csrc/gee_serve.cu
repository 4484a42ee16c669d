// gee_serve.cu -- the serving runtime behind gee_server_* (include/gee.h).
//
// One scheduler thread per server owns the GPU work.  Per loop it
//   1. polls the launch groups in flight (one CUDA event each) and
//      completes their requests,
//   2. admits waiting requests in arrival order while a slot (stream) is
//      free and their estimated device bytes fit in the budget next to the
//      resident graphs, folding compatible requests into one group:
//        edge lists     -> one gee_embed_batch launch sequence
//        re-labelings   -> one multi-label pass over the resident graph,
//                          with every waiting request for the same graph,
//                          K and variant
//   3. sleeps until a submission or a poll interval passes.
// A group is enqueued on its slot's stream in full -- host->device copies,
// kernels, status and Z back to the host (copies, or a split kernel that
// writes page-locked targets of a multi-label pass), event -- with its scratch
// freed stream-ordered behind it, so the thread never waits for the GPU and
// groups on different slots overlap.  An edge-list group's kernels are one
// CUDA graph launch: each slot captures the batch sequence once, over its
// own fixed header and problem table -- except a group whose cells belong
// mostly to large requests (Z beyond 2^24 cells), which runs the binned
// sequence instead (its launches are sized by the group).  Clients only
// touch the queue.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "gee_internal.cuh"

namespace gee {

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kDefaultBudget = int64_t(80) << 30;
constexpr int kDefaultStreams = 4;
constexpr int kMaxStreams = 16;
constexpr int kDefaultMaxBatch = 256;
constexpr int kMaxBatch = 4096;
constexpr int64_t kDefaultBatchEdges = int64_t(1) << 28;
constexpr int64_t kSlack = 64 << 10;  // per-group allowance for small scratch
constexpr auto kPoll = std::chrono::microseconds(50);

struct Req {
    int64_t ticket = 0;
    gee_request r{};
    int64_t n = 0, s = 0;      // rows of Z, edges
    int64_t bytes = 0;         // device bytes while in flight
    Clock::time_point t0, t1;
    gee_status status = GEE_OK;
    bool done = false;
    bool waited = false;       // a gee_server_wait has claimed it
};

struct GraphEntry {
    gee_graph *g = nullptr;
    int64_t n = 0, s = 0, hub_rows = 0, hub_arcs = 0;
    int64_t bytes = 0;
    bool weighted = false;
    bool lap_counted = false;
    int64_t users = 0;         // requests queued or in flight
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevStatus *host_st = nullptr;      // pinned [kMaxBatch]
    BatchProblem *host_tab = nullptr;  // pinned [kMaxBatch]
    BatchHeader *host_hdr = nullptr;   // pinned
    float **host_dst = nullptr;        // pinned [kMaxBatch]: split targets
    BatchHeader *dev_hdr = nullptr;    // the batch sequence's header and
    BatchProblem *dev_tab = nullptr;   // table [kMaxBatch], statuses
    DevStatus *dev_st = nullptr;       // [kMaxBatch], fixed per slot
    cudaGraphExec_t batch_graph = nullptr;  // the sequence, captured once
    bool busy = false;
    bool multi = false;                // re-label group
    bool binned = false;               // edge-list group run binned
    int64_t n = 0;                     // rows of the re-label group's graph
    int64_t bytes = 0;
    std::vector<Req *> reqs;
    gee_status launch_error = GEE_OK;
};

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Copies column block l of a multi-label Z (n rows of L*K floats, vector l
// in columns [l*K, (l+1)*K)) to dst[l] (n rows of K floats), one grid row
// per vector; a null dst[l] is skipped.  The targets are page-locked host
// buffers seen through their device addresses, so every store crosses the
// host link, whose rate depends on whole 128-byte lines and on the stores in
// flight: up to 31 leading scalars bring a target to a line boundary, the
// body goes out as 16-byte stores, and each thread loads four of them before
// it stores any.  A strided device-to-host copy with rows this short (K*4
// bytes) moves a fraction of the link rate.
constexpr int kSplitThreads = 256;
constexpr int kSplitQuads = 4;
constexpr int kSplitBlocks = 64;  // in all; enough for the link, few SMs

__global__ void __launch_bounds__(kSplitThreads)
k_split_vectors(const float *__restrict__ Z, int64_t n, int32_t L, int32_t K,
                float *const *__restrict__ dst)
{
    float *d = dst[blockIdx.y];
    if (d == nullptr)
        return;
    const int64_t cells = n * K;
    const int64_t LK = (int64_t)L * K;
    const int64_t col0 = (int64_t)blockIdx.y * K;
    const auto src = [&](int64_t c) {
        const int64_t u = c / K;
        return __ldg(Z + u * LK + col0 + (c - u * K));
    };
    // d is 4-byte aligned: head = floats up to the next 128-byte line
    int64_t head =
        (int64_t)(((128u - (uint32_t)(reinterpret_cast<uintptr_t>(d) & 127u)) &
                   127u) >> 2);
    if (head > cells)
        head = cells;
    const int64_t quads = (cells - head) >> 2;
    const int64_t tail0 = head + quads * 4;
    if (blockIdx.x == 0) {
        const int64_t t = threadIdx.x;
        if (t < head)
            d[t] = src(t);
        if (t < cells - tail0)
            d[tail0 + t] = src(tail0 + t);
    }
    float4 *dq = reinterpret_cast<float4 *>(d + head);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
         q0 < quads; q0 += stride * kSplitQuads) {
        float v[kSplitQuads][4];
#pragma unroll
        for (int j = 0; j < kSplitQuads; ++j) {
            const int64_t q = q0 + j * stride;
            if (q < quads) {
                const int64_t c = head + q * 4;
                int64_t u = c / K;
                int32_t k = (int32_t)(c - u * K);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    v[j][e] = __ldg(Z + u * LK + col0 + k);
                    if (++k == K) {
                        k = 0;
                        ++u;
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kSplitQuads; ++j) {
            const int64_t q = q0 + j * stride;
            if (q < quads)
                dq[q] = make_float4(v[j][0], v[j][1], v[j][2], v[j][3]);
        }
    }
}

#define GEE_CHECK_CUDA_RET(x)                                                  \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess)                                                 \
            return from_cuda(e_);                                              \
    } while (0)

}  // namespace

}  // namespace gee

using namespace gee;

struct gee_server {
    gee_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<int64_t, Req *> reqs;
    std::unordered_map<int64_t, GraphEntry> graphs;
    int64_t next_ticket = 1, next_graph = 0;
    int64_t resident_bytes = 0, inflight_bytes = 0;
    std::vector<Slot> slots;
    std::thread worker;
    bool stopping = false;
    gee_server_stats stats{};
    cudaStream_t setup_stream = nullptr;

    void loop();
    bool admit(std::unique_lock<std::mutex> &lk);
    void complete(Slot &sl);
    gee_status launch_edges(Slot &sl);
    gee_status launch_relabel(Slot &sl, GraphEntry &ge);
    void finish(Req *q, gee_status st);
};

namespace {

int64_t edge_request_bytes(int64_t s, int64_t n, int32_t K, bool weighted)
{
    int64_t b = align256(s * 8) + (weighted ? align256(s * 4) : 0) +
                align256(n * 4) + align256(n * (int64_t)K * 4) +
                align256(n + 16) + align256((int64_t)K * 4) +
                align256(sizeof(BatchProblem)) + 1024;
    // a large request makes its group run binned: record scratch (the
    // group's records are at most the sum of its requests')
    if (n * (int64_t)K > kBinnedMinCells) {
        const int64_t rows = bin_rows(K, weighted);
        b += (int64_t)bin_scratch_bytes(2 * s, (n + rows - 1) / rows, weighted);
    }
    return b;
}

int64_t relabel_request_bytes(int64_t n, int32_t K)
{
    return align256(n * 4) + align256(n * (int64_t)K * 4);
}

// Scratch of a re-label group of L vectors beyond its requests' own bytes:
// compact labels, class sizes, tiles or hub partials.
int64_t relabel_group_bytes(const GraphEntry &ge, int32_t L, int32_t K)
{
    const int64_t cols = (int64_t)L * K;
    const int64_t ls = L > 1 ? label_stride(L) : 1;
    const int64_t chunks = ge.hub_arcs / kHubChunk + ge.hub_rows + 1;
    const int64_t tiles =
        (2 * ge.s + ge.n * (cols > 16 ? cols : 16)) / kTileUnits + 2;
    return align256(ge.n * ls + 16) + align256(cols * 4) +
           align256(chunks * cols * 4) + align256(tiles * 4) + kSlack;
}

}  // namespace

void gee_server::finish(Req *q, gee_status st)
{
    q->status = st;
    q->done = true;
    q->t1 = Clock::now();
    ++stats.completed;
    if (st != GEE_OK)
        ++stats.failed;
    if (q->r.graph >= 0) {
        auto it = graphs.find(q->r.graph);
        if (it != graphs.end())
            --it->second.users;
    }
}

// Called with the lock held, after the slot's event has completed.
void gee_server::complete(Slot &sl)
{
    inflight_bytes -= sl.bytes;
    sl.busy = false;
    if (sl.launch_error != GEE_OK) {
        for (Req *q : sl.reqs)
            finish(q, sl.launch_error);
    } else if (!sl.multi) {
        if (!sl.binned)
            ++stats.graph_launches;
        for (size_t i = 0; i < sl.reqs.size(); ++i)
            finish(sl.reqs[i], static_cast<gee_status>(sl.host_st[i].code));
    } else {
        const gee_status st = static_cast<gee_status>(sl.host_st[0].code);
        if (st == GEE_ERR_LABEL_RANGE && sl.reqs.size() > 1 && sl.n > 0) {
            // the multi-label check names vector l = index / n: fail that
            // request, run the others again (at the head of the queue)
            const size_t bad = (size_t)(sl.host_st[0].index / (uint64_t)sl.n);
            for (size_t i = sl.reqs.size(); i-- > 0;) {
                if (i == bad)
                    finish(sl.reqs[i], st);
                else
                    pending.push_front(sl.reqs[i]);
            }
        } else {
            for (Req *q : sl.reqs)
                finish(q, st);
        }
    }
    sl.reqs.clear();
    cv_done.notify_all();
}

gee_status gee_server::launch_edges(Slot &sl)
{
    cudaStream_t st = sl.stream;
    const int count = (int)sl.reqs.size();
    Workspace ws(st);
    for (int i = 0; i < count; ++i) {
        const Req *q = sl.reqs[(size_t)i];
        BatchProblem &p = sl.host_tab[i];
        p = BatchProblem{};
        int32_t *E = nullptr, *Y = nullptr;
        float *W = nullptr, *Z = nullptr;
        GEE_CHECK_CUDA_RET(ws.alloc((void **)&E, (size_t)q->s * 8));
        GEE_CHECK_CUDA_RET(ws.alloc((void **)&Y, (size_t)q->n * 4));
        GEE_CHECK_CUDA_RET(ws.alloc((void **)&Z, (size_t)(q->n * q->r.K) * 4));
        if (q->r.weights_h != nullptr)
            GEE_CHECK_CUDA_RET(ws.alloc((void **)&W, (size_t)q->s * 4));
        if (q->s > 0)
            GEE_CHECK_CUDA_RET(cudaMemcpyAsync(E, q->r.edges_h, (size_t)q->s * 8,
                                               cudaMemcpyHostToDevice, st));
        if (W != nullptr && q->s > 0)
            GEE_CHECK_CUDA_RET(cudaMemcpyAsync(W, q->r.weights_h,
                                               (size_t)q->s * 4,
                                               cudaMemcpyHostToDevice, st));
        if (q->n > 0)
            GEE_CHECK_CUDA_RET(cudaMemcpyAsync(Y, q->r.Y_h, (size_t)q->n * 4,
                                               cudaMemcpyHostToDevice, st));
        p.E = E;
        p.w = W;
        p.Y = Y;
        p.Z = Z;
        p.s = q->s;
        p.n = q->n;
        p.K = q->r.K;
    }
    BatchHeader &hh = *sl.host_hdr;
    hh = BatchHeader{};
    batch_layout(sl.host_tab, count, hh);
    // header, table and statuses live in the slot's fixed buffers, which
    // the slot's captured batch sequence reads
    BatchHeader *dh = sl.dev_hdr;
    BatchProblem *dP = sl.dev_tab;
    DevStatus *dst = sl.dev_st;
    uint32_t *counts = nullptr;
    uint8_t *Yc = nullptr;
    GEE_CHECK_CUDA_RET(ws.alloc((void **)&counts, sizeof(uint32_t) * hh.count_cells));
    GEE_CHECK_CUDA_RET(ws.alloc((void **)&Yc, (size_t)hh.yc_bytes + 16));
    for (int i = 0; i < count; ++i) {
        BatchProblem &p = sl.host_tab[i];
        p.st = dst + i;
        p.counts = counts + p.counts_off;
        p.Yc = Yc + p.yc_off;
    }
    hh.counts = counts;
    GEE_CHECK_CUDA_RET(cudaMemcpyAsync(dh, &hh, sizeof(hh),
                                       cudaMemcpyHostToDevice, st));
    GEE_CHECK_CUDA_RET(cudaMemcpyAsync(dP, sl.host_tab,
                                       sizeof(BatchProblem) * count,
                                       cudaMemcpyHostToDevice, st));
    // large requests: labels, then one binned sequence over the group's
    // row tiles (launches sized by the group, so not the captured graph);
    // else the slot's captured batch sequence with pushed atomics
    sl.binned = batch_prefers_binned(sl.host_tab, count) &&
                binned_batch_tiles(sl.host_tab, count) > 0;
    if (sl.binned) {
        GEE_CHECK_CUDA_RET(batch_labels_enqueue(dh, dP, st));
        GEE_CHECK_CUDA_RET(launch_binned_batch(ws, sl.host_tab, count, st));
    } else {
        GEE_CHECK_CUDA_RET(cudaGraphLaunch(sl.batch_graph, st));
    }
    GEE_CHECK_CUDA_RET(cudaMemcpyAsync(sl.host_st, dst,
                                       sizeof(DevStatus) * count,
                                       cudaMemcpyDeviceToHost, st));
    for (int i = 0; i < count; ++i) {
        const Req *q = sl.reqs[(size_t)i];
        const size_t zb = (size_t)(q->n * q->r.K) * 4;
        if (zb > 0)
            GEE_CHECK_CUDA_RET(cudaMemcpyAsync(q->r.Z_h, sl.host_tab[i].Z, zb,
                                               cudaMemcpyDeviceToHost, st));
    }
    return GEE_OK;
}

gee_status gee_server::launch_relabel(Slot &sl, GraphEntry &ge)
{
    cudaStream_t st = sl.stream;
    const int32_t L = (int32_t)sl.reqs.size();
    const int32_t K = sl.reqs[0]->r.K;
    const int32_t lap = sl.reqs[0]->r.laplacian;
    const int64_t n = ge.n;
    Workspace ws(st);
    int32_t *Y = nullptr;
    float *Z = nullptr;
    GEE_CHECK_CUDA_RET(ws.alloc((void **)&Y, (size_t)(n * L) * 4));
    GEE_CHECK_CUDA_RET(ws.alloc((void **)&Z, (size_t)(n * L * K) * 4));
    for (int32_t l = 0; l < L; ++l)
        if (n > 0)
            GEE_CHECK_CUDA_RET(cudaMemcpyAsync(Y + (size_t)l * n,
                                               sl.reqs[(size_t)l]->r.Y_h,
                                               (size_t)n * 4,
                                               cudaMemcpyHostToDevice, st));
    DevStatus *dst = nullptr;
    gee_status rc = graph_pass_enqueue(ws, ge.g, Y, L, K, lap, Z, &dst, st);
    if (rc != GEE_OK)
        return rc;
    GEE_CHECK_CUDA_RET(cudaMemcpyAsync(sl.host_st, dst, sizeof(DevStatus),
                                       cudaMemcpyDeviceToHost, st));
    if (n == 0)
        return GEE_OK;
    if (L == 1) {
        GEE_CHECK_CUDA_RET(cudaMemcpyAsync(sl.reqs[0]->r.Z_h, Z,
                                           (size_t)(n * K) * 4,
                                           cudaMemcpyDeviceToHost, st));
        return GEE_OK;
    }
    // page-locked targets: one split kernel writes them over the link;
    // pageable ones: a strided copy each
    int32_t mapped = 0;
    for (int32_t l = 0; l < L; ++l) {
        sl.host_dst[l] = mapped_host(sl.reqs[(size_t)l]->r.Z_h);
        mapped += sl.host_dst[l] != nullptr ? 1 : 0;
    }
    if (mapped > 0) {
        float **dtab = nullptr;
        GEE_CHECK_CUDA_RET(ws.alloc((void **)&dtab, sizeof(float *) * L));
        GEE_CHECK_CUDA_RET(cudaMemcpyAsync(dtab, sl.host_dst,
                                           sizeof(float *) * L,
                                           cudaMemcpyHostToDevice, st));
        const dim3 grid((unsigned)((kSplitBlocks + L - 1) / L), (unsigned)L);
        k_split_vectors<<<grid, kSplitThreads, 0, st>>>(Z, n, L, K, dtab);
        GEE_CHECK_CUDA_RET(cudaGetLastError());
    }
    for (int32_t l = 0; l < L; ++l)
        if (sl.host_dst[l] == nullptr)
            GEE_CHECK_CUDA_RET(cudaMemcpy2DAsync(
                sl.reqs[(size_t)l]->r.Z_h, (size_t)K * 4, Z + (size_t)l * K,
                (size_t)L * K * 4, (size_t)K * 4, (size_t)n,
                cudaMemcpyDeviceToHost, st));
    return GEE_OK;
}

// Admits at most one group; returns whether one was launched.  Called with
// the lock held; the launch itself runs unlocked.
bool gee_server::admit(std::unique_lock<std::mutex> &lk)
{
    Slot *slot = nullptr;
    for (Slot &sl : slots)
        if (!sl.busy) {
            slot = &sl;
            break;
        }
    if (slot == nullptr || pending.empty())
        return false;
    const int64_t room = cfg.hbm_budget_bytes - resident_bytes;
    Req *head = pending.front();
    int64_t head_bytes = head->bytes;
    GraphEntry *ge = nullptr;
    if (head->r.graph >= 0) {
        ge = &graphs.at(head->r.graph);
        head_bytes += relabel_group_bytes(*ge, 1, head->r.K);
        if (head->r.laplacian && !ge->lap_counted)
            head_bytes += align256(ge->s * 8 + 16);
    }
    if (head_bytes > room) {
        // can never fit: fail it rather than block the queue for ever
        pending.pop_front();
        finish(head, GEE_ERR_OOM);
        cv_done.notify_all();
        return true;
    }
    if (inflight_bytes + head_bytes > room)
        return false;  // wait for running groups to finish
    std::vector<Req *> group{head};
    pending.pop_front();
    int64_t bytes = head_bytes;
    if (ge == nullptr) {
        int64_t edges = head->s;
        while (!pending.empty() && (int)group.size() < cfg.max_batch) {
            Req *q = pending.front();
            if (q->r.graph >= 0 || edges + q->s > cfg.max_batch_edges ||
                inflight_bytes + bytes + q->bytes > room)
                break;
            group.push_back(q);
            edges += q->s;
            bytes += q->bytes;
            pending.pop_front();
        }
    } else {
        const int32_t K = head->r.K;
        const int64_t lap_extra = head_bytes - head->bytes -
                                  relabel_group_bytes(*ge, 1, K);
        int64_t sum = head->bytes;
        for (auto it = pending.begin(); it != pending.end();) {
            Req *q = *it;
            const int32_t L = (int32_t)group.size() + 1;
            if ((int)group.size() >= cfg.max_batch ||
                (int64_t)L * K > GEE_MAX_COLUMNS)
                break;
            if (q->r.graph == head->r.graph && q->r.K == K &&
                q->r.laplacian == head->r.laplacian) {
                const int64_t total = sum + q->bytes +
                                      relabel_group_bytes(*ge, L, K) + lap_extra;
                if (inflight_bytes + total > room)
                    break;
                group.push_back(q);
                sum += q->bytes;
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
        bytes = sum + relabel_group_bytes(*ge, (int32_t)group.size(), K);
        if (lap_extra > 0) {
            // the Laplacian arc values stay with the graph
            ge->lap_counted = true;
            ge->bytes += lap_extra;
            resident_bytes += lap_extra;
        }
    }
    slot->busy = true;
    slot->multi = (ge != nullptr);
    slot->n = ge != nullptr ? ge->n : 0;
    slot->bytes = bytes;
    slot->reqs = group;
    slot->launch_error = GEE_OK;
    inflight_bytes += bytes;
    if (inflight_bytes > stats.peak_inflight_bytes)
        stats.peak_inflight_bytes = inflight_bytes;
    ++stats.groups;
    if (group.size() > 1)
        stats.batched_requests += (int64_t)group.size();
    if ((int64_t)group.size() > stats.max_group)
        stats.max_group = (int64_t)group.size();
    int64_t busy = 0;
    for (const Slot &sl : slots)
        busy += sl.busy ? 1 : 0;
    if (busy > stats.max_concurrent)
        stats.max_concurrent = busy;

    lk.unlock();
    gee_status rc = ge != nullptr ? launch_relabel(*slot, *ge) : launch_edges(*slot);
    cudaError_t e = cudaEventRecord(slot->done, slot->stream);
    lk.lock();
    if (rc == GEE_OK && e != cudaSuccess)
        rc = from_cuda(e);
    slot->launch_error = rc;
    if (rc != GEE_OK && e != cudaSuccess) {
        // no event to wait for: complete the group now
        complete(*slot);
    }
    return true;
}

void gee_server::loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        for (Slot &sl : slots) {
            if (sl.busy) {
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaSuccess) {
                    complete(sl);
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    sl.launch_error = from_cuda(q);
                    complete(sl);
                    progressed = true;
                }
            }
        }
        while (admit(lk))
            progressed = true;
        bool any_busy = false;
        for (const Slot &sl : slots)
            any_busy = any_busy || sl.busy;
        if (stopping && pending.empty() && !any_busy)
            break;
        if (!progressed) {
            if (any_busy)
                cv_work.wait_for(lk, kPoll);
            else
                cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
        }
    }
}

extern "C" {

gee_status gee_server_create(const gee_server_config *cfg, gee_server **out)
{
    if (out == nullptr)
        return GEE_ERR_INVALID_ARG;
    *out = nullptr;
    gee_server_config c{};
    if (cfg != nullptr)
        c = *cfg;
    if (c.hbm_budget_bytes < 0 || c.streams < 0 || c.streams > kMaxStreams ||
        c.max_batch < 0 || c.max_batch > kMaxBatch || c.max_batch_edges < 0 ||
        c.reserved[0] != 0 || c.reserved[1] != 0)
        return GEE_ERR_INVALID_ARG;
    if (c.hbm_budget_bytes == 0)
        c.hbm_budget_bytes = kDefaultBudget;
    if (c.streams == 0)
        c.streams = kDefaultStreams;
    if (c.max_batch == 0)
        c.max_batch = kDefaultMaxBatch;
    if (c.max_batch_edges == 0)
        c.max_batch_edges = kDefaultBatchEdges;
    gee_server *srv = new gee_server();
    srv->cfg = c;
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&srv->setup_stream, cudaStreamNonBlocking);
    srv->slots.resize((size_t)c.streams);
    for (Slot &sl : srv->slots) {
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&sl.host_st, sizeof(DevStatus) * kMaxBatch);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&sl.host_tab,
                               sizeof(BatchProblem) * kMaxBatch);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&sl.host_hdr, sizeof(BatchHeader));
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&sl.host_dst, sizeof(float *) * kMaxBatch);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.dev_hdr, sizeof(BatchHeader));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.dev_tab, sizeof(BatchProblem) * kMaxBatch);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.dev_st, sizeof(DevStatus) * kMaxBatch);
        if (e == cudaSuccess)
            e = batch_graph_create(sl.dev_hdr, sl.dev_tab, true, sl.stream,
                                   &sl.batch_graph);
    }
    if (e != cudaSuccess) {
        gee_server_destroy(srv);
        return from_cuda(e);
    }
    srv->worker = std::thread([srv] { srv->loop(); });
    *out = srv;
    return GEE_OK;
}

gee_status gee_server_add_graph(gee_server *srv, const int32_t *edges_h,
                                const float *weights_h, int64_t s, int64_t n,
                                int64_t *graph_id)
{
    if (srv == nullptr || graph_id == nullptr || s < 0 || n < 0 ||
        (s > 0 && edges_h == nullptr))
        return GEE_ERR_INVALID_ARG;
    if (n > INT32_MAX)
        return GEE_ERR_OVERFLOW;
    if (s > 0 && n == 0)
        return GEE_ERR_NODE_RANGE;
    // resident CSR: row pointers, ranks, arcs (+ values) and hub tables
    const int64_t est = align256((n + 1) * 12) + align256((n + 31) / 32 * 4 + 4) +
                        align256(2 * s * 4 + 64) +
                        (weights_h != nullptr ? align256(2 * s * 4 + 64) : 0) +
                        align256(2 * s / kHubDegree * 24 + 64) + kSlack;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->resident_bytes + est > srv->cfg.hbm_budget_bytes)
            return GEE_ERR_OOM;
        srv->resident_bytes += est;  // reserved while building
    }
    gee_graph *g = nullptr;
    gee_status rc = GEE_OK;
    {
        cudaStream_t st = srv->setup_stream;
        Workspace ws(st);
        int32_t *E = nullptr;
        float *W = nullptr;
        cudaError_t e = ws.alloc((void **)&E, (size_t)s * 8);
        if (e == cudaSuccess && weights_h != nullptr)
            e = ws.alloc((void **)&W, (size_t)s * 4);
        if (e == cudaSuccess && s > 0)
            e = cudaMemcpyAsync(E, edges_h, (size_t)s * 8,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && W != nullptr && s > 0)
            e = cudaMemcpyAsync(W, weights_h, (size_t)s * 4,
                                cudaMemcpyHostToDevice, st);
        rc = e == cudaSuccess ? gee_graph_create(E, W, s, n, st, &g)
                              : from_cuda(e);
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->resident_bytes -= est;
    if (rc != GEE_OK)
        return rc;
    GraphEntry ge;
    ge.g = g;
    int64_t bytes = 0;
    gee_graph_info(g, &ge.n, &ge.s, &ge.hub_rows, &ge.hub_arcs, &bytes);
    ge.bytes = bytes;
    ge.weighted = weights_h != nullptr;
    srv->resident_bytes += bytes;
    srv->stats.resident_bytes = srv->resident_bytes;
    *graph_id = srv->next_graph++;
    srv->graphs.emplace(*graph_id, ge);
    return GEE_OK;
}

gee_status gee_server_drop_graph(gee_server *srv, int64_t graph_id)
{
    if (srv == nullptr)
        return GEE_ERR_INVALID_ARG;
    gee_graph *g = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->graphs.find(graph_id);
        if (it == srv->graphs.end() || it->second.users > 0)
            return GEE_ERR_INVALID_ARG;
        g = it->second.g;
        srv->resident_bytes -= it->second.bytes;
        srv->stats.resident_bytes = srv->resident_bytes;
        srv->graphs.erase(it);
    }
    gee_graph_destroy(g);
    return GEE_OK;
}

gee_status gee_server_submit(gee_server *srv, const gee_request *req,
                             int64_t *ticket)
{
    if (srv == nullptr || req == nullptr || ticket == nullptr)
        return GEE_ERR_INVALID_ARG;
    const gee_request &r = *req;
    if (r.K < 1)
        return GEE_ERR_INVALID_ARG;
    if (r.K > kMaxClasses)
        return GEE_ERR_UNSUPPORTED;
    Req *q = new Req();
    q->r = r;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        gee_status rc = GEE_OK;
        if (r.graph >= 0) {
            auto it = srv->graphs.find(r.graph);
            if (it == srv->graphs.end())
                rc = GEE_ERR_INVALID_ARG;
            else {
                q->n = it->second.n;
                q->s = it->second.s;
                if (q->n > 0 && (r.Y_h == nullptr || r.Z_h == nullptr))
                    rc = GEE_ERR_INVALID_ARG;
                q->bytes = relabel_request_bytes(q->n, r.K);
            }
        } else {
            if (r.laplacian)
                rc = GEE_ERR_UNSUPPORTED;
            else if (r.s < 0 || r.n < 0 || (r.s > 0 && r.edges_h == nullptr) ||
                     (r.n > 0 && (r.Y_h == nullptr || r.Z_h == nullptr)))
                rc = GEE_ERR_INVALID_ARG;
            else if (r.n > INT32_MAX || r.s > (INT64_MAX / 16))
                rc = GEE_ERR_OVERFLOW;
            else if (r.s > 0 && r.n == 0)
                rc = GEE_ERR_NODE_RANGE;
            q->n = r.n;
            q->s = r.s;
            q->bytes = edge_request_bytes(r.s, r.n, r.K, r.weights_h != nullptr);
        }
        if (rc != GEE_OK) {
            delete q;
            return rc;
        }
        if (srv->stopping) {
            delete q;
            return GEE_ERR_INVALID_ARG;
        }
        if (r.graph >= 0)
            ++srv->graphs.at(r.graph).users;
        q->ticket = srv->next_ticket++;
        q->t0 = Clock::now();
        srv->reqs.emplace(q->ticket, q);
        srv->pending.push_back(q);
        ++srv->stats.submitted;
        *ticket = q->ticket;
    }
    srv->cv_work.notify_one();
    return GEE_OK;
}

gee_status gee_server_wait(gee_server *srv, int64_t ticket, double *latency_ms)
{
    if (srv == nullptr)
        return GEE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end())
        return GEE_ERR_INVALID_ARG;
    Req *q = it->second;
    if (q->waited)
        return GEE_ERR_INVALID_ARG;  // another thread waits for it already
    q->waited = true;
    srv->cv_done.wait(lk, [q] { return q->done; });
    const gee_status st = q->status;
    if (latency_ms != nullptr)
        *latency_ms =
            std::chrono::duration<double, std::milli>(q->t1 - q->t0).count();
    srv->reqs.erase(it);
    delete q;
    return st;
}

gee_status gee_server_cancel(gee_server *srv, int64_t ticket)
{
    if (srv == nullptr)
        return GEE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end())
        return GEE_ERR_INVALID_ARG;
    for (auto p = srv->pending.begin(); p != srv->pending.end(); ++p)
        if (*p == it->second) {
            srv->pending.erase(p);
            srv->finish(it->second, GEE_ERR_CANCELLED);
            srv->cv_done.notify_all();
            return GEE_OK;
        }
    return GEE_ERR_INVALID_ARG;  // admitted or done
}

gee_status gee_server_get_stats(gee_server *srv, gee_server_stats *out)
{
    if (srv == nullptr || out == nullptr)
        return GEE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->resident_bytes = srv->resident_bytes;
    return GEE_OK;
}

void gee_server_destroy(gee_server *srv)
{
    if (srv == nullptr)
        return;
    if (srv->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stopping = true;
        }
        srv->cv_work.notify_all();
        srv->worker.join();
    }
    for (auto &kv : srv->graphs)
        gee_graph_destroy(kv.second.g);
    for (auto &kv : srv->reqs)
        delete kv.second;
    for (Slot &sl : srv->slots) {
        if (sl.stream != nullptr)
            cudaStreamSynchronize(sl.stream);
        if (sl.done != nullptr)
            cudaEventDestroy(sl.done);
        if (sl.stream != nullptr)
            cudaStreamDestroy(sl.stream);
        if (sl.host_st != nullptr)
            cudaFreeHost(sl.host_st);
        if (sl.host_tab != nullptr)
            cudaFreeHost(sl.host_tab);
        if (sl.host_hdr != nullptr)
            cudaFreeHost(sl.host_hdr);
        if (sl.host_dst != nullptr)
            cudaFreeHost(sl.host_dst);
        if (sl.batch_graph != nullptr)
            cudaGraphExecDestroy(sl.batch_graph);
        if (sl.dev_hdr != nullptr)
            cudaFree(sl.dev_hdr);
        if (sl.dev_tab != nullptr)
            cudaFree(sl.dev_tab);
        if (sl.dev_st != nullptr)
            cudaFree(sl.dev_st);
    }
    if (srv->setup_stream != nullptr)
        cudaStreamDestroy(srv->setup_stream);
    delete srv;
}

}  // extern "C"
