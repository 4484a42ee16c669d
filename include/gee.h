/*
 * gee.h -- C ABI of libgee: One-Hot Graph Encoder Embedding (GEE) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: "Edge-Parallel Graph Encoder Embedding" (Lubonja, Shen, Priebe,
 * Burns; arXiv 2402.04403), Algorithm 1.  Given an edge list E (s edges
 * (u, v, w)) and a label vector Y over n nodes with K classes, GEE builds the
 * projection W(i, Y(i)) = 1 / count(Y = Y(i)) (Alg. 1, W initialisation) and
 * in one pass over the edges accumulates
 *     Z(u, Y(v)) += W(v, Y(v)) * w      and      Z(v, Y(u)) += W(u, Y(u)) * w
 * (Alg. 1, loop body), i.e. Z = A W with A = M + M^T.
 *
 * Conventions shared by every entry point:
 *   - edges: int32 [s][2] row-major, (u, v) per edge, 0 <= u, v < n,
 *     8-byte aligned (one pair per load; GEE_ERR_INVALID_ARG otherwise).
 *     Each listed edge applies both updates (Section II: an undirected graph
 *     is two symmetric directed graphs; list each undirected edge once).  A
 *     self-loop adds 2w / n_k to Z[u, Y[u]].  Repeated edges add up.
 *   - weights: float32 [s] or NULL for unit weights (Section II).
 *   - Y: int32 [n]; 0..K-1 are classes, -1 means "class unknown" (the paper's
 *     label 0).  Unknown nodes contribute nothing but still receive a Z row.
 *     A class with no member gives an all-zero column.
 *   - K: 1 <= K <= GEE_MAX_CLASSES.
 *   - Z: float32 [n][K] row-major, written in full by every successful call.
 *   - laplacian != 0 selects the Laplacian variant, which the paper leaves
 *     out (Section II, end of the GEE paragraph).  Reading used: with
 *     d_u = sum of the weights of u's edges (a self-loop counts twice), every
 *     weight becomes w / sqrt(d_u d_v) before the pass.  Needs w >= 0.
 *   - Precision: unit weights without the Laplacian accumulate exact uint32
 *     counts C and give Z = RN32(C / n_k) (round to nearest float32 of the
 *     exact quotient), identical bit for bit on every run.  Weighted and
 *     Laplacian results accumulate in float32 and are scaled once per cell.
 *   - Pointers named *_h are host memory; all others are device memory of
 *     the current CUDA device.  The caller owns every buffer it passes.
 *     Device arrays of 4-byte elements (Y, weights, Z, counts) must be
 *     4-byte aligned (GEE_ERR_INVALID_ARG otherwise); wider alignment is
 *     used where present, never required.
 *   - Every call is enqueued on `stream` and returns after the stream has
 *     finished the call's work (it reads back a device status word), so the
 *     result is ready when the call returns GEE_OK.
 *   - Inputs are validated on the device before Z is touched: with
 *     GEE_ERR_LABEL_RANGE, or GEE_ERR_NODE_RANGE under the default options,
 *     Z is left unmodified.  Scratch memory comes from a stream-ordered pool
 *     owned by the library (one per device, kept between calls).
 *   - Calls on different streams may run concurrently.  A gee_graph may be
 *     used from several streams at once.
 */
#ifndef GEE_H
#define GEE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GEE_API __attribute__((visibility("default")))
#else
#define GEE_API
#endif

/* Same handle type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *gee_stream_t;

#define GEE_MAX_CLASSES 255
/* Z columns of one multi-label pass (label vectors x classes). */
#define GEE_MAX_COLUMNS 1024

typedef enum gee_status {
    GEE_OK = 0,
    GEE_ERR_INVALID_ARG = 1,  /* bad scalar, NULL pointer, negative weight with
                                 the Laplacian variant */
    GEE_ERR_LABEL_RANGE = 2,  /* some Y[i] outside [-1, K) */
    GEE_ERR_NODE_RANGE = 3,   /* some endpoint outside [0, n) */
    GEE_ERR_OVERFLOW = 4,     /* a size does not fit the index types */
    GEE_ERR_OOM = 5,          /* device memory exhausted */
    GEE_ERR_CUDA = 6,         /* a CUDA runtime call failed */
    GEE_ERR_TIMEOUT = 7,      /* a bounded device wait expired */
    GEE_ERR_UNSUPPORTED = 8,  /* e.g. K > GEE_MAX_CLASSES */
    GEE_ERR_CANCELLED = 9     /* a server request cancelled before it ran */
} gee_status;

/* Edge-pass strategy of the edge-list entry points.  AUTO takes BINNED when
 * Z has more than 2^24 cells (n*K; beyond the autotuner's grid, where
 * updates pushed into Z miss L2), else the choice gee_autotune measured for
 * the nearest problem shape when the device has a tuning table, else
 * PRIVATE when n*K fits in shared memory and every CTA would merge several
 * edges per cell, ATOMIC otherwise.  SEGMENTED (CSR by row, each Z row
 * written once, no global atomics) is what a gee_graph always uses. */
typedef enum gee_strategy {
    GEE_AUTO = 0,
    GEE_ATOMIC = 1,    /* edge stream, red.global atomics into Z */
    GEE_PRIVATE = 2,   /* per-CTA copy of Z in shared memory, then merged */
    GEE_SEGMENTED = 3, /* build CSR by row, then one pull pass per row tile */
    GEE_BINNED = 4     /* updates written as records grouped by Z row tile
                          (two partition passes), each tile summed in shared
                          memory and written once: no atomics on Z.  Float
                          sums keep each addition's rounding error beside
                          them (about one rounding per cell whatever the
                          row's degree).  Scratch: 6 bytes per update slot
                          (2s slots), 14 with weights or the Laplacian.
                          Endpoints are always checked before Z is written. */
} gee_strategy;

typedef struct gee_options {
    int32_t strategy;          /* gee_strategy */
    int32_t validate_edges;    /* 1: check all endpoints before touching Z
                                  (one extra read of the edge list in the
                                  ATOMIC/PRIVATE paths); 0: the pass checks
                                  endpoints itself and skips bad edges, Z is
                                  then unspecified on GEE_ERR_NODE_RANGE */
    int64_t private_max_cells; /* PRIVATE only when n*K <= this (0 = the
                                  shared-memory limit) */
    int32_t block;             /* threads per CTA of the ATOMIC/PRIVATE pass
                                  (0 = 256; multiple of 32, <= 1024) */
    int32_t deterministic;     /* 1: bitwise reproducible float sums.  Each
                                  weighted or Laplacian arc value is added as
                                  a 64-bit fixed-point integer (units of 2^-S,
                                  S = floor(62 - log2(longest row's arcs x
                                  bound)), bound = max |w|, or 1 for Laplacian
                                  values) and each cell is divided by n_k
                                  once in FP64, so results depend neither on
                                  the order of the additions nor on the arc
                                  order of a rebuilt graph; every arc value is
                                  rounded to a multiple of 2^-S.  Resident-
                                  graph passes and SEGMENTED edge-list calls
                                  (AUTO then picks SEGMENTED); with ATOMIC,
                                  PRIVATE or BINNED, with 8 or more label vectors of a
                                  weighted graph and in gee_embed_batch for
                                  weighted problems: GEE_ERR_UNSUPPORTED.
                                  Unit weights are exact counts either way. */
} gee_options;

/* Fills *opts with the defaults (AUTO, validate_edges = 1,
 * deterministic = 0). */
GEE_API void gee_options_default(gee_options *opts);

/* Human-readable name of a status code (static string). */
GEE_API const char *gee_status_string(gee_status status);

/*
 * Class sizes n_k = #{i : Y[i] = k} (Alg. 1, W initialisation; Alg. 2 runs it
 * as a parallel loop over k).  counts: device uint32 [K], overwritten.
 * GEE_ERR_LABEL_RANGE if a label is outside [-1, K); counts is then
 * unspecified.
 */
GEE_API gee_status gee_histogram(const int32_t *Y, int64_t n, int32_t K,
                         uint32_t *counts, gee_stream_t stream);

/*
 * Z = A W for an edge list (Alg. 1 / Alg. 2 of the paper): one call from
 * edges and labels to the embedding.  edges: device int32 [s][2]; weights:
 * device float [s] or NULL; Y: device int32 [n]; Z: device float [n][K],
 * written in full (caller-owned).  opts may be NULL (defaults).  Errors:
 * GEE_ERR_LABEL_RANGE / GEE_ERR_NODE_RANGE before Z is touched (see
 * validate_edges), GEE_ERR_INVALID_ARG for a negative weight with the
 * Laplacian variant, GEE_ERR_OOM when the scratch does not fit.
 */
GEE_API gee_status gee_embed(const int32_t *edges, const float *weights, int64_t s,
                     const int32_t *Y, int64_t n, int32_t K, int32_t laplacian,
                     float *Z, const gee_options *opts, gee_stream_t stream);

/* Same as gee_embed with host buffers: copies edges/weights/Y to the device,
 * runs the pass and copies Z back to Z_h (pinned host memory is fastest).
 * Same errors as gee_embed; Z_h is untouched unless the call succeeds. */
GEE_API gee_status gee_embed_host(const int32_t *edges_h, const float *weights_h,
                          int64_t s, const int32_t *Y_h, int64_t n, int32_t K,
                          int32_t laplacian, float *Z_h,
                          const gee_options *opts, gee_stream_t stream);

/*
 * A graph kept resident on the device: the edge list is sorted by row into a
 * symmetric CSR once (each edge (u,v,w) becomes arcs u->v and v->u; the
 * arcs of rows with more than GEE_HUB_DEGREE arcs are kept apart and split
 * into chunks).  This is the layout the paper's Ligra version iterates
 * (Section III: edgeMapDense walks each node's edge list); repeated
 * embeddings of the same graph with new label vectors then skip the upload
 * and the sort.  edges/weights are device pointers and are not referenced
 * after return; the graph owns its device arrays until gee_graph_destroy.
 * Negative weights are accepted (a Laplacian pass on such a graph fails).
 * Errors, with *out set to NULL: GEE_ERR_INVALID_ARG (out NULL, edges NULL
 * with s > 0, misaligned edges or weights, negative s or n),
 * GEE_ERR_OVERFLOW (n >= 2^31), GEE_ERR_NODE_RANGE (an endpoint outside
 * [0, n)), GEE_ERR_OOM.
 */
#define GEE_HUB_DEGREE 128
typedef struct gee_graph gee_graph;

GEE_API gee_status gee_graph_create(const int32_t *edges, const float *weights,
                            int64_t s, int64_t n, gee_stream_t stream,
                            gee_graph **out);

/* Z = A W for a resident graph and a label vector: Y device int32 [n],
 * Z device float [n][K] written in full, n the graph's.  Unit-weight
 * graphs give the bit-exact counts result.  opts may be NULL; of it only
 * deterministic is read (the resident pass has no strategy choice; block,
 * if set, must still be valid).  Calls on different streams may use one
 * graph at the same time.  Errors: GEE_ERR_INVALID_ARG (graph, Y or Z NULL,
 * Y or Z misaligned, Laplacian on a graph with a negative weight),
 * GEE_ERR_UNSUPPORTED (K > GEE_MAX_CLASSES), GEE_ERR_LABEL_RANGE with Z
 * untouched, GEE_ERR_OOM when the scratch does not fit. */
GEE_API gee_status gee_embed_graph(gee_graph *graph, const int32_t *Y, int32_t K,
                           int32_t laplacian, float *Z,
                           const gee_options *opts, gee_stream_t stream);

/*
 * L label vectors on one resident graph in a single pass: a W widened to
 * L*K columns, so every arc is read and its target's L labels gathered once
 * for all L embeddings (used for repeated re-labelings, e.g. unsupervised
 * GEE iterations).  Y: device int32 [L][n], vector l at Y + l*n.  Z: device
 * float [n][L*K] row-major, Z[u][l*K + k] = the embedding of node u for
 * label vector l.  Each vector has its own class sizes.  L >= 1, L*K <=
 * GEE_MAX_COLUMNS.  Same results as L separate gee_embed_graph calls.
 * Errors as gee_embed_graph, plus GEE_ERR_INVALID_ARG for L < 1 and
 * GEE_ERR_UNSUPPORTED for L*K > GEE_MAX_COLUMNS; a bad label in any vector
 * fails the whole call with Z untouched.
 */
GEE_API gee_status gee_embed_graph_multi(gee_graph *graph, const int32_t *Y,
                                         int32_t L, int32_t K,
                                         int32_t laplacian, float *Z,
                                         const gee_options *opts,
                                         gee_stream_t stream);

/* Same with host Y_h and Z_h.  A page-locked Z_h (cudaMallocHost or
 * cudaHostRegister) is written directly by the pass over the host link, so
 * the transfer overlaps the computation; pageable Z_h is filled by a copy
 * after the pass.  Either way Z_h is untouched when labels fail the check. */
GEE_API gee_status gee_embed_graph_host(gee_graph *graph, const int32_t *Y_h,
                                int32_t K, int32_t laplacian, float *Z_h,
                                const gee_options *opts, gee_stream_t stream);

/* Sizes of a resident graph: nodes, edges, rows kept in the hub CSR (more
 * than GEE_HUB_DEGREE arcs), their arcs, device bytes held by the CSR.  The
 * graph also keeps the row-tile split of up to 8 column counts it has been
 * embedded with (4 * ((2s + n * max(cols, 16)) / 1024 + 2) bytes each), so
 * later passes with the same K skip that step.  Any output pointer may be
 * NULL. */
GEE_API gee_status gee_graph_info(const gee_graph *graph, int64_t *n,
                                  int64_t *s, int64_t *hub_rows,
                                  int64_t *hub_arcs, int64_t *device_bytes);

/* Label gathers of one single-vector pass with K classes on a resident
 * graph (a measurement aid; no counterpart in the paper): arcs of hub rows
 * whose target's label the hub kernel reads from its shared-memory copy of
 * the most referenced labels (131,072 of them, or 163,840 as 6-bit codes
 * when K <= 63 and the graph has at least 2^25 nodes), the other arcs of
 * hub rows (gathered through L1 and L2),
 * and the arcs of the other rows.  Counts the first on the device and
 * waits for the stream.  Any output pointer may be NULL;
 * GEE_ERR_INVALID_ARG for a NULL graph or K outside [1, GEE_MAX_CLASSES]. */
GEE_API gee_status gee_graph_gathers(const gee_graph *graph, int32_t K,
                                     int64_t *hub_shared, int64_t *hub_other,
                                     int64_t *light, gee_stream_t stream);

/* Frees the graph after all device work has finished.  NULL is a no-op. */
GEE_API void gee_graph_destroy(gee_graph *graph);

/* The strategy gee_embed would run for these sizes and options. */
GEE_API gee_strategy gee_pick_strategy(int64_t s, int64_t n, int32_t K,
                               const gee_options *opts);

/* Upper bound of the scratch bytes gee_embed draws from the pool. */
GEE_API size_t gee_workspace_bytes(int64_t s, int64_t n, int32_t K,
                           int32_t weighted, int32_t laplacian,
                           const gee_options *opts);

/*
 * Unsupervised GEE on a resident unweighted graph.  Section II allows Y to
 * come from unsupervised clustering; the clustering here is k-means on the
 * embedding (Lloyd's assignment step), alternated with the pass: each round
 * embeds the current labels and moves every node to the nearest class mean
 * of that embedding, until a round moves no node or max_iter rounds ran.
 *   Y      device int32 [n], the starting labels, every one in 0..K-1;
 *          updated in place to the final labels
 *   K      1..64
 *   Z      device float [n][K]: the embedding of the final labels
 *   rounds host: rounds run (the last moved nothing unless max_iter ended
 *          the loop); moved: host int64 [max_iter] nodes moved per round,
 *          or NULL
 * With C the exact neighbour counts, m_k the class sizes, Z = RN32(C/m_j)
 * and S[k][j] the exact class sums of C, node i moves to the non-empty class
 * k with the smallest sum over j = 0..K-1 (in order, FP32, each operation
 * rounded on its own) of (Z[i][j] - RN32(S[k][j]/(m_k m_j)))^2, the lowest k
 * on ties, so every run takes the same decisions.  The paper fixes no
 * precision for this step; the FP32 distances differ from exact ones by at
 * most (K + 4) 2^-24 sum_j (|Z[i][j]| + |c[k][j]|)^2, so only classes whose
 * means are that close to equally near can be chosen differently from an
 * exact computation.  The counts are recovered from Z as rint(Z m_j), exact
 * below 2^23: a graph with a row of 2^23 or more arcs returns
 * GEE_ERR_OVERFLOW before any round runs.
 * GEE_ERR_UNSUPPORTED for weighted graphs or K > 64.
 */
GEE_API gee_status gee_unsupervised(gee_graph *graph, int32_t *Y, int32_t K,
                                    int32_t max_iter, float *Z,
                                    int32_t *rounds, int64_t *moved,
                                    gee_stream_t stream);

/*
 * Autotuning of GEE_AUTO for edge-list calls (no counterpart in the paper).
 * gee_autotune times ATOMIC (block sizes 128, 256, 512), PRIVATE (where Z
 * fits in shared memory) and SEGMENTED on seeded synthetic problems (K = 16,
 * uniform random edges) over a grid of Z sizes 2^10..2^24 cells and edge
 * densities 2s/cells = 2^-2..2^4 -- every second power of two with
 * effort 0, every one with efforts 1 and 2 (2 also takes more repetitions)
 * -- and installs the fastest choice per grid point for the current
 * device; it takes seconds (effort 0) to a minute.  GEE_AUTO then uses the
 * grid point nearest in (log2 cells, log2 density).  gee_tune_get copies
 * the current device's table (returns its size; 0 = not tuned, the built-in
 * rule applies); gee_tune_set installs a saved table (count 0 resets).
 */
typedef struct gee_tune_cell {
    int32_t log2_cells;      /* n*K of the grid point */
    int32_t log2_density;    /* 2s / (n*K) */
    int32_t strategy;        /* GEE_ATOMIC, GEE_PRIVATE or GEE_SEGMENTED */
    int32_t block;           /* threads per block (0: the default) */
    float ms_atomic;         /* measured median call times; -1 if not run */
    float ms_private;
    float ms_segmented;
    float reserved;
} gee_tune_cell;

GEE_API gee_status gee_autotune(int32_t effort, gee_stream_t stream);
GEE_API int32_t gee_tune_get(gee_tune_cell *out, int32_t max_cells);
GEE_API gee_status gee_tune_set(const gee_tune_cell *cells, int32_t count);

/*
 * Batched embedding: `count` independent problems, each with the arguments
 * of gee_embed (its own edges, weights, Y, n, K and Z; no Laplacian), run
 * by one sequence of persistent launches over all of them -- the batched
 * form of Alg. 1 for many small graphs, which would each leave most of the
 * GPU idle and pay several launches and a host round trip one call at a
 * time.  Per problem the result equals gee_embed's: bit for bit with unit
 * weights, within float32 summation order with weights.
 *
 * problems: host array [count]; the buffers it points to are device memory
 * and must not overlap between problems (Z of one problem is written while
 * others are read).  statuses: host array [count] filled with each
 * problem's status, or NULL.  A problem whose labels or endpoints fail the
 * device checks gets GEE_ERR_LABEL_RANGE / GEE_ERR_NODE_RANGE and its Z is
 * left unmodified (with opts->validate_edges = 0, a bad endpoint is skipped,
 * reported, and that problem's Z is undefined); the other problems are
 * still computed.  Returns GEE_OK when every problem succeeded, else the
 * status of the first failing problem (argument errors are found on the
 * host before anything runs).
 *
 * Edge pass: with opts->strategy GEE_BINNED, or GEE_AUTO when most of the
 * batch's Z cells belong to problems of more than 2^24 cells each (smaller
 * Z stay in L2 while pushed atomics land), the updates of all problems go through
 * one binned sequence (records grouped by row tile, each tile summed in
 * shared memory; float sums with their rounding errors kept beside them,
 * and if any problem has weights every problem is summed in float, which
 * is exact for counts below 2^24); endpoints are then always checked
 * before Z is written, whatever validate_edges says.  Otherwise updates
 * are pushed into Z with red.global atomics.  opts->block is ignored.
 */
typedef struct gee_problem {
    const int32_t *edges;    /* int32 [s][2], 8-byte aligned */
    const float *weights;    /* float [s], or NULL for unit weights */
    int64_t s;
    const int32_t *Y;        /* int32 [n] */
    int64_t n;
    int32_t K;
    int32_t reserved;        /* must be 0 */
    float *Z;                /* float [n][K], written */
} gee_problem;

GEE_API gee_status gee_embed_batch(const gee_problem *problems, int32_t count,
                                   gee_status *statuses,
                                   const gee_options *opts,
                                   gee_stream_t stream);

/*
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper, which embeds one graph per call).  Clients submit embedding
 * requests -- an edge list with its labels, or a new label vector for a
 * graph kept resident on the device (re-labeling, as in the unsupervised
 * GEE loop) -- from any thread, and wait for them by ticket.  One scheduler
 * thread admits requests in arrival order while the device memory they need
 * fits in the budget (with the resident graphs), and launches them as soon
 * as one of `streams` slots is free, so work that arrives while other
 * requests run overlaps with them on the GPU:
 *   - consecutive edge-list requests are fused into one gee_embed_batch
 *     launch sequence (up to max_batch requests / max_batch_edges edges),
 *     replayed as one CUDA graph captured per slot, or run binned when most
 *     of the group's cells belong to requests beyond 2^24 cells (as
 *     gee_embed_batch with GEE_AUTO);
 *   - re-labelings of the same resident graph with the same K and variant
 *     waiting anywhere in the queue are fused into one multi-label pass
 *     (W widened to L*K <= GEE_MAX_COLUMNS columns).
 * Each request's Z equals the result of the corresponding plain call (bit
 * for bit with unit weights; within float32 summation order and the
 * multi-label pass's reciprocal scaling, far below 1e-5 relative, with
 * weights).  Edge-list requests have no Laplacian variant here
 * (GEE_ERR_UNSUPPORTED).
 *
 * Host buffers of a request (edges_h, weights_h, Y_h, Z_h) must stay valid
 * until gee_server_wait returns for it; Z_h is written by then.  Page-locked
 * host buffers let copies overlap with other requests' kernels; pageable
 * ones work but make the scheduler wait for each copy.  If a request fails
 * (its status is returned by gee_server_wait), its Z_h is unspecified.
 */
typedef struct gee_server gee_server;

typedef struct gee_server_config {
    int64_t hbm_budget_bytes;  /* device bytes for resident graphs plus the
                                  requests in flight; 0: 80 GiB */
    int32_t streams;           /* launch groups in flight at once, 1..16;
                                  0: 4 */
    int32_t max_batch;         /* requests per launch group, 1..4096; 0: 256 */
    int64_t max_batch_edges;   /* edges per edge-list launch group; 0: 2^28 */
    int64_t reserved[2];       /* must be 0 */
} gee_server_config;

typedef struct gee_request {
    int64_t graph;             /* resident graph id, or -1 for an edge list */
    const int32_t *edges_h;    /* graph == -1: int32 [s][2] */
    const float *weights_h;    /* graph == -1: float [s] or NULL */
    int64_t s;                 /* graph == -1: edges */
    int64_t n;                 /* graph == -1: nodes (a resident graph has
                                  its own n) */
    const int32_t *Y_h;        /* int32 [n] */
    int32_t K;
    int32_t laplacian;         /* resident graphs only */
    float *Z_h;                /* float [n][K], written on completion */
} gee_request;

typedef struct gee_server_stats {
    int64_t submitted, completed, failed;
    int64_t groups;            /* launch groups */
    int64_t batched_requests;  /* requests that shared a group with others */
    int64_t max_group;         /* largest group */
    int64_t max_concurrent;    /* most groups in flight at once */
    int64_t resident_bytes;    /* estimated bytes of resident graphs */
    int64_t peak_inflight_bytes;
    int64_t graph_launches;    /* edge-list groups run as one CUDA graph
                                  (the others ran binned) */
} gee_server_stats;

/* cfg may be NULL (defaults).  Uses the current CUDA device. */
GEE_API gee_status gee_server_create(const gee_server_config *cfg,
                                     gee_server **out);
/* Builds a resident graph from a host edge list (synchronous); fails with
 * GEE_ERR_OOM if its estimated size does not fit in the budget. */
GEE_API gee_status gee_server_add_graph(gee_server *srv, const int32_t *edges_h,
                                        const float *weights_h, int64_t s,
                                        int64_t n, int64_t *graph_id);
/* Releases a resident graph; GEE_ERR_INVALID_ARG while requests use it. */
GEE_API gee_status gee_server_drop_graph(gee_server *srv, int64_t graph_id);
/* Queues a request (argument errors are returned here); *ticket identifies
 * it for gee_server_wait.  A request larger than the whole budget completes
 * with GEE_ERR_OOM. */
GEE_API gee_status gee_server_submit(gee_server *srv, const gee_request *req,
                                     int64_t *ticket);
/* Blocks until the request is done; returns its status and, if latency_ms
 * is not NULL, the time from submission to completion.  Each ticket can be
 * waited for once: a second wait, also one from another thread while the
 * first is still blocked, returns GEE_ERR_INVALID_ARG. */
GEE_API gee_status gee_server_wait(gee_server *srv, int64_t ticket,
                                   double *latency_ms);
/* Cancels a request that is still waiting for admission: it is removed
 * from the queue and finishes with GEE_ERR_CANCELLED (returned by its
 * gee_server_wait, its Z_h untouched).  GEE_ERR_INVALID_ARG for an unknown
 * ticket or one already running or done (it then completes as usual). */
GEE_API gee_status gee_server_cancel(gee_server *srv, int64_t ticket);
GEE_API gee_status gee_server_get_stats(gee_server *srv,
                                        gee_server_stats *out);
/* Finishes every queued request, then releases the server and its graphs.
 * Call it after every client thread's gee_server_wait has returned. */
GEE_API void gee_server_destroy(gee_server *srv);

/*
 * Allocation-free edge-list embedding.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory once
 * they are running -- for example a service whose device memory was divided
 * up at start-up by another allocator, or latency-critical code that must
 * not call into the driver's allocator mid-flight.
 *
 * Same result as gee_embed(edges, weights, s, Y, n, K, laplacian = 0, Z)
 * with the ATOMIC strategy and endpoint validation on, but it allocates
 * nothing: its scratch (status word, n_k, compact labels) lives in one fixed
 * array of GEE_NOALLOC_SCRATCH_BYTES in device global memory that belongs to
 * the library image, so every GPU that loads libgee holds those bytes until
 * the process exits.  The first call on a device looks up that array's
 * device address (once per device, kept for the life of the process); make
 * that first call before any stream capture.  A cudaDeviceReset destroys
 * the context the kept address belongs to, so do not call this entry point
 * on a device after resetting it.  Each call waits for its stream to
 * finish, to read the status word back.  n above GEE_NOALLOC_MAX_NODES
 * returns GEE_ERR_UNSUPPORTED.  The array is shared by all calls and keeps
 * the last call's contents (each call clears what must start at zero), so
 * calls whose work overlaps on the GPU race on it: run them one at a time.
 * No Laplacian variant.
 */
#define GEE_NOALLOC_SCRATCH_BYTES (16u << 20)
#define GEE_NOALLOC_MAX_NODES (GEE_NOALLOC_SCRATCH_BYTES - 2048u)
GEE_API gee_status gee_embed_noalloc(const int32_t *edges,
                                     const float *weights, int64_t s,
                                     const int32_t *Y, int64_t n, int32_t K,
                                     float *Z, gee_stream_t stream);

/*
 * Tracing.  While enabled (process-wide), every kernel launch of the library
 * is bracketed by two CUDA events on the stream it is launched on.
 * gee_profile_read waits for the recorded events, fills up to max_entries
 * per-kernel totals (sorted by name), clears the record and returns the
 * number of distinct kernels seen.  Adds two event records per launch.
 */
typedef struct gee_kernel_time {
    char name[32];      /* kernel name, NUL-terminated */
    int64_t launches;   /* launches recorded */
    double total_ms;    /* sum of event-to-event durations */
    double max_ms;      /* longest launch */
} gee_kernel_time;

GEE_API void gee_profile_enable(int32_t on);
GEE_API int32_t gee_profile_read(gee_kernel_time *out, int32_t max_entries);

/* Fault injection for tests: the next `count` device allocations made by
 * the library (scratch of a call, arrays of a resident graph) fail as if the
 * device were out of memory, so the calls that make them return GEE_ERR_OOM
 * and release what they had taken; 0 clears it.  The failure is made on the
 * host -- no allocation is attempted -- and the library stays usable. */
GEE_API void gee_debug_fail_allocs(int32_t count);

#ifdef __cplusplus
}
#endif

#endif /* GEE_H */
