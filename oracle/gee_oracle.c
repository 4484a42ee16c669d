/*
 * gee_oracle.c -- serial FP64 CPU oracle for One-Hot Graph Encoder Embedding
 * (GEE), "Edge-Parallel Graph Encoder Embedding" (Lubonja, Shen, Priebe,
 * Burns; arXiv 2402.04403), Algorithm 1.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path must compute.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Conventions (readings of the paper, each one listed in the design notes):
 *   - Edge list E is s rows of (u, v) int32 node ids, row-major (s x 2), with
 *     an optional float32 weight per edge; no weights means every edge
 *     weighs 1 (Section II).
 *   - Labels Y are int32: classes 0..K-1 and -1 for "class unknown".  The paper
 *     writes Y in {0..K} with 0 = unknown and classes 1..K (Alg. 1 input and
 *     the comment in its W-initialisation loop); -1/0..K-1 is the same
 *     encoding shifted by one.
 *   - Every listed edge applies both updates of Alg. 1 (the loop body): an
 *     undirected graph is listed once per edge, a self-loop (u,u,w) therefore
 *     adds 2w/n_k to Z[u,Y[u]].
 *   - Z is n x K, row-major, FP64.
 *
 * Laplacian variant: the paper omits its preprocessing (Section II, last
 * sentence of the GEE paragraph).  Reading used here, from the GEE work the
 * paper cites: d_u = sum over listed edges incident to u of w (a self-loop
 * adds 2w), and every edge weight is replaced by w / sqrt(d_u d_v) before the
 * same edge loop runs.  A node with d = 0 contributes nothing.
 *
 * Pins (tests under -m "not gpu"): hand-worked cases in tests/golden, the
 * dense closed form (M + M^T) W, exhaustive enumeration of all edge sets on
 * three, four and five nodes against exact rationals (on four nodes also
 * with signed dyadic weights, and in Laplacian form against a 40-digit
 * decimal evaluation), row/column-sum invariants, equivariance under edge
 * shuffles and node/class permutations, the K = 1 degree special case, SBM
 * block means, and scipy's normalised Laplacian for the Laplacian reading.
 * The paper prints no embedding values, so nothing here is pinned to a
 * printed number.
 *
 * Build: cc -O2 -std=c99 -ffp-contract=off -shared -fPIC gee_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum separately rounded, so x86
 * and Arm hosts give identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_BAD_ARG 1
#define ORC_BAD_LABEL 2
#define ORC_BAD_NODE 3
#define ORC_NO_MEMORY 4
#define ORC_BAD_WEIGHT 5

/*
 * Mutation switch for the test suite only: a non-zero value plants one known
 * mistake so the tests can show that their pins catch it.  0 = the oracle as
 * written.  Codes:
 *   1  drop the second update of the loop body (Z[v,Y[u]])
 *   2  first update indexes the class of u instead of v
 *   3  first update writes row v instead of row u
 *   4  treat an unknown label as class 0
 *   5  divide by the class size of the receiving node's class
 *   6  Laplacian: scale by 1/d_u instead of 1/sqrt(d_u d_v)
 *   7  self-loop applied once
 *   8  class sizes count unknown labels as class K-1
 *   9  unsupervised loop: centroids divided by m_k only (not m_k * m_j)
 */
int gee_oracle_mutation = 0;

void gee_oracle_set_mutation(int m) { gee_oracle_mutation = m; }

/*
 * Alg. 1, W initialisation (the loop over k): n_k = #{i : Y[i] = k}.  W itself
 * is W(i, Y(i)) = 1/n_{Y(i)} and zero elsewhere; every use below reads it as
 * 1/nk[Y[i]].
 */
int gee_oracle_class_counts(const int32_t *Y, int64_t n, int32_t K, int64_t *nk)
{
    if (K < 1 || n < 0 || (n > 0 && Y == NULL) || nk == NULL)
        return ORC_BAD_ARG;
    for (int32_t k = 0; k < K; ++k)
        nk[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t y = Y[i];
        if (y < -1 || y >= K)
            return ORC_BAD_LABEL;
        if (y == -1) {
            if (gee_oracle_mutation == 8)
                nk[K - 1] += 1;
            continue;
        }
        nk[y] += 1;
    }
    return ORC_OK;
}

/* Shared argument checks for the embedding entry points. */
static int check_inputs(const int32_t *E, const float *w, int64_t s,
                        const int32_t *Y, int64_t n, int32_t K, int laplacian)
{
    if (K < 1 || n < 0 || s < 0)
        return ORC_BAD_ARG;
    if ((s > 0 && E == NULL) || (n > 0 && Y == NULL))
        return ORC_BAD_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (Y[i] < -1 || Y[i] >= K)
            return ORC_BAD_LABEL;
    for (int64_t i = 0; i < s; ++i) {
        int64_t u = E[2 * i], v = E[2 * i + 1];
        if (u < 0 || u >= n || v < 0 || v >= n)
            return ORC_BAD_NODE;
        if (laplacian && w != NULL && !(w[i] >= 0.0f))
            return ORC_BAD_WEIGHT;
    }
    return ORC_OK;
}

/*
 * Laplacian reading: weighted degree d_u = sum_v A[u,v] with A = M + M^T,
 * i.e. every listed edge (u,v,w) adds w to d_u and w to d_v (2w to d_u for a
 * self-loop).
 */
int gee_oracle_degrees(const int32_t *E, const float *w, int64_t s, int64_t n,
                       double *d)
{
    if (n < 0 || s < 0 || (s > 0 && E == NULL) || (n > 0 && d == NULL))
        return ORC_BAD_ARG;
    for (int64_t i = 0; i < n; ++i)
        d[i] = 0.0;
    for (int64_t i = 0; i < s; ++i) {
        int64_t u = E[2 * i], v = E[2 * i + 1];
        if (u < 0 || u >= n || v < 0 || v >= n)
            return ORC_BAD_NODE;
        double wt = (w != NULL) ? (double)w[i] : 1.0;
        d[u] += wt;
        d[v] += wt;
    }
    return ORC_OK;
}

/* Edge weight after the optional Laplacian scaling w / sqrt(d_u d_v). */
static double edge_weight(const float *w, int64_t i, const double *d,
                          int64_t u, int64_t v)
{
    double wt = (w != NULL) ? (double)w[i] : 1.0;
    if (d == NULL)
        return wt;
    if (gee_oracle_mutation == 6)
        return d[u] > 0.0 ? wt / d[u] : 0.0;
    double dd = d[u] * d[v];
    return dd > 0.0 ? wt / sqrt(dd) : 0.0;
}

/*
 * One edge of Alg. 1's loop body, applied to a row-major Z (row stride K),
 * with only rows for which row_index() >= 0 stored.  W(x, Y(x)) = 1/n_{Y(x)}.
 */
typedef int64_t (*row_index_fn)(const void *ctx, int64_t node);

static void apply_edge(double *Z, int32_t K, const int32_t *Y,
                       const int64_t *nk, int64_t u, int64_t v, double wt,
                       row_index_fn row_index, const void *ctx)
{
    int32_t yu = Y[u], yv = Y[v];
    if (gee_oracle_mutation == 4) {
        if (yu < 0) yu = 0;
        if (yv < 0) yv = 0;
    }
    /* Z(u, Y(v)) += W(v, Y(v)) * w  (skipped when Y(v) is unknown: W row 0) */
    if (yv >= 0) {
        int64_t row = u;
        int32_t cls = yv;
        int64_t div = nk[yv];
        if (gee_oracle_mutation == 2 && yu >= 0)
            cls = yu;
        if (gee_oracle_mutation == 3)
            row = v;
        if (gee_oracle_mutation == 5 && yu >= 0)
            div = nk[yu];
        int64_t r = row_index(ctx, row);
        if (r >= 0 && div > 0)
            Z[r * K + cls] += (1.0 / (double)div) * wt;
    }
    if (gee_oracle_mutation == 1)
        return;
    if (gee_oracle_mutation == 7 && u == v)
        return;
    /* Z(v, Y(u)) += W(u, Y(u)) * w */
    if (yu >= 0) {
        int64_t r = row_index(ctx, v);
        if (r >= 0 && nk[yu] > 0)
            Z[r * K + yu] += (1.0 / (double)nk[yu]) * wt;
    }
}

static int64_t all_rows(const void *ctx, int64_t node)
{
    (void)ctx;
    return node;
}

/*
 * Alg. 1 in FP64: Z (n x K, row-major) from E, optional weights w and labels
 * Y.  With laplacian != 0 the edge weights are first replaced by
 * w / sqrt(d_u d_v) (reading above).
 */
int gee_oracle_embed(const int32_t *E, const float *w, int64_t s,
                     const int32_t *Y, int64_t n, int32_t K, int laplacian,
                     double *Z)
{
    int st = check_inputs(E, w, s, Y, n, K, laplacian);
    if (st != ORC_OK)
        return st;
    if (n > 0 && Z == NULL)
        return ORC_BAD_ARG;
    int64_t *nk = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    double *d = NULL;
    if (nk == NULL)
        return ORC_NO_MEMORY;
    gee_oracle_class_counts(Y, n, K, nk);
    if (laplacian) {
        d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (d == NULL) {
            free(nk);
            return ORC_NO_MEMORY;
        }
        gee_oracle_degrees(E, w, s, n, d);
    }
    memset(Z, 0, sizeof(double) * (size_t)n * (size_t)K);
    for (int64_t i = 0; i < s; ++i) {
        int64_t u = E[2 * i], v = E[2 * i + 1];
        apply_edge(Z, K, Y, nk, u, v, edge_weight(w, i, d, u, v), all_rows,
                   NULL);
    }
    free(d);
    free(nk);
    return ORC_OK;
}

/*
 * Unit-weight form of Alg. 1 with exact integer arithmetic: C[u,k] counts the
 * edge endpoints of class k adjacent to u, so that Z[u,k] = C[u,k] / n_k.
 */
int gee_oracle_counts(const int32_t *E, int64_t s, const int32_t *Y, int64_t n,
                      int32_t K, uint64_t *C)
{
    int st = check_inputs(E, NULL, s, Y, n, K, 0);
    if (st != ORC_OK)
        return st;
    if (n > 0 && C == NULL)
        return ORC_BAD_ARG;
    memset(C, 0, sizeof(uint64_t) * (size_t)n * (size_t)K);
    for (int64_t i = 0; i < s; ++i) {
        int64_t u = E[2 * i], v = E[2 * i + 1];
        int32_t yu = Y[u], yv = Y[v];
        if (yv >= 0)
            C[u * K + yv] += 1;
        if (gee_oracle_mutation == 1)
            continue;
        if (yu >= 0)
            C[v * K + yu] += 1;
    }
    return ORC_OK;
}

/*
 * Z32[u,k] = round-to-nearest float of C[u,k] / n_k.  The quotient is formed
 * in double (correctly rounded) and then rounded to float; for integers below
 * 2^24 this double rounding equals a single correct rounding because
 * 53 >= 2*24 + 2 (Figueroa, "When is double rounding innocuous?", 1995).
 * Empty classes (n_k = 0) have C = 0 and give 0.
 */
int gee_oracle_round_counts(const uint64_t *C, int64_t n, int32_t K,
                            const int64_t *nk, float *Z32)
{
    if (n < 0 || K < 1 || (n > 0 && (C == NULL || Z32 == NULL)) || nk == NULL)
        return ORC_BAD_ARG;
    for (int64_t u = 0; u < n; ++u)
        for (int32_t k = 0; k < K; ++k) {
            uint64_t c = C[u * K + k];
            Z32[u * K + k] =
                (nk[k] > 0) ? (float)((double)c / (double)nk[k]) : 0.0f;
        }
    return ORC_OK;
}

/* Row lookup for the sampled-rows form: a bitmap filter, then binary search. */
typedef struct {
    const int64_t *rows; /* sorted, distinct */
    int64_t nrows;
    const uint8_t *bitmap;
} rows_ctx;

static int64_t sampled_row(const void *ctxp, int64_t node)
{
    const rows_ctx *ctx = (const rows_ctx *)ctxp;
    if (!(ctx->bitmap[node >> 3] & (1u << (node & 7))))
        return -1;
    int64_t lo = 0, hi = ctx->nrows - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ctx->rows[mid] == node)
            return mid;
        if (ctx->rows[mid] < node)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/*
 * The rows `rows` (sorted, distinct node ids) of Alg. 1's Z, for graphs too
 * large for a full n x K FP64 matrix.  Same arithmetic as gee_oracle_embed,
 * restricted to the sampled rows.  Crows (optional, unit weights only) gets
 * the exact integer counts of those rows.
 */
int gee_oracle_embed_rows(const int32_t *E, const float *w, int64_t s,
                          const int32_t *Y, int64_t n, int32_t K,
                          int laplacian, const int64_t *rows, int64_t nrows,
                          double *Zrows, uint64_t *Crows)
{
    int st = check_inputs(E, w, s, Y, n, K, laplacian);
    if (st != ORC_OK)
        return st;
    if (nrows < 0 || (nrows > 0 && (rows == NULL || Zrows == NULL)))
        return ORC_BAD_ARG;
    for (int64_t j = 0; j < nrows; ++j) {
        if (rows[j] < 0 || rows[j] >= n)
            return ORC_BAD_NODE;
        if (j > 0 && rows[j] <= rows[j - 1])
            return ORC_BAD_ARG;
    }
    int64_t *nk = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    uint8_t *bitmap = (uint8_t *)calloc((size_t)(n / 8 + 1), 1);
    double *d = NULL;
    if (nk == NULL || bitmap == NULL) {
        free(nk);
        free(bitmap);
        return ORC_NO_MEMORY;
    }
    gee_oracle_class_counts(Y, n, K, nk);
    if (laplacian) {
        d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (d == NULL) {
            free(nk);
            free(bitmap);
            return ORC_NO_MEMORY;
        }
        gee_oracle_degrees(E, w, s, n, d);
    }
    for (int64_t j = 0; j < nrows; ++j)
        bitmap[rows[j] >> 3] |= (uint8_t)(1u << (rows[j] & 7));
    rows_ctx ctx = {rows, nrows, bitmap};
    memset(Zrows, 0, sizeof(double) * (size_t)nrows * (size_t)K);
    if (Crows != NULL)
        memset(Crows, 0, sizeof(uint64_t) * (size_t)nrows * (size_t)K);
    for (int64_t i = 0; i < s; ++i) {
        int64_t u = E[2 * i], v = E[2 * i + 1];
        int in_u = (bitmap[u >> 3] >> (u & 7)) & 1;
        int in_v = (bitmap[v >> 3] >> (v & 7)) & 1;
        if (!in_u && !in_v)
            continue;
        apply_edge(Zrows, K, Y, nk, u, v, edge_weight(w, i, d, u, v),
                   sampled_row, &ctx);
        if (Crows != NULL) {
            if (in_u && Y[v] >= 0)
                Crows[sampled_row(&ctx, u) * K + Y[v]] += 1;
            if (in_v && Y[u] >= 0)
                Crows[sampled_row(&ctx, v) * K + Y[u]] += 1;
        }
    }
    free(d);
    free(bitmap);
    free(nk);
    return ORC_OK;
}

/*
 * Unsupervised GEE.  Section II notes that Y may come from unsupervised
 * clustering instead of known labels; here the clustering is k-means on the
 * embedding itself (Lloyd, "Least squares quantization in PCM", IEEE Trans.
 * Inf. Theory 1982), alternated with Alg. 1 from the given starting labels:
 * each round embeds the current labels and moves every node to the nearest
 * class mean of that embedding, until a round changes no label or max_iter
 * rounds ran.  Unit weights, every label known (0..K-1).  With
 *   C       integer counts of the current labels (Alg. 1, unit weights)
 *   m_k     class sizes
 *   Z[i,j]  = C[i,j] / m_j                         (FP64, one division)
 *   S[k,j]  = sum of C[i,j] over i of class k      (exact integers)
 *   c[k,j]  = S[k,j] / (m_k * m_j)                 (FP64 product, one division)
 *   d(i,k)  = sum over j = 0..K-1, in that order, of (Z[i,j] - c[k,j])^2
 *             in FP64
 * node i moves to the k with the smallest d(i,k) among classes with
 * m_k > 0, the lowest k on ties.  The paper fixes no precision for the
 * clustering step, so the oracle takes it in FP64, close to the exact
 * rational distances (the tests pin it to them); a faster implementation
 * may take different decisions only where two class means are nearly
 * equally near, which gee_oracle_unsup_round's distances let a test bound.
 * The labels are updated in place in Y; *rounds receives the number of
 * rounds run (the last one changed nothing unless max_iter ended the loop)
 * and changes[r] (if not NULL, length max_iter) the number of nodes round r
 * moved.
 */

/* One assignment step from labels Y (all in 0..K-1) with counts C[n][K]
 * and class sizes m[K] already taken: next[i] = the chosen class,
 * D[i*K + k] (if not NULL) = d(i,k) (0 for empty classes) and T[i*K + k]
 * (if not NULL) = sum over j of (|Z[i,j]| + |c[k,j]|)^2, the scale of the
 * rounding error a finite-precision d(i,k) can carry.  Returns the nodes
 * moved. */
static int64_t unsup_assign(const uint64_t *C, const int64_t *m,
                            const int32_t *Y, int64_t n, int32_t K,
                            uint64_t *S, double *cen, int32_t *next,
                            double *D, double *T)
{
    memset(S, 0, sizeof(uint64_t) * (size_t)K * (size_t)K);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < K; ++j)
            S[(int64_t)Y[i] * K + j] += C[i * K + j];
    for (int32_t k = 0; k < K; ++k)
        for (int32_t j = 0; j < K; ++j) {
            double den = (gee_oracle_mutation == 9)
                             ? (double)m[k]
                             : (double)m[k] * (double)m[j];
            cen[k * K + j] = den > 0.0 ? (double)S[k * K + j] / den : 0.0;
        }
    int64_t moved = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t best = -1;
        double bd = 0.0;
        for (int32_t k = 0; k < K; ++k) {
            double d = 0.0, t = 0.0;
            if (m[k] != 0) {
                for (int32_t j = 0; j < K; ++j) {
                    double z = m[j] > 0
                                   ? (double)C[i * K + j] / (double)m[j]
                                   : 0.0;
                    double c = cen[k * K + j];
                    double diff = z - c;
                    d = d + diff * diff;
                    double a = fabs(z) + fabs(c);
                    t = t + a * a;
                }
                if (best < 0 || d < bd) {
                    best = k;
                    bd = d;
                }
            }
            if (D != NULL)
                D[i * K + k] = d;
            if (T != NULL)
                T[i * K + k] = t;
        }
        next[i] = best;
        moved += (best != Y[i]);
    }
    return moved;
}

/* One round of the loop (embed Y, then one assignment step), with the
 * per-node distances to every class mean: next[n], D[n][K], T[n][K] as in
 * unsup_assign (D and T may be NULL).  Y is not modified. */
int gee_oracle_unsup_round(const int32_t *E, int64_t s, int64_t n, int32_t K,
                           const int32_t *Y, int32_t *next, double *D,
                           double *T)
{
    if (next == NULL && n > 0)
        return ORC_BAD_ARG;
    int st = check_inputs(E, NULL, s, Y, n, K, 0);
    if (st != ORC_OK)
        return st;
    for (int64_t i = 0; i < n; ++i)
        if (Y[i] < 0)
            return ORC_BAD_LABEL;
    uint64_t *C = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    uint64_t *S = malloc(sizeof(uint64_t) * (size_t)K * (size_t)K);
    double *cen = malloc(sizeof(double) * (size_t)K * (size_t)K);
    int64_t *m = malloc(sizeof(int64_t) * (size_t)K);
    if (!C || !S || !cen || !m) {
        free(C); free(S); free(cen); free(m);
        return ORC_NO_MEMORY;
    }
    gee_oracle_counts(E, s, Y, n, K, C);
    gee_oracle_class_counts(Y, n, K, m);
    unsup_assign(C, m, Y, n, K, S, cen, next, D, T);
    free(C); free(S); free(cen); free(m);
    return ORC_OK;
}

int gee_oracle_unsupervised(const int32_t *E, int64_t s, int64_t n, int32_t K,
                            int32_t max_iter, int32_t *Y, int32_t *rounds,
                            int64_t *changes)
{
    if (rounds == NULL || max_iter < 0)
        return ORC_BAD_ARG;
    *rounds = 0;
    int st = check_inputs(E, NULL, s, Y, n, K, 0);
    if (st != ORC_OK)
        return st;
    for (int64_t i = 0; i < n; ++i)
        if (Y[i] < 0)
            return ORC_BAD_LABEL;
    uint64_t *C = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    uint64_t *S = malloc(sizeof(uint64_t) * (size_t)K * (size_t)K);
    double *cen = malloc(sizeof(double) * (size_t)K * (size_t)K);
    int64_t *m = malloc(sizeof(int64_t) * (size_t)K);
    int32_t *next = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!C || !S || !cen || !m || !next) {
        free(C); free(S); free(cen); free(m); free(next);
        return ORC_NO_MEMORY;
    }
    for (int32_t r = 0; r < max_iter; ++r) {
        gee_oracle_counts(E, s, Y, n, K, C);
        gee_oracle_class_counts(Y, n, K, m);
        int64_t moved = unsup_assign(C, m, Y, n, K, S, cen, next, NULL, NULL);
        memcpy(Y, next, sizeof(int32_t) * (size_t)n);
        if (changes != NULL)
            changes[r] = moved;
        *rounds = r + 1;
        if (moved == 0)
            break;
    }
    free(C); free(S); free(cen); free(m); free(next);
    return ORC_OK;
}
